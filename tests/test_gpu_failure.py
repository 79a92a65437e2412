"""Failure detection without a GPU fault (needs a GB300): a bounded device-side wait that nothing
satisfies gives up and reports ILE_E_TIMEOUT, and a context whose memory cap is exhausted reports
ILE_E_NOMEM before allocating; in both cases the context stays usable and its results unchanged."""
import time

import numpy as np
import pytest

from paper_2210_07912_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ile():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_07912_gb300 import ile as I
    I.load()
    return I


def test_bounded_wait_gives_up_and_context_survives(ile):
    point = S.workload_point(S.SMALL)
    th = S.workload_samples(S.SMALL, 2000)
    ctx = ile.Context(0, None, "bf16x3")
    ctx.set_data(point)
    before = ctx.eval(th)
    t0 = time.perf_counter()
    with pytest.raises(ile.IleError) as e:
        ctx.check_wait_timeout(0.05)
    assert e.value.status == ile.ILE_E_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    # the flag was consumed with the status: the next calls succeed and agree bit for bit
    np.testing.assert_array_equal(ctx.eval(th), before)
    res = ctx.adapt_run(ile.make_adapt_cfg(seed=3, n_per_iter=4096, n_iter=2))
    assert np.isfinite(res["ln_L"])
    for bad in (0.0, -1.0, 11.0, float("nan")):
        with pytest.raises(ile.IleError) as e:
            ctx.check_wait_timeout(bad)
        assert e.value.status == ile.ILE_E_ARG


def test_memory_cap_refuses_before_allocating(ile):
    point = S.workload_point(S.FULL)
    th = S.workload_samples(S.FULL, 1 << 16)
    ctx = ile.Context(0, None, "bf16x3")
    ctx.set_data(point)
    held = ctx.memory_used()
    assert held > 0
    ctx.set_memory_limit(held + 4096)  # far below what 2^16 samples need
    with pytest.raises(ile.IleError) as e:
        ctx.eval(th)
    assert e.value.status == ile.ILE_E_NOMEM
    assert ctx.memory_used() <= held + 4096
    with pytest.raises(ile.IleError) as e:
        ctx.adapt_run(ile.make_adapt_cfg(seed=1, n_per_iter=1 << 16))
    assert e.value.status == ile.ILE_E_NOMEM
    # lifting the cap: the same call succeeds, and matches a context that never had one
    ctx.set_memory_limit(0)
    got = ctx.eval(th)
    ref = ile.Context(0, None, "bf16x3")
    ref.set_data(point)
    np.testing.assert_array_equal(got, ref.eval(th))
    assert ctx.memory_used() > held
