"""Q, U, V of Eq. (eq:QUV) built on the device (ile_build_quv) against the FP64 oracle, and the
likelihood of a point built that way (needs a GB300)."""
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


def _modes_psd_data(seed, K=3, M=5, L=4096, fs=4096.0):
    """Synthetic mode waveforms (band-limited, two-sided, FFT order), coloured PSDs, and data =
    a random combination of the modes, shifted in time per detector, plus white noise."""
    rng = np.random.default_rng(seed)
    df = fs / L
    f = np.fft.fftfreq(L, 1.0 / fs)
    env = np.exp(-0.5 * (f / 250.0) ** 2) * (np.abs(f) > 15.0)
    hf = (rng.normal(size=(M, L)) + 1j * rng.normal(size=(M, L))) * env
    psd = 1.0 + (np.abs(f)[None, :] / 300.0) ** 2 + rng.uniform(0.2, 1.0, (K, 1))
    shifts = rng.uniform(-0.01, 0.01, K)
    coef = rng.normal(size=(K, M)) + 1j * rng.normal(size=(K, M))
    d = np.array([(coef[k] @ hf) * np.exp(-2j * np.pi * f * shifts[k]) for k in range(K)])
    d += (rng.normal(size=(K, L)) + 1j * rng.normal(size=(K, L))) * np.sqrt(psd / (2 * df))
    return hf, psd, d, df, fs


def test_build_quv_matches_oracle(ile, orc):
    hf, psd, d, df, fs = _modes_psd_data(3)
    ctx = ile.Context(0, None, "fp32")
    T_ext, t_start = 300, -150 / fs
    Q, U, V = ctx.build_quv(hf, psd, d, df, 20.0, t_start, fs, T_ext)
    Qr, Ur, Vr = orc.quv_from_modes(hf, psd, d, df, 20.0, t_start, fs, T_ext)
    for name, got, ref in (("Q", Q, Qr), ("U", U, Ur), ("V", V, Vr)):
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() < 1e-10 * scale, name


def test_point_from_built_quv_likelihood(ile, orc):
    """A 21-mode, three-detector point whose Q/U/V come from ile_build_quv: the device likelihood
    of the loaded point equals the oracle's on the oracle-built arrays."""
    K, M, Nt = 3, 21, 128
    hf, psd, d, df, fs = _modes_psd_data(5, K=K, M=M, L=2048)
    tens, pos = S.detector_arrays(K)
    T_ext = S.t_ext_for(Nt, pos, fs)
    t_start = -(T_ext // 2) / fs
    ctx = ile.Context(0, None, "bf16x3")
    Q, U, V = ctx.build_quv(hf, psd, d, df, 15.0, t_start, fs, T_ext)
    Qr, Ur, Vr = orc.quv_from_modes(hf, psd, d, df, 15.0, t_start, fs, T_ext)
    lm = np.array(S.mode_list(M), np.int32)
    mk = lambda Q_, U_, V_: S.Point(lm=lm, det_tensor=tens, det_pos=pos, Q=Q_, U=U_, V=V_, t_start=t_start, fs=fs,
                                    n_window=Nt)
    ctx.set_data(mk(Q, U, V))
    th = S.prior_samples(np.random.default_rng(6), 500)
    got = ctx.eval(th)
    ref = orc.lnL_t(mk(Qr, Ur, Vr), th)
    # |lnL_t| reaches ~750 here: the loud samples go through the FP64 refinement, so the absolute
    # bar of the path applies as it stands
    assert np.abs(ref).max() > 100.0
    assert np.abs(got - ref).max() < 1e-3


def test_build_quv_errors(ile):
    ctx = ile.Context(0, None, "fp32")
    hf, psd, d, df, fs = _modes_psd_data(1, K=1, M=2, L=64)
    with pytest.raises(ile.IleError) as e:
        ctx.build_quv(hf, psd, d, -1.0, 0.0, 0.0, fs, 10)
    assert e.value.status == ile.ILE_E_ARG
