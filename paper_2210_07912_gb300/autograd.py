"""torch.autograd.Function wrappers of libile's adjoint kernels (include/ile.h, ile_eval_grad and
ile_integrate_grad).  Argument marshalling only: the forward values come from ile_eval /
ile_integrate and the gradients from the hand-written adjoint kernels; PyTorch supplies device
memory, the stream and the autograd graph.

Q, U and V are passed as autograd leaves so that their gradients can be routed; their VALUES must
be the ones loaded into the context with Context.set_data (the functions do not re-upload them).
Layouts: samples (7, N) float64; Q (K, M, T_ext, 2); U, V (K, M, M, 2) (real, imaginary part of
each entry, every entry an independent variable).
"""
from __future__ import annotations

import torch

from .ile import NDIM, Context


def _bind_stream(ile_ctx: Context, device):
    ile_ctx.set_stream(torch.cuda.current_stream(device))


def _check_leaves(ile_ctx: Context, Q, U, V):
    K, M, T = ile_ctx.shape
    for name, t, shape in (("Q", Q, (K, M, T, 2)), ("U", U, (K, M, M, 2)), ("V", V, (K, M, M, 2))):
        if t is not None and tuple(t.shape) != shape:
            raise ValueError(f"{name} has shape {tuple(t.shape)}, the context holds {shape}")


class LnLt(torch.autograd.Function):
    """lnL_t(n) of every sample (S1-S5); backward = ile_eval_grad."""

    @staticmethod
    def forward(fctx, ile_ctx: Context, samples, Q=None, U=None, V=None):
        if samples.dtype != torch.float64 or samples.dim() != 2 or samples.shape[0] != NDIM:
            raise ValueError("samples must be a float64 (7, N) CUDA tensor")
        _check_leaves(ile_ctx, Q, U, V)
        samples = samples.contiguous()
        _bind_stream(ile_ctx, samples.device)
        out = torch.empty(samples.shape[1], dtype=torch.float64, device=samples.device)
        ile_ctx.eval_device(samples, out)
        ile_ctx.sync()
        fctx.ile = ile_ctx
        fctx.save_for_backward(samples)
        return out

    @staticmethod
    def backward(fctx, g):
        (samples,) = fctx.saved_tensors
        ile_ctx = fctx.ile
        K, M, T = ile_ctx.shape
        need = fctx.needs_input_grad
        dev = samples.device
        gs = torch.empty_like(samples) if need[1] else None
        gQ = torch.empty((K, M, T, 2), dtype=torch.float64, device=dev) if need[2] else None
        gU = torch.empty((K, M, M, 2), dtype=torch.float64, device=dev) if need[3] else None
        gV = torch.empty((K, M, M, 2), dtype=torch.float64, device=dev) if need[4] else None
        if gs is None and gQ is None and gU is None and gV is None:
            return None, None, None, None, None
        _bind_stream(ile_ctx, dev)
        ile_ctx.eval_grad_device(samples, g.contiguous().to(torch.float64), gs, gQ, gU, gV)
        ile_ctx.sync()
        return None, gs, gQ, gU, gV


class LnLMarg(torch.autograd.Function):
    """ln L_marg of Eq. (eq:lnL:MonteCarlo) (0-d tensor); backward = ile_integrate_grad.
    ln_prior and ln_ps are constants of the integral (no gradient)."""

    @staticmethod
    def forward(fctx, ile_ctx: Context, samples, ln_prior=None, ln_ps=None, Q=None, U=None, V=None):
        if samples.dtype != torch.float64 or samples.dim() != 2 or samples.shape[0] != NDIM:
            raise ValueError("samples must be a float64 (7, N) CUDA tensor")
        _check_leaves(ile_ctx, Q, U, V)
        samples = samples.contiguous()
        lp = None if ln_prior is None else ln_prior.contiguous()
        lps = None if ln_ps is None else ln_ps.contiguous()
        _bind_stream(ile_ctx, samples.device)
        res = torch.empty(8, dtype=torch.float64, device=samples.device)
        ile_ctx.integrate_device(samples, res, lp, lps)
        ile_ctx.sync()
        fctx.ile = ile_ctx
        fctx.lp, fctx.lps = lp, lps
        fctx.save_for_backward(samples)
        return res[0].clone()

    @staticmethod
    def backward(fctx, g):
        (samples,) = fctx.saved_tensors
        ile_ctx = fctx.ile
        K, M, T = ile_ctx.shape
        need = fctx.needs_input_grad
        dev = samples.device
        gs = torch.empty_like(samples) if need[1] else None
        gQ = torch.empty((K, M, T, 2), dtype=torch.float64, device=dev) if need[4] else None
        gU = torch.empty((K, M, M, 2), dtype=torch.float64, device=dev) if need[5] else None
        gV = torch.empty((K, M, M, 2), dtype=torch.float64, device=dev) if need[6] else None
        if gs is None and gQ is None and gU is None and gV is None:
            return (None,) * 7
        _bind_stream(ile_ctx, dev)
        res = torch.empty(8, dtype=torch.float64, device=dev)
        scale = g.detach().to(torch.float64).reshape(1).contiguous()
        ile_ctx.integrate_grad_device(samples, res, scale, fctx.lp, fctx.lps, gs, gQ, gU, gV)
        ile_ctx.sync()
        return None, gs, None, None, gQ, gU, gV


def lnL_t(ile_ctx: Context, samples, Q=None, U=None, V=None):
    return LnLt.apply(ile_ctx, samples, Q, U, V)


def lnL_marg(ile_ctx: Context, samples, ln_prior=None, ln_ps=None, Q=None, U=None, V=None):
    return LnLMarg.apply(ile_ctx, samples, ln_prior, ln_ps, Q, U, V)
