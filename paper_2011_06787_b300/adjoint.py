"""Differentiable impulse response of a filter bank (spiir_impulse_forward / _backward).

``impulse_response(a1, b0, s0, delay, n)`` returns u [T][n] (complex64) for coefficient
tensors of shape [T][F].  Its backward pass runs the library's adjoint kernel, which
recomputes the filter states from checkpoints taken every ``ckpt_every`` samples, so memory
grows with n / ckpt_every rather than n.  Gradients follow PyTorch's convention for complex
tensors (dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import ctypes

from . import native
from .native import check


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _impulse_fn():
    import torch

    class IIRImpulse(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a1, b0, s0, delay, n, ckpt_every):
            for x, nm in ((a1, "a1"), (b0, "b0"), (s0, "s0")):
                if x.dtype != torch.complex64 or not x.is_cuda or x.dim() != 2:
                    raise TypeError(f"{nm} must be a [T][F] complex64 CUDA tensor")
            if delay.dtype != torch.int32 or not delay.is_cuda or delay.shape != a1.shape:
                raise TypeError("delay must be an int32 CUDA tensor of the coefficients' shape")
            a1c, b0c, s0c, dc = a1.contiguous(), b0.contiguous(), s0.contiguous(), delay.contiguous()
            T, F = a1c.shape
            u = torch.empty((T, n), dtype=torch.complex64, device=a1.device)
            nck = (n + ckpt_every - 1) // ckpt_every
            ck = torch.empty((nck, T, F), dtype=torch.complex64, device=a1.device)
            check(native.lib().spiir_impulse_forward(T, F, _p(a1c), _p(b0c), _p(dc), _p(s0c), n, _p(u), ckpt_every,
                                                     _p(ck), _stream()))
            ctx.save_for_backward(a1c, b0c, dc, ck)
            ctx.n, ctx.ckpt_every = n, ckpt_every
            return u

        @staticmethod
        def backward(ctx, grad_u):
            a1c, b0c, dc, ck = ctx.saved_tensors
            T, F = a1c.shape
            g = grad_u.contiguous()
            ga = torch.empty_like(a1c)
            gb = torch.empty_like(b0c)
            gs = torch.empty_like(a1c)
            work = torch.empty((ck.shape[0] + 2, T, F), dtype=torch.complex64, device=ck.device)
            check(native.lib().spiir_impulse_backward(T, F, _p(a1c), _p(b0c), _p(dc), ctx.n, _p(g), ctx.ckpt_every,
                                                      _p(ck), _p(ga), _p(gb), _p(gs), _p(work), _stream()))
            return ga, gb, gs, None, None, None

    return IIRImpulse


_FN = None


def impulse_response(a1, b0, s0, delay, n: int, ckpt_every: int = 1024):
    """u_t[k] = sum_l y_l[k], y_l[-1] = s0, y_l[k] = a1 y_l[k-1] + b0 [k == delay]; differentiable
    in a1, b0 and s0."""
    global _FN
    if _FN is None:
        _FN = _impulse_fn()
    return _FN.apply(a1, b0, s0, delay, int(n), int(ckpt_every))


def overlap_loss(h, u):
    """1 - |sum conj(h) u| / (|h| |u|) per template (Sec. II.B.1 Eq. (overlap), modulus form),
    written with torch operations so that autograd supplies dL/du."""
    import torch
    c = torch.sum(torch.conj(h) * u, dim=-1)
    return 1.0 - torch.abs(c) / (torch.linalg.vector_norm(h, dim=-1) * torch.linalg.vector_norm(u, dim=-1))
