"""Differentiable Helmholtz solve for PyTorch (adjoint state; not in the paper).

``HzSolve.apply(m, f, context, checkpoint)`` returns u = H(m)^{-1} f from a factored
context built for the squared slowness m (``device_ptrs=True``; the tensors
are contiguous complex128 CUDA tensors).  Its backward calls ``hz_adjoint``:
one transposed solve with the forward factors (the row-scaled operator is
complex symmetric) and a pointwise kernel give

    dL/dm_i = omega^2 sum_s Re(mu_{s,i} u_{s,i}),   mu = H^{-T} conj(dL/du),
    dL/df   = conj(mu),

with PyTorch's gradient convention dL/du = dL/dRe(u) + i dL/dIm(u).  PyTorch
only carries the tensors; every step runs in libhz.

``checkpoint=True`` keeps only the interface traces of the forward fields
(``hz_traces``: 2(L-1) rows of every field instead of the whole volume) and
recomputes the fields from their sources and traces in the backward pass
(``hz_reconstruct``: local solves and the reconstruction stage, no GMRES).
"""
from __future__ import annotations

import torch

from . import hz


class HzSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, f, context, checkpoint=False):
        if not context.device:
            raise ValueError("HzSolve needs a context created with device_ptrs=True")
        f = f.contiguous()
        u, _ = context.hz_solve(f)
        ctx.context = context
        ctx.checkpoint = bool(checkpoint)
        if ctx.checkpoint:
            ctx.save_for_backward(f.detach(), context.hz_traces(u))
        else:
            ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, gu):
        if ctx.checkpoint:
            f, tr = ctx.saved_tensors
            u = ctx.context.hz_reconstruct(f, tr)
        else:
            (u,) = ctx.saved_tensors
        grad_m, grad_f, _ = ctx.context.hz_adjoint(u, gu.contiguous(), want_grad_f=ctx.needs_input_grad[1])
        return (grad_m if ctx.needs_input_grad[0] else None), (grad_f if ctx.needs_input_grad[1] else None), None, None


def helmholtz_solve(m, f, context, checkpoint=False):
    """u = H(m)^{-1} f, differentiable in m and f (see HzSolve)."""
    return HzSolve.apply(m, f, context, checkpoint)


class HelmholtzOperator:
    """Owns a factored context for one medium and frequency and refactors it
    when the medium tensor changes (compared by value)."""

    def __init__(self, m, n_x, n_z, omega, h, n_pml, L, C, checkpoint=False, **opts):
        self.args = (n_x, n_z, omega, h, n_pml, L, C)
        self.checkpoint = checkpoint
        self.opts = dict(opts)
        self.opts["device_ptrs"] = True
        self._m = None
        self.context = None
        self._refactor(m)

    def _refactor(self, m):
        if self.context is not None:
            self.context.close()
        mm = m.detach().to("cpu", torch.float64).contiguous().numpy()
        n_x, n_z, omega, h, n_pml, L, C = self.args
        self.context = hz.Context(mm, n_x, n_z, omega, h, n_pml, L, C, **self.opts)
        self.context.hz_factor()
        self._m = m.detach().clone()

    def __call__(self, m, f):
        if self._m is None or self._m.shape != m.shape or not torch.equal(self._m.to(m.device), m.detach()):
            self._refactor(m)
        return HzSolve.apply(m, f, self.context, self.checkpoint)

    def close(self):
        if self.context is not None:
            self.context.close()
            self.context = None
