"""Differentiable projection step (Eqs. 2b–2c) on top of the C ABI.

``Projection(...)(ustar)`` returns u = u* − G·solve(D·u*) for a stacked
staggered velocity ``ustar`` of shape (3, n_z, n_y, n_x) (face i of a component
is the face on the low side of cell i; on a Neumann axis face 0 is the wall and
passes through unchanged). Backward applies the hand-written adjoint
ḡ* = ḡ − Dᵀ·solveᵀ(Gᵀ·ḡ), where solveᵀ is the transpose solve
(W·solve(W⁻¹·) with W = diag(Δz^f)). Every step runs in the CUDA library; this
module only allocates the intermediate tensors and passes pointers.
"""

import ctypes

import torch

from . import binding as lib


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


class _ProjectionFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ustar, proj):
        ctx.proj = proj
        return proj.forward(ustar)

    @staticmethod
    def backward(ctx, g):
        return ctx.proj.vjp(g.contiguous()), None


class Projection:
    """u = u* − G·solve(D·u*), differentiable through torch.autograd.

    precision "fp32" (float fields) or "fp64" (double fields). Axes must be
    periodic ("P") or Neumann–Neumann ("NN").
    """

    def __init__(self, nx, ny, nz, dx, dy, zf=None, dz=None, bcs=("P", "P", "NN"), precision="fp32"):
        if precision not in ("fp32", "fp64"):
            raise ValueError("precision must be fp32 or fp64")
        self.plan = lib.Plan(nx, ny, nz, dx, dy, zf=zf, dz=dz, bcs=bcs, precision=precision)
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.shape = (nz, ny, nx)

    def _check(self, u):
        if not (u.is_cuda and u.is_contiguous() and u.dtype == self.dtype and tuple(u.shape) == (3,) + self.shape):
            raise ValueError(f"expected a contiguous CUDA {self.dtype} tensor of shape {(3,) + self.shape}")

    def forward(self, ustar):
        self._check(ustar)
        st = lib._stream_ptr(None)
        f = torch.empty(self.shape, dtype=self.dtype, device=ustar.device)
        lib._check(lib.ps_div(self.plan.handle, _vp(ustar), _vp(f), st), self.plan.handle)
        phi = self.plan.solve(f)
        u = torch.empty_like(ustar)
        lib._check(lib.ps_grad_correct(self.plan.handle, _vp(ustar), _vp(phi), _vp(u), st), self.plan.handle)
        return u

    def vjp(self, g):
        self._check(g)
        st = lib._stream_ptr(None)
        h = torch.empty(self.shape, dtype=self.dtype, device=g.device)
        lib._check(lib.ps_grad_adjoint(self.plan.handle, _vp(g), _vp(h), st), self.plan.handle)
        s = self.plan.solve_transpose(h)
        out = torch.empty_like(g)
        lib._check(lib.ps_div_adjoint_correct(self.plan.handle, _vp(g), _vp(s), _vp(out), st), self.plan.handle)
        return out

    def __call__(self, ustar):
        return _ProjectionFn.apply(ustar, self)

    def close(self):
        self.plan.close()
