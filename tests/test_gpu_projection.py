"""GPU parity of the differentiable projection (Eqs. 2b–2c) and its adjoint.

* 16³ subcase (P/P/NN, tanh z 1.5): forward and vector–Jacobian product against
  the FP64 oracle (explicit sparse D, G and their transposes): 1e-12 for the
  FP64 plan, 1e-4 relative for the FP32 plan.
* torch.autograd.gradcheck of the FP64 path on a small grid.
* central finite differences of a scalar loss along a random direction.
* 512×256×256 FP32 (the channel-like size): divergence of the projected field
  (measured with plain torch ops, independent of the library) and the
  dot-product test ⟨P u, g⟩ = ⟨u, Pᵀ g⟩.
"""

import numpy as np
import pytest

from oracle import adjoint as AD
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu

BCS = ("P", "P", "NN")


def _field(nx, ny, nz, seed):
    u = np.random.default_rng(seed).standard_normal((3, nz, ny, nx))
    u[2, 0] = 0.0   # wall face of w
    return u


@pytest.fixture(scope="module")
def projmod(lib):
    from paper_1802_10323_gb300 import autograd
    return autograd


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_projection_and_vjp_vs_oracle_16(projmod, precision, tol):
    import torch
    n = 16
    zf = synth.tanh_faces(n, 1.0, 1.5)
    dx, dy = 6.0 / n, 3.0 / n
    P = projmod.Projection(n, n, n, dx, dy, zf=zf, bcs=BCS, precision=precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    u = _field(n, n, n, 1)
    g = np.random.default_rng(2).standard_normal(u.shape)
    ut = torch.as_tensor(u, dtype=dt, device="cuda").contiguous().requires_grad_(True)
    out = P(ut)
    out.backward(torch.as_tensor(g, dtype=dt, device="cuda"))
    torch.cuda.synchronize()
    ref = AD.project(u, dx, dy, zf, *BCS)
    refg = AD.project_vjp(g, dx, dy, zf, *BCS)
    e1 = np.abs(out.detach().double().cpu().numpy() - ref).max() / np.abs(ref).max()
    e2 = np.abs(ut.grad.double().cpu().numpy() - refg).max() / np.abs(refg).max()
    assert e1 <= tol, e1
    assert e2 <= tol, e2
    P.close()


def test_gradcheck_fp64(projmod):
    import torch
    nx, ny, nz = 8, 4, 6
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    P = projmod.Projection(nx, ny, nz, 0.3, 0.5, zf=zf, bcs=BCS, precision="fp64")
    u = torch.as_tensor(_field(nx, ny, nz, 3), device="cuda").contiguous().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: P(x), (u,), eps=1e-6, atol=1e-7, rtol=1e-6)
    P.close()


def test_central_differences_fp64_16(projmod):
    import torch
    n = 16
    zf = synth.tanh_faces(n, 1.0, 1.5)
    P = projmod.Projection(n, n, n, 6.0 / n, 3.0 / n, zf=zf, bcs=BCS, precision="fp64")
    rng = np.random.default_rng(4)
    u = torch.as_tensor(_field(n, n, n, 5), device="cuda").contiguous()
    w = torch.as_tensor(rng.standard_normal(u.shape), device="cuda")
    d = torch.as_tensor(_field(n, n, n, 6), device="cuda").contiguous()
    ug = u.clone().requires_grad_(True)
    (P(ug) * w).sum().backward()
    h = 1e-6
    fd = ((P(u + h * d) * w).sum() - (P(u - h * d) * w).sum()).item() / (2 * h)
    an = (ug.grad * d).sum().item()
    assert abs(fd - an) <= 1e-6 * abs(an)
    P.close()


def _torch_div(u, dx, dy, zf):
    """Cell divergence with plain torch ops (P, P, NN walls), FP64."""
    import torch
    dzf = torch.as_tensor(np.diff(zf), device=u.device, dtype=torch.float64)
    ux, uy, uz = u[0].double(), u[1].double(), u[2].double()
    f = (torch.roll(ux, -1, 2) - ux) / dx + (torch.roll(uy, -1, 1) - uy) / dy
    hi = torch.zeros_like(uz)
    hi[:-1] = uz[1:]
    lo = uz.clone()
    lo[0] = 0.0
    return f + (hi - lo) / dzf[:, None, None]


def test_projection_full_size_fp32(projmod):
    """512×256×256 channel-like box, FP32: divergence-free and adjoint-consistent."""
    import torch
    nx, ny, nz = 512, 256, 256
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    dx, dy = 6.0 / nx, 3.0 / ny
    P = projmod.Projection(nx, ny, nz, dx, dy, zf=zf, bcs=BCS, precision="fp32")
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    u = torch.randn((3, nz, ny, nx), generator=g, device="cuda", dtype=torch.float32)
    u[2, 0] = 0
    pu = P(u)
    div0 = _torch_div(u, dx, dy, zf).abs().max().item()
    div1 = _torch_div(pu, dx, dy, zf).abs().max().item()
    assert div1 <= 1e-4 * div0, (div0, div1)
    gg = torch.randn(u.shape, generator=g, device="cuda", dtype=torch.float32)
    ptg = P.vjp(gg)
    lhs = (pu.double() * gg.double()).sum().item()
    rhs = (u.double() * ptg.double()).sum().item()
    assert abs(lhs - rhs) <= 1e-4 * (pu.double().norm() * gg.double().norm()).item()
    P.close()
