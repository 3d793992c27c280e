"""GPU parity of Helmholtz plans, (A − α·I)·p = f (§2: implicit diffusion; §4),
through the C ABI against the FP64 oracle with the same shift.

The shift moves every diagonal of Eq. 5 by −α and adds −α·U to the residual
stencils; with α > 0 no problem is singular (f keeps its mean, p has no mean
constraint). Tolerances as for the Poisson plans: FP64 1e-12·‖p‖∞, FP32 2e-5,
refined solves to a device-measured residual ≤ 1e-10 that equals the oracle's
residual of the returned p within rtol/10.
"""

import numpy as np
import pytest

from oracle import solve as S
from oracle import operator as O
from oracle import adjoint as AD
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(lib, f, dx, dy, zf, bcs, alpha, precision="fp64", transpose=False, **kw):
    import torch
    nz, ny, nx = f.shape
    plan = lib.Plan(nx, ny, nz, dx, dy, zf=zf, bcs=bcs, precision=precision, alpha=alpha, **kw)
    dt = torch.float32 if precision == "fp32" else torch.float64
    ft = torch.as_tensor(f, dtype=dt, device="cuda").contiguous()
    info = lib.info_tensor()
    out = (plan.solve_transpose if transpose else plan.solve)(ft, info=info)
    torch.cuda.synchronize()
    res = out.double().cpu().numpy(), lib.read_info(info)
    plan.close()
    return res


def _relerr(p, q):
    return np.abs(p - q).max() / max(np.abs(q).max(), 1e-300)


def _faces(nz, bcz):
    return synth.tanh_faces(nz, 1.0, 1.5) if bcz != "P" else synth.uniform_faces(nz, 1.0)


# α from weak (below the smallest nonzero |λ|) to dominant (above ‖A‖ on the x/y rows)
CASES = [(("P", "P", "NN"), 0.5), (("NN", "NN", "NN"), 40.0), (("P", "P", "P"), 3e3),
         (("DD", "ND", "P"), 2.0), (("ND", "NN", "DD"), 1e5), (("NN", "P", "ND"), 7.0)]
IDS = ["-".join(b) + f"-a{a:g}" for b, a in CASES]


@pytest.mark.parametrize("bcs,alpha", CASES, ids=IDS)
def test_fp64_helmholtz(lib, bcs, alpha):
    nz, ny, nx = 12, 16, 24
    zf = _faces(nz, bcs[2])
    f = np.random.default_rng(31).uniform(-1, 1, (nz, ny, nx)) + 0.25  # a mean that must survive
    p, _ = _run(lib, f, 1.0 / nx, 2.0 / ny, zf, bcs, alpha)
    q = S.solve(f, 1.0 / nx, 2.0 / ny, zf, *bcs, alpha=alpha)
    assert _relerr(p, q) <= 1e-12


@pytest.mark.parametrize("bcs,alpha", CASES[:4], ids=IDS[:4])
def test_fp32_helmholtz(lib, bcs, alpha):
    nz, ny, nx = 24, 48, 64
    zf = _faces(nz, bcs[2])
    f = np.random.default_rng(32).uniform(-1, 1, (nz, ny, nx)) + 0.25
    p, _ = _run(lib, f, 1.0 / nx, 1.0 / ny, zf, bcs, alpha, precision="fp32")
    q = S.solve(f, 1.0 / nx, 1.0 / ny, zf, *bcs, alpha=alpha)
    assert _relerr(p, q) <= 2e-5


REFINE = [((32, 48, 64), ("P", "P", "NN"), 0.5, 1e-10), ((24, 32, 32), ("DD", "ND", "DD"), 40.0, 1e-10),
          ((16, 24, 24), ("NN", "NN", "NN"), 3.0, 1e-13),   # several corrections
          ((64, 64, 64), ("P", "P", "NN"), 1e4, 1e-10),
          ((6, 512, 512), ("P", "P", "NN"), 2.0, 1e-10),     # M = 256 line kernels
          ((4, 1024, 512), ("DD", "ND", "DD"), 5e3, 1e-10)]  # M = 512 y columns


@pytest.mark.parametrize("shape,bcs,alpha,rtol", REFINE,
                         ids=["x".join(map(str, s)) + "-" + "-".join(b) + f"-a{a:g}-{r:g}" for s, b, a, r in REFINE])
def test_refine_helmholtz(lib, shape, bcs, alpha, rtol):
    nz, ny, nx = shape
    lx, ly = 6.0, 3.0
    zf = _faces(nz, bcs[2])
    f = np.random.default_rng(nx + nz).uniform(-1, 1, shape) + 0.25
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, alpha, precision="fp32_refine", rtol=rtol, max_iter=8)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs, alpha=alpha)
    assert info.status == 0 and info.rel_residual <= rtol, (info.status, info.rel_residual, rr)
    assert rr <= rtol * 1.5 and abs(info.rel_residual - rr) <= rtol / 10, (info.rel_residual, rr)
    q = S.solve(f, lx / nx, ly / ny, zf, *bcs, alpha=alpha)
    assert _relerr(p, q) <= 1e-8


def test_refine_helmholtz_smooth_stiff(lib):
    """A smooth right-hand side on a stretched grid with a weak shift: ‖A‖·max|p| ≫ ‖f‖,
    so pass 0 and the exact pass need their three-level splits (with the −α·U term)."""
    nz, ny, nx = 64, 64, 64
    lx, ly = 6.0, 3.0
    bcs = ("P", "P", "NN")
    zf = _faces(nz, bcs[2])
    _, f = synth.manufactured(nx, ny, lx, ly, zf, bcs)
    alpha = 0.05  # ‖A − α‖∞·max|p|/‖f‖∞ ≈ 9.5e3: both splits take three levels at rtol 1e-10
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, alpha, precision="fp32_refine", rtol=1e-10, max_iter=8)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs, alpha=alpha)
    assert info.status == (0 if rr <= 1e-10 else 5), (info.status, info.rel_residual, rr)
    assert abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)


@pytest.mark.parametrize("bcs,alpha", [(("P", "P", "NN"), 2.0), (("DD", "NN", "ND"), 300.0)])
def test_fp64_helmholtz_transpose(lib, bcs, alpha):
    nz, ny, nx = 10, 12, 16
    zf = _faces(nz, bcs[2])
    g = np.random.default_rng(33).standard_normal((nz, ny, nx))
    p, _ = _run(lib, g, 0.3, 0.6, zf, bcs, alpha, transpose=True)
    q = AD.solve_transpose(g, 0.3, 0.6, zf, *bcs, alpha=alpha)
    assert _relerr(p, q) <= 1e-12


def test_helmholtz_from_host_buffers(lib):
    import torch
    nz, ny, nx = 6, 128, 128
    bcs = ("P", "P", "NN")
    zf = _faces(nz, bcs[2])
    f = np.random.default_rng(34).uniform(-1, 1, (nz, ny, nx))
    plan = lib.Plan(nx, ny, nz, 1.0 / nx, 1.0 / ny, zf=zf, bcs=bcs, precision="fp32_refine",
                    rtol=1e-10, max_iter=6, alpha=12.0)
    fd = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    pd = torch.empty_like(fd)
    fh = torch.as_tensor(f).pin_memory()
    ph = torch.empty_like(fh).pin_memory()
    info = plan.solve_host(fh, ph, fd, pd)
    plan.close()
    rr = O.relative_residual(ph.numpy(), f, 1.0 / nx, 1.0 / ny, zf, *bcs, alpha=12.0)
    assert info.status == 0 and rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11
