"""GPU parity of the D-N boundary pair (Dirichlet at the low end, Neumann at the
high end; not in Table 1), read as the N-D problem on the reversed axis: the
DCT-IV line transforms with the two reals of each pair swapped on the physical
side, N-D's eigenvalues, the Dirichlet ghost at the low end of the stencils and
of the z system. Every transform kernel family is exercised (the generic one at
small sizes through the all-triples test of test_gpu_solve.py; here the fast,
row and column kernels), in FP64, FP32 and the refined mode (its row kernels
read FP64 input and write FP64 output with the Φ_0 base), plus the transpose
and a Helmholtz plan. Tolerances as for the Table 1 pairs.
"""

import numpy as np
import pytest

from oracle import solve as S
from oracle import operator as O
from oracle import adjoint as AD
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(lib, f, dx, dy, zf, bcs, precision="fp64", transpose=False, **kw):
    import torch
    nz, ny, nx = f.shape
    plan = lib.Plan(nx, ny, nz, dx, dy, zf=zf, bcs=bcs, precision=precision, **kw)
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


# fast kernels (n = 16 … 96 along x), row kernels (n_x = 128 … 1024), column kernels
# (n_y = 128 … 1024 with n_x a multiple of 16), and the small-n generic ones
SHAPES = [(4, 16, 1024), (4, 1024, 16), (3, 128, 256), (2, 512, 128), (2, 256, 512), (5, 48, 96), (6, 24, 36)]
BCXY = [("DN", "DN"), ("DN", "ND"), ("ND", "DN"), ("P", "DN")]


@pytest.mark.parametrize("shape", SHAPES, ids=["x".join(map(str, s)) for s in SHAPES])
@pytest.mark.parametrize("bcxy", BCXY, ids=["-".join(b) for b in BCXY])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_dn_transform_sizes(lib, shape, bcxy, precision, tol):
    nz, ny, nx = shape
    bcs = (bcxy[0], bcxy[1], "DN")
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(nx + 5 * ny).standard_normal(shape)
    p, _ = _run(lib, f, 1.0 / nx, 2.0 / ny, zf, bcs, precision=precision)
    q = S.solve(f, 1.0 / nx, 2.0 / ny, zf, *bcs)
    assert _relerr(p, q) <= tol


REFINE = [((8, 128, 256), ("DN", "DN", "DN")), ((6, 512, 512), ("DN", "P", "NN")),
          ((4, 1024, 512), ("ND", "DN", "DN")), ((5, 512, 1024), ("DN", "ND", "P")),
          ((10, 12, 18), ("DN", "DN", "DN")), ((16, 24, 72), ("DN", "DD", "DN"))]


@pytest.mark.parametrize("shape,bcs", REFINE, ids=["x".join(map(str, s)) + "-" + "-".join(b) for s, b in REFINE])
def test_dn_refine(lib, shape, bcs):
    nz, ny, nx = shape
    lx, ly = 6.0, 3.0
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    f = np.random.default_rng(nx + nz).uniform(-1, 1, shape)
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs)
    assert info.status == 0 and info.rel_residual <= 1e-10, (info.status, info.rel_residual, rr)
    assert rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)
    q = S.solve(f, lx / nx, ly / ny, zf, *bcs)
    assert _relerr(p, q) <= 1e-8


@pytest.mark.parametrize("bcs", [("DN", "NN", "DN"), ("P", "DN", "ND")])
def test_dn_transpose(lib, bcs):
    nz, ny, nx = 10, 12, 16
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    g = np.random.default_rng(41).standard_normal((nz, ny, nx))
    p, _ = _run(lib, g, 0.3, 0.6, zf, bcs, transpose=True)
    q = AD.solve_transpose(g, 0.3, 0.6, zf, *bcs)
    assert _relerr(p, q) <= 1e-12


def test_dn_helmholtz_refine(lib):
    nz, ny, nx = 16, 128, 256
    bcs = ("DN", "P", "DN")
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(42).uniform(-1, 1, (nz, ny, nx))
    p, info = _run(lib, f, 6.0 / nx, 3.0 / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6,
                   alpha=25.0)
    rr = O.relative_residual(p, f, 6.0 / nx, 3.0 / ny, zf, *bcs, alpha=25.0)
    assert info.status == 0 and rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11, (info.status, rr)
