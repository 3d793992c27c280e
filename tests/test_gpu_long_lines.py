"""GPU parity for x and y lines longer than 1024 cells (up to 8192; n/2 = 2^a·3^b).

Lines of n ≤ 1024 run in the register-resident transform kernels. Lines of 2048,
4096 and 8192 run in the one-line-per-CTA kernel; y lines of those lengths are
transposed plane by plane into a scratch array first, stay transposed through the
z solve (whose x and y roles then swap) and are transposed back after the
backward y pass. Other long lengths (1536, …) run in the generic shared-memory
kernel. Checked against the FP64 oracle (dense Table 2 matrices) in FP64, FP32 and
the refined mode, for each BC family including D-N, along x and along y; the
transposed z solve with the singular column, a periodic z, and an FP64 rectangle
of low wavenumbers that is not square.
"""

import numpy as np
import pytest

from oracle import solve as S
from oracle import operator as O
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(lib, f, dx, dy, zf, bcs, precision="fp64", **kw):
    import torch
    nz, ny, nx = f.shape
    plan = lib.Plan(nx, ny, nz, dx, dy, zf=zf, bcs=bcs, precision=precision, **kw)
    dt = torch.float32 if precision == "fp32" else torch.float64
    ft = torch.as_tensor(f, dtype=dt, device="cuda").contiguous()
    info = lib.info_tensor()
    out = plan.solve(ft, info=info)
    torch.cuda.synchronize()
    res = out.double().cpu().numpy(), lib.read_info(info)
    plan.close()
    return res


def _relerr(p, q):
    return np.abs(p - q).max() / max(np.abs(q).max(), 1e-300)


CASES = [((2, 6, 2048), ("P", "NN", "DD")), ((2, 2048, 8), ("DD", "P", "NN")),
         ((3, 4, 1536), ("ND", "DD", "NN")), ((2, 1536, 16), ("NN", "DN", "ND")),
         ((2, 4, 4096), ("DN", "P", "P")), ((2, 4096, 4), ("P", "ND", "DD")),
         ((2, 2, 8192), ("P", "NN", "NN")), ((2, 8192, 2), ("NN", "DD", "DN"))]
IDS = ["x".join(map(str, s)) + "-" + "-".join(b) for s, b in CASES]


@pytest.mark.parametrize("shape,bcs", CASES, ids=IDS)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_long_lines(lib, shape, bcs, precision, tol):
    nz, ny, nx = shape
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    f = np.random.default_rng(nx + ny).uniform(-1, 1, shape)
    p, _ = _run(lib, f, 4.0 / nx, 4.0 / ny, zf, bcs, precision=precision)
    q = S.solve(f, 4.0 / nx, 4.0 / ny, zf, *bcs)
    assert _relerr(p, q) <= tol


REFINE = [((4, 8, 8192), ("P", "P", "NN")), ((4, 8192, 8), ("DD", "NN", "ND")),
          ((3, 2048, 1536), ("P", "DN", "NN"))]


@pytest.mark.parametrize("shape,bcs", REFINE, ids=["x".join(map(str, s)) + "-" + "-".join(b) for s, b in REFINE])
def test_long_lines_refine(lib, shape, bcs):
    nz, ny, nx = shape
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(nx * 3 + ny).uniform(-1, 1, shape)
    lx, ly = 6.0 * nx / 1024, 3.0 * ny / 1024
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs)
    assert info.status == 0 and info.rel_residual <= 1e-10, (info.status, info.rel_residual, rr)
    assert rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)


# y lines of 2048 … 8192: the z solve on transposed planes. Case 1 has a 24 × 31 box, so
# the FP64 rectangle of ill-conditioned columns (|λ| below 10^-4 of the z operator's
# norm) is about 9 × 11 (q_x × q_y), not square, while κ stays near 10^6.
TRANSPOSED = [((4, 2048, 24), ("P", "NN", "NN"), 1.0, 0.015), ((2, 4096, 6), ("NN", "P", "P"), None, None),
              ((3, 2048, 36), ("DD", "NN", "DN"), None, None), ((4, 8192, 16), ("P", "P", "NN"), None, None)]


@pytest.mark.parametrize("shape,bcs,dx,dy", TRANSPOSED,
                         ids=["x".join(map(str, c[0])) + "-" + "-".join(c[1]) for c in TRANSPOSED])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5), ("fp32_refine", 1e-8)])
def test_long_y_z_solve_on_transposed_planes(lib, shape, bcs, dx, dy, precision, tol):
    nz, ny, nx = shape
    dx = dx or 4.0 / nx
    dy = dy or 4.0 / ny
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    f = np.random.default_rng(nx * ny + nz).uniform(-1, 1, shape)
    kw = dict(rtol=1e-10, max_iter=6) if precision == "fp32_refine" else {}
    if precision == "fp32" and bcs == ("P", "NN", "NN"):
        # the FP32 path solves columns of κ up to 10^4 in FP32 (the rest go to the FP64
        # rectangle): its error bound is about κ·ε_32 ≈ 6e-4 on this machine, not 2e-5
        tol = 6e-4
    p, info = _run(lib, f, dx, dy, zf, bcs, precision=precision, **kw)
    q = S.solve(f, dx, dy, zf, *bcs)
    assert _relerr(p, q) <= tol
    if precision == "fp32_refine":
        rr = O.relative_residual(p, f, dx, dy, zf, *bcs)
        assert info.status == 0 and rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)


@pytest.mark.parametrize("bcx", ["DN", "ND"])
def test_long_lines_first_line_of_every_cta(lib, bcx):
    """Eight x lines of 4096, so each CTA of the long-line kernel does one line and every
    line is its CTA's first: the forward gather of the DCT-IV family reads the shared
    twiddle tables right after they are filled. Twenty solves, each against the oracle
    (a missing barrier there gave wrong first lines now and then)."""
    import torch
    shape, bcs = (2, 4, 4096), (bcx, "P", "P")
    zf = synth.uniform_faces(2, 1.0)
    f = np.random.default_rng(11).uniform(-1, 1, shape)
    q = S.solve(f, 4.0 / 4096, 1.0, zf, *bcs)
    plan = lib.Plan(4096, 4, 2, 4.0 / 4096, 1.0, zf=zf, bcs=bcs, precision="fp32")
    ft = torch.as_tensor(f, dtype=torch.float32, device="cuda").contiguous()
    for _ in range(20):
        p = plan.solve(ft).double().cpu().numpy()
        assert _relerr(p, q) <= 2e-5
    plan.close()


@pytest.mark.parametrize("shape,bcs", [((2, 2048, 8), ("DD", "P", "NN")), ((3, 4096, 6), ("P", "NN", "DN"))],
                         ids=["2x2048x8-DD-P-NN", "3x4096x6-P-NN-DN"])
def test_long_y_transpose_solve(lib, shape, bcs):
    """The transpose solve (the projection's backward) with y lines of 2048/4096: the z
    solve runs on transposed planes between the y passes, the Δz weighting in x."""
    import torch
    from oracle import adjoint as AD
    nz, ny, nx = shape
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    g = np.random.default_rng(nx * ny).uniform(-1, 1, shape)
    plan = lib.Plan(nx, ny, nz, 4.0 / nx, 4.0 / ny, zf=zf, bcs=bcs, precision="fp64")
    out = plan.solve_transpose(torch.as_tensor(g, device="cuda").contiguous())
    torch.cuda.synchronize()
    q = AD.solve_transpose(g, 4.0 / nx, 4.0 / ny, zf, *bcs)
    assert _relerr(out.cpu().numpy(), q) <= 1e-12
    plan.close()
