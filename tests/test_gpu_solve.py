"""GPU parity: the CUDA solve (through the C ABI) against the FP64 oracle.

Tolerances: the FP64 path must match the oracle to 1e-12·‖p‖∞ (the eigen-
expansion reaches the exact discrete solution up to rounding, §1); the FP32
path to 2e-5·‖p‖∞ (FP32 rounding through log n FFT stages and a Thomas sweep
on columns whose condition grows like (n·Δ/Δz_min)²); the refined path to a
device-measured and oracle-checked relative residual ≤ 1e-10.
"""

import itertools

import numpy as np
import pytest

from oracle import solve as S
from oracle import operator as O
from oracle import adjoint as AD
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu

BCS = ("P", "NN", "DD", "ND", "DN")  # DN: not in Table 1, the reversed ND axis


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


ALL = list(itertools.product(BCS, repeat=3))


@pytest.mark.parametrize("bcs", ALL, ids=["-".join(b) for b in ALL])
def test_fp64_all_bc_triples(lib, bcs):
    nx, ny, nz = 12, 8, 10
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    f = np.random.default_rng(1).uniform(-1, 1, (nz, ny, nx))
    p, info = _run(lib, f, 0.3, 0.45, zf, bcs)
    q = S.solve(f, 0.3, 0.45, zf, *bcs)
    assert info.status == 0
    assert _relerr(p, q) <= 1e-12


def test_fp64_small_channel_32_cubed(lib):
    """32³ unit cube, P/P/NN uniform, U[−1,1] mean removed."""
    n = 32
    f = synth.uniform_noise((n, n, n), seed=0)
    zf = synth.uniform_faces(n, 1.0)
    p, _ = _run(lib, f, 1.0 / n, 1.0 / n, zf, ("P", "P", "NN"))
    q = S.solve(f, 1.0 / n, 1.0 / n, zf, "P", "P", "NN")
    assert _relerr(p, q) <= 1e-12
    assert O.relative_residual(p, f, 1.0 / n, 1.0 / n, zf, "P", "P", "NN") <= 1e-12


@pytest.mark.parametrize("shape", [(2, 2, 2), (6, 4, 2), (4, 96, 48), (3, 2, 1024), (5, 1024, 2),
                                   (8, 24, 192), (2, 64, 6)])
@pytest.mark.parametrize("bcs", [("P", "NN", "DD"), ("ND", "P", "NN"), ("DD", "ND", "P")])
def test_fp64_ragged_and_extreme_sizes(lib, shape, bcs):
    nz, ny, nx = shape
    zf = synth.tanh_faces(nz, 2.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 2.0)
    f = np.random.default_rng(nz * 7 + nx).standard_normal(shape)
    p, _ = _run(lib, f, 1.0 / nx, 3.0 / ny, zf, bcs)
    q = S.solve(f, 1.0 / nx, 3.0 / ny, zf, *bcs)
    assert _relerr(p, q) <= 1e-12


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("NN", "DD", "ND"), ("ND", "ND", "P"), ("DD", "P", "DD")])
def test_fp32_parity(lib, bcs):
    nz, ny, nx = 24, 48, 64
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    f = np.random.default_rng(5).uniform(-1, 1, (nz, ny, nx))
    p, _ = _run(lib, f, 1.0 / nx, 1.0 / ny, zf, bcs, precision="fp32")
    q = S.solve(f, 1.0 / nx, 1.0 / ny, zf, *bcs)
    assert _relerr(p, q) <= 2e-5


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("NN", "NN", "NN"), ("DD", "ND", "DD"), ("P", "DD", "P")])
def test_refine_reaches_1e10(lib, bcs):
    nz, ny, nx = 32, 48, 64
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    f = np.random.default_rng(6).uniform(-1, 1, (nz, ny, nx))
    p, info = _run(lib, f, 6.0 / nx, 3.0 / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6)
    assert info.status == 0, (info.status, info.rel_residual)
    assert info.rel_residual <= 1e-10
    rr = O.relative_residual(p, f, 6.0 / nx, 3.0 / ny, zf, *bcs)
    assert rr <= 1e-10
    q = S.solve(f, 6.0 / nx, 3.0 / ny, zf, *bcs)
    assert _relerr(p, q) <= 1e-8


def test_refine_not_converged_is_reported(lib):
    nz, ny, nx = 16, 16, 16
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(8).uniform(-1, 1, (nz, ny, nx))
    _, info = _run(lib, f, 1.0 / nx, 1.0 / ny, zf, ("P", "P", "NN"), precision="fp32_refine",
                   rtol=1e-30, max_iter=1)
    assert info.status == 5 and info.iterations == 1
    _, info = _run(lib, f, 1.0 / nx, 1.0 / ny, zf, ("P", "P", "NN"), precision="fp32_refine",
                   rtol=1e-10, max_iter=0)
    assert info.status == 5 and info.iterations == 0


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("DD", "NN", "ND"), ("NN", "NN", "NN")])
def test_fp64_transpose(lib, bcs):
    nz, ny, nx = 16, 12, 8
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    g = np.random.default_rng(9).standard_normal((nz, ny, nx))
    p, _ = _run(lib, g, 0.2, 0.3, zf, bcs, transpose=True)
    q = AD.solve_transpose(g, 0.2, 0.3, zf, *bcs)
    assert _relerr(p, q) <= 1e-12


def test_fp64_in_place(lib):
    import torch
    nz, ny, nx = 8, 16, 32
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(10).standard_normal((nz, ny, nx))
    plan = lib.Plan(nx, ny, nz, 0.1, 0.1, zf=zf, bcs=("DD", "P", "NN"))
    t = torch.as_tensor(f, device="cuda").contiguous()
    plan.solve(t, out=t)
    torch.cuda.synchronize()
    q = S.solve(f, 0.1, 0.1, zf, "DD", "P", "NN")
    assert _relerr(t.cpu().numpy(), q) <= 1e-12
    plan.close()


FAST = [(4, 16, 1024), (4, 1024, 16), (3, 128, 256), (2, 512, 128), (2, 256, 512)]


@pytest.mark.parametrize("shape", FAST, ids=[f"{s[0]}x{s[1]}x{s[2]}" for s in FAST])
@pytest.mark.parametrize("bcxy", [("P", "NN"), ("NN", "DD"), ("DD", "ND"), ("ND", "P")])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_register_resident_transform_sizes(lib, shape, bcxy, precision, tol):
    """Line lengths 128…1024 along x and y (the register-resident kernels)."""
    nz, ny, nx = shape
    bcs = (bcxy[0], bcxy[1], "NN")
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(nx + 3 * ny).standard_normal(shape)
    p, _ = _run(lib, f, 1.0 / nx, 2.0 / ny, zf, bcs, precision=precision)
    q = S.solve(f, 1.0 / nx, 2.0 / ny, zf, *bcs)
    assert _relerr(p, q) <= tol


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("DD", "ND", "DD")])
def test_refine_register_resident_sizes(lib, bcs):
    nz, ny, nx = 8, 128, 256
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(11).uniform(-1, 1, (nz, ny, nx))
    p, info = _run(lib, f, 6.0 / nx, 3.0 / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6)
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert O.relative_residual(p, f, 6.0 / nx, 3.0 / ny, zf, *bcs) <= 1e-10


# Refinement on sizes that reach the scalar-copy path of the later residual
# passes (n_x not a multiple of 4), a ragged last x tile under the 16-byte copies
# (n_x = 72), and two rows per thread (n_y < 32); Dirichlet ends on every axis.
ODD = [(10, 12, 18), (12, 24, 54), (16, 24, 72), (6, 36, 6)]


@pytest.mark.parametrize("shape", ODD, ids=["x".join(map(str, s)) for s in ODD])
@pytest.mark.parametrize("bcs", [("DD", "DD", "DD"), ("ND", "P", "NN"), ("P", "ND", "DD")])
def test_refine_unaligned_and_ragged_sizes(lib, shape, bcs):
    nz, ny, nx = shape
    lx, ly = 2.0, 3.0
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(nx * 5 + ny).uniform(-1, 1, shape)
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6)
    assert info.status == 0 and info.rel_residual <= 1e-10, (info.status, info.rel_residual)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs)
    assert rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)
    q = S.solve(f, lx / nx, ly / ny, zf, *bcs)
    assert _relerr(p, q) <= 1e-8


@pytest.mark.parametrize("shape,bcs", [((16, 24, 24), ("P", "P", "NN")), ((12, 16, 18), ("DD", "NN", "ND"))])
def test_refine_several_corrections(lib, shape, bcs):
    """A tolerance near the FP64 floor takes more than one correction, so the stored
    residuals of the later passes (the output repeats) feed the next corrections."""
    nz, ny, nx = shape
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(13).uniform(-1, 1, shape)
    p, info = _run(lib, f, 1.0 / nx, 1.0 / ny, zf, bcs, precision="fp32_refine", rtol=1e-13, max_iter=8)
    rr = O.relative_residual(p, f, 1.0 / nx, 1.0 / ny, zf, *bcs)
    assert info.iterations >= 2, info.iterations
    assert info.status == 0 and info.rel_residual <= 1e-13, (info.status, info.rel_residual, rr)
    assert rr <= 1.5e-13 and abs(info.rel_residual - rr) <= 2e-14, (info.rel_residual, rr)


# Refinement with the line lengths of the 1024^3 workload's kernels (n_x, n_y ∈
# {512, 1024}: the M = 256 and M = 512 row and column transforms), few planes.
LONG = [((6, 512, 512), ("P", "P", "NN")), ((4, 1024, 512), ("DD", "ND", "DD")),
        ((5, 512, 1024), ("NN", "P", "P"))]


@pytest.mark.parametrize("shape,bcs", LONG, ids=["x".join(map(str, s)) + "-" + "-".join(b) for s, b in LONG])
def test_refine_long_lines(lib, shape, bcs):
    nz, ny, nx = shape
    lx, ly = 6.0, 3.0
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    f = np.random.default_rng(nx + nz).uniform(-1, 1, shape)
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6)
    assert info.status == 0 and info.rel_residual <= 1e-10, (info.status, info.rel_residual)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs)
    assert rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)
    q = S.solve(f, lx / nx, ly / ny, zf, *bcs)
    assert _relerr(p, q) <= 1e-8


HOST = [((12, 24, 32), "fp64", 1e-10, 6), ((12, 24, 32), "fp32_refine", 1e-10, 6),
        ((6, 128, 128), "fp32_refine", 1e-10, 6),   # copies overlapped with the first/last passes
        ((6, 128, 128), "fp32_refine", 1e-10, 0),   # loop ends at pass 0: p copied again
        ((6, 128, 128), "fp32_refine", 1e-13, 8)]   # several corrections: p copied again


@pytest.mark.parametrize("shape,precision,rtol,max_iter", HOST,
                         ids=[f"{'x'.join(map(str, s))}-{p}-{r:g}-{m}" for s, p, r, m in HOST])
def test_solve_from_host_buffers(lib, shape, precision, rtol, max_iter):
    """ps_solve_host: the copies in and out inside the call (overlapped with the first and
    last passes for refinement with the register-resident kernels), the same bits and
    the same status as the device-buffer call, and the oracle's solution."""
    import torch
    nz, ny, nx = shape
    bcs = ("P", "NN", "DD")
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(21).uniform(-1, 1, shape)
    plan = lib.Plan(nx, ny, nz, 1.0 / nx, 1.0 / ny, zf=zf, bcs=bcs, precision=precision,
                    rtol=rtol, max_iter=max_iter)
    fh = torch.from_numpy(f.copy()).pin_memory()
    ph = torch.zeros_like(fh).pin_memory()
    fd = torch.empty(shape, dtype=torch.float64, device="cuda")
    pd = torch.empty_like(fd)
    info_h = plan.solve_host(fh, ph, fd, pd)
    info = lib.info_tensor()
    p_dev = plan.solve(torch.as_tensor(f, device="cuda").contiguous(), info=info)
    torch.cuda.synchronize()
    info_d = lib.read_info(info)
    plan.close()
    assert (info_h.status, info_h.iterations) == (info_d.status, info_d.iterations)
    assert np.array_equal(ph.numpy(), p_dev.cpu().numpy())
    if max_iter == 0:
        assert info_h.iterations == 0
    if rtol < 1e-12:
        assert info_h.iterations >= 2
    q = S.solve(f, 1.0 / nx, 1.0 / ny, zf, *bcs)
    assert _relerr(ph.numpy(), q) <= (1e-12 if precision == "fp64" else (1e-5 if max_iter == 0 else 1e-8))


REPORTED = [
    ("rough", (32, 48, 64), ("P", "P", "NN")),
    ("rough", (24, 32, 32), ("DD", "ND", "DD")),
    ("smooth", (64, 64, 64), ("P", "P", "NN")),
    ("smooth", (128, 96, 128), ("NN", "P", "NN")),
    ("smooth", (48, 64, 64), ("DD", "NN", "ND")),
]


@pytest.mark.parametrize("kind,shape,bcs", REPORTED, ids=[f"{k}-{'x'.join(map(str, s))}-{'-'.join(b)}"
                                                          for k, s, b in REPORTED])
def test_refine_reported_residual_is_the_solution_residual(lib, kind, shape, bcs):
    """The loop's residuals are incremental (r_m = r_{m−1} − A·e); the reported one
    must still be the residual of the returned FP64 p, within a tenth of rtol —
    for rough right-hand sides (no confirmation pass needed) and for smooth ones
    on stretched grids, where the FP64 rounding of p += e is amplified by ‖A‖ and
    the exact confirmation pass decides."""
    nz, ny, nx = shape
    lx, ly = 6.0, 3.0
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    if kind == "rough":
        f = np.random.default_rng(nx + ny).uniform(-1, 1, (nz, ny, nx))
    else:
        _, f = synth.manufactured(nx, ny, lx, ly, zf, bcs)
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs)
    assert info.status == (0 if rr <= 1e-10 else 5), (info.status, info.rel_residual, rr)
    assert abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)


# Long z columns (n_z from 64 to 1040) for the FP32 z solve: ragged last chunks of
# the checkpointed elimination (n_z not a multiple of 16), column counts that leave a
# partial CTA, and the FP64 low-wavenumber rectangle solved beside the FP32 columns.
# The domain is narrow in x and y (0.05 × 0.05 × 1) so that every column with
# κ > 10^4 lies in the FP64 rectangle (with few columns on a wide domain nearly all
# would, and the rectangle is capped at 1/8 of them).
ZPART = [((64, 24, 32), ("P", "P", "NN")), ((65, 12, 6), ("DD", "NN", "DD")),
         ((200, 16, 24), ("NN", "DD", "ND")), ((1040, 8, 6), ("P", "NN", "NN")),
         ((1024, 12, 6), ("ND", "P", "DD")), ((1023, 8, 12), ("NN", "NN", "ND"))]


@pytest.mark.parametrize("shape,bcs", ZPART, ids=["x".join(map(str, s)) + "-" + "-".join(b) for s, b in ZPART])
def test_fp32_and_refine_long_z_columns(lib, shape, bcs):
    nz, ny, nx = shape
    lx, ly = 0.05, 0.05
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(nz + nx).uniform(-1, 1, shape)
    q = S.solve(f, lx / nx, ly / ny, zf, *bcs)
    p32, _ = _run(lib, f, lx / nx, ly / ny, zf, bcs, precision="fp32")
    # FP32 columns have κ ≤ 10^4 (the rest are solved in FP64), so an elimination
    # in FP32 errs by up to ~κ·ε_32 relative to its column; 1e-4 of ‖p‖∞ still
    # fails any wrong coupling between blocks by orders of magnitude
    assert _relerr(p32, q) <= 1e-4
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6)
    assert info.status == 0 and info.rel_residual <= 1e-10, (info.status, info.rel_residual)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs)
    assert rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)
    assert _relerr(p, q) <= 1e-8
