"""GPU parity for face-centred x and y unknowns between two walls
(PS_BC_FACE_DIRICHLET on a transformed axis, "FD"): the velocity normal to walls on
x or y in an implicit diffusion step (§2), transformed by a DST-I of the interior
faces with the wall entry copied (the non-staggered transforms named at the end
of §2.1). Entry 0 of a line is the low wall face, the high wall face is implicit.

Checked against the FP64 oracle with the same operator: FP64 to 1e-12, FP32 to
2e-5, the refined mode to a residual of 1e-10 with the reported residual equal to
the oracle's residual of the returned p, the transpose solve, with and without a
Helmholtz shift; ragged and radix-3 line lengths; x lines and y lines (the
shared-memory transform kernel); the wall contract (f = 0 on the wall faces gives
p = 0 there); plans the other paths refuse.
"""

import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import operator as O
from oracle import solve as S
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(lib, f, dx, dy, zf, bcs, precision="fp64", transpose=False, **kw):
    import torch
    nz, ny, nx = f.shape
    plan = lib.Plan(nx, ny, nz, dx, dy, zf=zf, bcs=bcs, precision=precision, **kw)
    dt = torch.float32 if precision == "fp32" else torch.float64
    ft = torch.as_tensor(f, dtype=dt, device="cuda").contiguous()
    info = lib.info_tensor()
    out = plan.solve_transpose(ft, info=info) if transpose else plan.solve(ft, info=info)
    torch.cuda.synchronize()
    res = out.double().cpu().numpy(), lib.read_info(info)
    plan.close()
    return res


def _relerr(p, q):
    return np.abs(p - q).max() / max(np.abs(q).max(), 1e-300)


CASES = [((6, 8, 12), ("FD", "P", "NN"), 0.0), ((5, 12, 24), ("NN", "FD", "DD"), 0.0),
         ((4, 48, 36), ("FD", "FD", "P"), 0.0), ((6, 16, 96), ("FD", "DN", "FD"), 3.0),
         ((3, 64, 64), ("DD", "FD", "ND"), 40.0), ((4, 72, 36), ("FD", "NN", "NN"), 0.0),
         # face-centred x with y lines of 2048: the z solve on transposed planes carries the
         # wall row's eigenvalue in its swapped x/y tables
         ((3, 2048, 24), ("FD", "P", "NN"), 0.0)]
IDS = [f"{'x'.join(map(str, s))}-{'-'.join(b)}-a{a:g}" for s, b, a in CASES]


def _grid(shape, bcs):
    nz, ny, nx = shape
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] not in ("P",) else synth.uniform_faces(nz, 1.0)
    return 1.0 / nx, 2.0 / ny, zf


@pytest.mark.parametrize("shape,bcs,alpha", CASES, ids=IDS)
def test_face_xy_fp64_fp32_transpose(lib, shape, bcs, alpha):
    dx, dy, zf = _grid(shape, bcs)
    f = np.random.default_rng(sum(shape)).uniform(-1, 1, shape)
    if bcs[2] == "FD":
        f[0] = 0.0
    q = S.solve(f, dx, dy, zf, *bcs, alpha=alpha)
    p, _ = _run(lib, f, dx, dy, zf, bcs, alpha=alpha)
    assert _relerr(p, q) <= 1e-12
    p32, _ = _run(lib, f, dx, dy, zf, bcs, precision="fp32", alpha=alpha)
    assert _relerr(p32, q) <= 2e-5
    if bcs[2] != "FD":  # (face-centred z has no transpose solve)
        qt = AD.solve_transpose(f, dx, dy, zf, *bcs, alpha=alpha)
        pt, _ = _run(lib, f, dx, dy, zf, bcs, alpha=alpha, transpose=True)
        assert _relerr(pt, qt) <= 1e-12


@pytest.mark.parametrize("shape,bcs,alpha", CASES, ids=IDS)
def test_face_xy_refine(lib, shape, bcs, alpha):
    dx, dy, zf = _grid(shape, bcs)
    f = np.random.default_rng(2 * sum(shape)).uniform(-1, 1, shape)
    if bcs[2] == "FD":
        f[0] = 0.0
    p, info = _run(lib, f, dx, dy, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=8, alpha=alpha)
    rr = O.relative_residual(p, f, dx, dy, zf, *bcs, alpha=alpha)
    assert info.status == 0 and info.rel_residual <= 1e-10 and rr <= 1e-10, (info.status, info.rel_residual, rr)
    assert abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)
    q = S.solve(f, dx, dy, zf, *bcs, alpha=alpha)
    assert _relerr(p, q) <= 1e-8


def test_face_xy_wall_contract(lib):
    """f = 0 on the wall faces of x and y gives p = 0 there, in every mode."""
    shape, bcs = (6, 24, 36), ("FD", "FD", "NN")
    dx, dy, zf = _grid(shape, bcs)
    f = np.random.default_rng(7).uniform(-1, 1, shape)
    f[:, :, 0] = 0.0
    f[:, 0, :] = 0.0
    for prec in ("fp64", "fp32", "fp32_refine"):
        p, _ = _run(lib, f, dx, dy, zf, bcs, precision=prec, rtol=1e-10, max_iter=8)
        assert np.abs(p[:, :, 0]).max() == 0.0 and np.abs(p[:, 0, :]).max() == 0.0, prec


def test_face_xy_refused_where_unsupported(lib):
    """Lines longer than 4096 and the batched solve refuse face-centred x/y."""
    with pytest.raises(lib.PoissonError):
        lib.Plan(8192, 4, 4, 1.0 / 8192, 0.25, zf=synth.uniform_faces(4, 1.0), bcs=("FD", "P", "NN"))
    grids = [dict(nx=16, ny=16, nz=8, dx=1 / 16, dy=1 / 16, zf=synth.uniform_faces(8, 1.0), bcs=("FD", "P", "NN"))]
    with pytest.raises(Exception):
        lib.Batch(grids, rtol=1e-10, max_iter=4)
