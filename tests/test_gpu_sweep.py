"""GPU parity at the sizes of the BC sweep and the channel workload.

* The BC sweep at 256³: x and y each drawn from {P, NN, DD, ND}, all 16 pairs, z
  Neumann–Neumann on the tanh grid (stretch 1.5); f = the analytic Laplacian of a
  product of per-axis profiles that satisfy each BC, plus 10 % seeded uniform noise
  (mean removed where the problem is singular). FP64 against the FP64 oracle to
  1e-12 of ‖p‖∞, every element.
* FP64 on full 1024 × 1024 planes (the channel's x and y lines, P/P/NN tanh z) and
  with n_z = 1024 columns (the z length of the channel workload), against the oracle.
"""

import itertools

import numpy as np
import pytest

from oracle import operator as O
from oracle import solve as S
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu

PAIRS = list(itertools.product(("P", "NN", "DD", "ND"), repeat=2))


def _solve(lib, f, dx, dy, zf, bcs, precision="fp64", **kw):
    import torch
    nz, ny, nx = f.shape
    plan = lib.Plan(nx, ny, nz, dx, dy, zf=zf, bcs=bcs, precision=precision, **kw)
    ft = torch.as_tensor(f, device="cuda").contiguous()
    info = lib.info_tensor()
    p = plan.solve(ft, info=info)
    torch.cuda.synchronize()
    out = p.cpu().numpy(), lib.read_info(info)
    plan.close()
    del ft, p
    return out


@pytest.mark.parametrize("bcx,bcy", PAIRS, ids=[f"{a}-{b}" for a, b in PAIRS])
def test_bc_sweep_256(lib, bcx, bcy):
    n = 256
    bcs = (bcx, bcy, "NN")
    zf = synth.tanh_faces(n, 1.0, 1.5)
    seed = 100 + PAIRS.index((bcx, bcy))
    _, f = synth.manufactured(n, n, 1.0, 1.0, zf, bcs, noise=0.1, seed=seed)
    f = O.compatible_part(f, 1.0 / n, 1.0 / n, zf, *bcs)
    q = S.solve(f, 1.0 / n, 1.0 / n, zf, *bcs)
    p, _ = _solve(lib, f, 1.0 / n, 1.0 / n, zf, bcs)
    assert np.abs(p - q).max() <= 1e-12 * np.abs(q).max()


def test_fp64_full_1024_planes(lib):
    nz, ny, nx = 4, 1024, 1024
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    dx, dy = 6.0 / nx, 3.0 / ny
    u, v, w = synth.staggered_velocity(nx, ny, nz, 3)
    f = synth.divergence_rhs(u, v, w, dx, dy, zf)
    q = S.solve(f, dx, dy, zf, "P", "P", "NN")
    p, _ = _solve(lib, f, dx, dy, zf, ("P", "P", "NN"))
    assert np.abs(p - q).max() <= 1e-12 * np.abs(q).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refine", 1e-8)])
def test_nz_1024_columns(lib, precision, tol):
    """The channel's z length (1024 tanh-stretched planes) with its right-hand side
    (the divergence of a Gaussian staggered velocity) on a 128 × 64 cross-section of
    the 6 × 3 box. (With i.i.d. noise on a coarse 32 × 8 cross-section the two FP64
    computations differ by ~2e-12: the lowest columns' z systems are conditioned at
    ~10^7 there, and both sides round.)"""
    nz, ny, nx = 1024, 64, 128
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    dx, dy = 6.0 / nx, 3.0 / ny
    u, v, w = synth.staggered_velocity(nx, ny, nz, 4)
    f = synth.divergence_rhs(u, v, w, dx, dy, zf)
    q = S.solve(f, dx, dy, zf, "P", "P", "NN")
    p, info = _solve(lib, f, dx, dy, zf, ("P", "P", "NN"), precision=precision, rtol=1e-10, max_iter=6)
    assert np.abs(p - q).max() <= tol * np.abs(q).max()
    if precision == "fp32_refine":
        assert info.status == 0 and info.rel_residual <= 1e-10
