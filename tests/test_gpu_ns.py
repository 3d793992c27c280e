"""GPU parity of the RK3 fractional step around the solve (§2, Eqs. 2a–2d):
ps_ns_substep against the FP64 oracle (oracle/navier_stokes.py), substep by
substep — u^{k+1}, p^{k+1/2}, Φ and AD^k — on periodic and wall-bounded grids
(walls on z, stretched or not; on y and z as in a duct; on every axis; on x only),
for FP64, refined and FP32 plans; the result is discretely divergence-free.
"""

import numpy as np
import pytest

from oracle import navier_stokes as NS
from oracle import adjoint as AD
from oracle import operator as O
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(shape, bcs, stretched, seed):
    nz, ny, nx = shape
    dx, dy = 0.7 / nx, 0.45 / ny
    zf = synth.tanh_faces(nz, 1.0, 1.5) if stretched else O.uniform_faces(nz, 0.6 / nz)
    rng = np.random.default_rng(seed)
    u3 = rng.standard_normal((3,) + shape)
    if bcs[0] != "P":
        u3[0, :, :, 0] = 0.0
    if bcs[1] != "P":
        u3[1, :, 0, :] = 0.0
    if bcs[2] != "P":
        u3[2, 0] = 0.0
    u3 = AD.project(u3, dx, dy, zf, *bcs)
    p = rng.standard_normal(shape)
    return u3, p, dx, dy, zf


# periodic box, channel (walls on z), duct (walls on y and z), cavity-like box
# (walls on every axis), walls on x only
CASES = [((8, 12, 16), ("P", "P", "P"), False), ((10, 8, 12), ("P", "P", "NN"), True),
         ((12, 16, 8), ("P", "P", "NN"), False), ((10, 12, 16), ("P", "NN", "NN"), True),
         ((8, 12, 12), ("NN", "NN", "NN"), True), ((6, 8, 18), ("NN", "P", "P"), False)]


# u and AD at the path's precision; p and Φ come straight out of the solve, whose solution
# error is its residual accuracy (rtol = 1e-13 refined, ε_32 plain FP32) times the operator's
# condition number (~10^4 at these sizes), while u only sees the small correction G·Φ'
@pytest.mark.parametrize("precision,tol,tol_p", [("fp64", 1e-12, 1e-12), ("fp32_refine", 1e-9, 2e-8),
                                                 ("fp32", 2e-5, 3e-4)])
@pytest.mark.parametrize("shape,bcs,stretched", CASES, ids=["x".join(map(str, c[0])) + "-" + "-".join(c[1]) +
                                                             ("-tanh" if c[2] else "") for c in CASES])
def test_rk3_substeps_match_oracle(lib, shape, bcs, stretched, precision, tol, tol_p):
    import torch
    nz, ny, nx = shape
    u3, p, dx, dy, zf = _setup(shape, bcs, stretched, nx + ny)
    dt, nu = 2e-3, 0.03
    plan = lib.Plan(nx, ny, nz, dx, dy, zf=zf, bcs=bcs, precision=precision, rtol=1e-13, max_iter=8)
    dtp = torch.float32 if precision == "fp32" else torch.float64
    ut = torch.as_tensor(u3, dtype=dtp, device="cuda").contiguous()
    pt = torch.as_tensor(p, dtype=dtp, device="cuda").contiguous()
    ad_t = torch.full_like(ut, float("nan"))   # substep 1 must not read it
    us, phi, rhs = torch.empty_like(ut), torch.empty_like(pt), torch.empty_like(pt)
    info = lib.info_tensor()
    ad = np.zeros_like(u3)
    for k in (1, 2, 3):
        u3, p, ad, ph = NS.substep(u3, p, ad, k, dt, nu, dx, dy, zf, bcs)
        plan.ns_substep(k, dt, nu, ut, us, ad_t, pt, phi, rhs, info=info)
        torch.cuda.synchronize()
        for name, got, ref in (("u", ut, u3), ("p", pt, p), ("phi", phi, ph), ("ad", ad_t, ad)):
            g = got.double().cpu().numpy()
            err = np.abs(g - ref).max() / np.abs(ref).max()
            assert err <= (tol_p if name in ("p", "phi") else tol), (k, name, err)
    D = AD.divergence_matrix(nx, ny, dx, dy, zf, *bcs)
    div = np.abs(D @ ut.double().cpu().numpy().ravel()).max()
    scale = np.abs(D).max() * np.abs(u3).max()
    assert div <= (1e-5 if precision == "fp32" else 1e-11) * scale, div
    plan.close()


def test_rk3_taylor_green_decays_on_gpu(lib):
    """Twenty steps of the 2-D Taylor–Green vortex on 32² (×4 planes): the GPU follows
    the exact decay e^{−2νt} to O(Δx²) (the oracle's pin at the same sizes)."""
    import torch
    n, nz, nu, T, steps = 32, 4, 0.1, 0.2, 20
    h = 2 * np.pi / n
    xf, xc = np.arange(n) * h, (np.arange(n) + 0.5) * h

    def tg(t):
        d = np.exp(-2 * nu * t)
        Z, Y, X = np.meshgrid(xc[:nz], xc, xf, indexing="ij")
        u = d * np.sin(X) * np.cos(Y)
        Z, Y, X = np.meshgrid(xc[:nz], xf, xc, indexing="ij")
        v = -d * np.cos(X) * np.sin(Y)
        return np.stack([u, v, np.zeros_like(u)])

    zf = O.uniform_faces(nz, h)
    plan = lib.Plan(n, n, nz, h, h, zf=zf, bcs=("P", "P", "P"), precision="fp64")
    ut = torch.as_tensor(tg(0.0), device="cuda").contiguous()
    pt = torch.zeros((nz, n, n), dtype=torch.float64, device="cuda")
    ad_t, us = torch.zeros_like(ut), torch.empty_like(ut)
    phi, rhs = torch.empty_like(pt), torch.empty_like(pt)
    for _ in range(steps):
        for k in (1, 2, 3):
            plan.ns_substep(k, T / steps, nu, ut, us, ad_t, pt, phi, rhs)
    torch.cuda.synchronize()
    err = np.abs(ut.cpu().numpy() - tg(T)).max()
    assert err < 1.5e-3, err
    plan.close()


def test_substep_refuses_overlapping_arrays(lib):
    """Every pair of the substep's arrays (and the workspace) must be disjoint: p
    equal to phi, or ustar starting inside u, is refused before any launch."""
    import torch
    shape, bcs = (8, 12, 16), ("P", "P", "P")
    nz, ny, nx = shape
    plan = lib.Plan(nx, ny, nz, 0.1, 0.1, zf=O.uniform_faces(nz, 0.1), bcs=bcs, precision="fp64")
    ut = torch.zeros((3,) + shape, dtype=torch.float64, device="cuda")
    big = torch.zeros((4,) + shape, dtype=torch.float64, device="cuda")
    pt = torch.zeros(shape, dtype=torch.float64, device="cuda")
    ad_t, us = torch.zeros_like(ut), torch.zeros_like(ut)
    phi, rhs = torch.zeros_like(pt), torch.zeros_like(pt)
    with pytest.raises(lib.PoissonError, match="p and phi overlap"):
        plan.ns_substep(1, 1e-3, 0.01, ut, us, ad_t, pt, pt, rhs)
    # ustar = the last three components of a 4-component buffer whose first three are u
    with pytest.raises(lib.PoissonError, match="u and ustar overlap"):
        plan.ns_substep(1, 1e-3, 0.01, big[:3], big[1:], ad_t, pt, phi, rhs)
    with pytest.raises(lib.PoissonError, match="phi and rhs overlap"):
        plan.ns_substep(1, 1e-3, 0.01, ut, us, ad_t, pt, phi, phi)
    plan.ns_substep(1, 1e-3, 0.01, ut, us, ad_t, pt, phi, rhs)   # disjoint: accepted
    torch.cuda.synchronize()
    plan.close()
