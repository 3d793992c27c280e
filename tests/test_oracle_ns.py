"""Pins for the oracle's Navier–Stokes substep (§2, Eqs. 2a–2d): no GPU.

* AD converges at second order to the analytic −(u·∇)u + ν∇²u of the 3-D
  Taylor–Green field (periodic box).
* The wall rule: ν∂²u/∂z² of u = sin(πz) (odd about both walls, so the mirrored
  ghost is exact) converges at second order on the stretched tanh grid.
* Conservation: the flux form sums to zero over each component's control volumes
  (momentum; with walls, the viscous part to the two discrete wall shear fluxes),
  and for a discretely divergence-free field on uniform spacings the advective
  part does no work (kinetic energy), periodic or wall-bounded.
* The full RK3 step: the 2-D Taylor–Green vortex (an exact solution decaying as
  e^{−2νt}) is followed to O(Δx² + Δt²), and every substep leaves D u = 0.
"""

import numpy as np
import pytest

from oracle import navier_stokes as NS
from oracle import adjoint as AD
from oracle import operator as O
from paper_1802_10323_gb300 import synth


def _tg3(n, L=2 * np.pi):
    h = L / n
    xf = np.arange(n) * h           # faces (low side of cell i)
    xc = (np.arange(n) + 0.5) * h   # centres
    Z, Y, X = np.meshgrid(xc, xc, xf, indexing="ij")
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    Z, Y, X = np.meshgrid(xc, xf, xc, indexing="ij")
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    return np.stack([u, v, np.zeros_like(u)]), h


def _tg3_ad(n, nu, L=2 * np.pi):
    h = L / n
    xf = np.arange(n) * h
    xc = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(xc, xc, xf, indexing="ij")
    adu = -0.5 * np.sin(2 * X) * np.cos(Z) ** 2 - 3 * nu * np.sin(X) * np.cos(Y) * np.cos(Z)
    Z, Y, X = np.meshgrid(xc, xf, xc, indexing="ij")
    adv = -0.5 * np.sin(2 * Y) * np.cos(Z) ** 2 + 3 * nu * np.cos(X) * np.sin(Y) * np.cos(Z)
    return np.stack([adu, adv, np.zeros_like(adu)])


def test_ad_taylor_green_second_order():
    nu = 0.05
    err = []
    for n in (16, 32):
        u3, h = _tg3(n)
        zf = O.uniform_faces(n, h)
        ad = NS.advection_diffusion(u3, nu, h, h, zf, ("P", "P", "P"))
        err.append(np.abs(ad - _tg3_ad(n, nu)).max())
    assert err[1] < 0.3 * err[0] and err[1] < 2e-2, err


def test_wall_diffusion_second_order_on_tanh_grid():
    nu = 1.0
    err = []
    for nz in (16, 32, 64):
        zf = synth.tanh_faces(nz, 1.0, 1.5)
        zc = 0.5 * (zf[:-1] + zf[1:])
        u = np.broadcast_to(np.sin(np.pi * zc)[:, None, None], (nz, 4, 4)).copy()
        u3 = np.stack([u, np.zeros_like(u), np.zeros_like(u)])
        ad = NS.advection_diffusion(u3, nu, 0.5, 0.5, zf, ("P", "P", "NN"))
        exact = -np.pi ** 2 * np.sin(np.pi * zc)
        err.append(np.abs(ad[0, :, 0, 0] - exact).max())
        assert np.abs(ad[1:]).max() == 0.0
    assert err[1] < 0.3 * err[0] and err[2] < 0.3 * err[1], err


def _random_div_free(shape, zf, bcs, seed, dx, dy):
    u3 = np.random.default_rng(seed).standard_normal((3,) + shape)
    if bcs[2] != "P":
        u3[2, 0] = 0.0
    return AD.project(u3, dx, dy, zf, *bcs)


@pytest.mark.parametrize("bcs,stretched", [(("P", "P", "P"), False), (("P", "P", "NN"), True),
                                           (("P", "P", "NN"), False)])
def test_momentum_and_energy_conservation(bcs, stretched):
    nz, ny, nx, dx, dy = 10, 8, 12, 0.4, 0.3
    zf = synth.tanh_faces(nz, 1.0, 1.5) if stretched else O.uniform_faces(nz, 0.1)
    u3 = _random_div_free((nz, ny, nx), zf, bcs, 5, dx, dy)
    dzf, dzc = O.metrics(zf)
    hdn = np.concatenate([[0.5 * (dzf[0] + dzf[-1]) if bcs[2] == "P" else dzf[0]], dzc])
    vol = [dzf[:, None, None], dzf[:, None, None], hdn[:, None, None]]
    if bcs[2] != "P":
        vol[2] = vol[2].copy()
        vol[2][0] = 0.0                      # the wall face carries no momentum
    for nu in (0.0, 0.7):
        ad = NS.advection_diffusion(u3, nu, dx, dy, zf, bcs)
        for c in (0, 1):                     # periodic directions: momentum conserved,
            s = (vol[c] * ad[c]).sum()       # but for the shear stress on walls
            wall = 0.0
            if bcs[2] != "P":                # telescoped fluxes through the mirrored ghosts
                wall = nu * (-2 * u3[c, -1] / dzf[-1] - 2 * u3[c, 0] / dzf[0]).sum()
            assert abs(s - wall) < 1e-11 * np.abs(vol[c] * ad[c]).sum(), (c, nu, s, wall)
        if nu == 0.0 and not stretched:  # exact on uniform spacings only (arithmetic averages)
            work = sum((vol[c] * u3[c] * ad[c]).sum() for c in range(3))
            scale = sum(np.abs(vol[c] * u3[c] * ad[c]).sum() for c in range(3))
            assert abs(work) < 1e-11 * scale, (work, scale)


def _tg2(n, t, nu):
    h = 2 * np.pi / n
    xf = np.arange(n) * h
    xc = (np.arange(n) + 0.5) * h
    d = np.exp(-2 * nu * t)
    Z, Y, X = np.meshgrid(xc, xc, xf, indexing="ij")
    u = d * np.sin(X) * np.cos(Y)
    Z, Y, X = np.meshgrid(xc, xf, xc, indexing="ij")
    v = -d * np.cos(X) * np.sin(Y)
    return np.stack([u, v, np.zeros_like(u)]), h


def test_rk3_taylor_green_decay_and_divergence():
    nu, T = 0.1, 0.2
    err = []
    for n, steps in ((8, 4), (16, 8)):
        u3, h = _tg2(n, 0.0, nu)
        zf = O.uniform_faces(4, h)
        u3 = u3[:, :4]                       # z-independent: four planes suffice
        p = np.zeros(u3.shape[1:])
        D = AD.divergence_matrix(n, n, h, h, zf, "P", "P", "P")
        dt = T / steps
        ad = np.zeros_like(u3)
        for _ in range(steps):
            for k in (1, 2, 3):
                u3, p, ad, _ = NS.substep(u3, p, ad, k, dt, nu, h, h, zf, ("P", "P", "P"))
                assert np.abs(D @ u3.ravel()).max() < 1e-11
        exact, _ = _tg2(n, T, nu)
        err.append(np.abs(u3 - exact[:, :4]).max())
    assert err[1] < 0.35 * err[0] and err[1] < 1e-3, err   # measured 1.8e-3 → 4.8e-4


def test_planted_mistakes_are_caught(monkeypatch):
    """A wall ghost with the wrong sign fails the wall-diffusion pin; RK3 without its
    β_k terms fails the Taylor–Green pin."""
    orig_cm = NS._Z.cm

    def cm_plus(self, a):
        out = orig_cm(self, a)
        if not self.per:
            out = out.copy()
            out[0] = a[0]
        return out

    monkeypatch.setattr(NS._Z, "cm", cm_plus)
    with pytest.raises(AssertionError):
        test_wall_diffusion_second_order_on_tanh_grid()
    monkeypatch.setattr(NS._Z, "cm", orig_cm)
    monkeypatch.setattr(NS, "BETA", (0.0, 0.0, 0.0))
    with pytest.raises(AssertionError):
        test_rk3_taylor_green_decay_and_divergence()
