"""Pins for the oracle's Navier–Stokes substep (§2, Eqs. 2a–2d): no GPU.

* AD converges at second order to the analytic −(u·∇)u + ν∇²u of the 3-D
  Taylor–Green field (periodic box).
* The wall rule: ν∂²u/∂z² of u = sin(πz) (odd about both walls, so the mirrored
  ghost is exact) converges at second order on the stretched tanh grid.
* The wall-normal component on the stretched grid: for w = sin(2πx) sin(πz) on
  the z faces (zero on both walls) and u = v = 0, the advective part of AD_w
  converges at second order to −∂(w²)/∂z and the viscous part to
  −ν((2π)² + π²)w on the tanh grid (the w equation's own metrics: the centre
  distance across a z face, the cell widths between z faces).
* Conservation: the flux form sums to zero over each component's control volumes
  (momentum; with walls, the viscous part of u and v to the two discrete wall
  shear fluxes, and w's flux of w² and of ∂w/∂z to its values at the cells
  next to the walls), and for a discretely divergence-free field on uniform
  spacings the advective part does no work (kinetic energy), periodic or
  wall-bounded.
* The full RK3 step: the 2-D Taylor–Green vortex (an exact solution decaying as
  e^{−2νt}) is followed to O(Δx² + Δt²), and every substep leaves D u = 0.
"""

import inspect
import types

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


def _wall_flux(ns, u3, c, nu, dzf):
    """What the fluxes of component c leave behind at the walls when the control
    volumes of a wall-bounded z are summed (the interior faces telescope away).

    u, v: the viscous flux through the mirrored ghost, −2u/Δz^f at each wall.
    w (faces 1 … n−1): the flux of w² at the cell centres next to the walls,
    with the centre value the mean of the two faces of the cell (wall faces 0),
    and the viscous flux (w_1 − w_0)/Δz^f_0, (w_n − w_{n−1})/Δz^f_{n−1}.
    """
    if c < 2:
        return nu * (-2 * u3[c, -1] / dzf[-1] - 2 * u3[c, 0] / dzf[0]).sum()
    w = u3[2]
    top, bot = 0.5 * w[-1], 0.5 * w[1]
    return (-(top ** 2 - bot ** 2) + nu * (-w[-1] / dzf[-1] - w[1] / dzf[0])).sum()


def _w_errors(ns, nz):
    """Max errors of AD_w's advective and viscous parts against the analytic values
    for w = sin(2πx) sin(πz), u = v = 0, on the tanh grid with n_x = n_z."""
    nx, ny = nz, 2
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    dx = 1.0 / nx
    xc = (np.arange(nx) + 0.5) * dx
    Zf, _, X = np.meshgrid(zf[:-1], np.arange(ny), xc, indexing="ij")
    w = np.sin(2 * np.pi * X) * np.sin(np.pi * Zf)
    u3 = np.stack([np.zeros_like(w), np.zeros_like(w), w])
    bcs = ("P", "P", "NN")
    ad0 = ns.advection_diffusion(u3, 0.0, dx, 0.5, zf, bcs)[2]
    ad1 = ns.advection_diffusion(u3, 1.0, dx, 0.5, zf, bcs)[2]
    adv = -np.pi * np.sin(2 * np.pi * X) ** 2 * np.sin(2 * np.pi * Zf)  # −∂(w²)/∂z
    lap = -((2 * np.pi) ** 2 + np.pi ** 2) * w
    inner = slice(1, None)                  # face 0 is the wall (AD not formed)
    return (np.abs(ad0[inner] - adv[inner]).max(),
            np.abs((ad1 - ad0)[inner] - lap[inner]).max())


def _w_pin(ns):
    e = np.array([_w_errors(ns, nz) for nz in (16, 32, 64)])
    for part in (0, 1):                     # advective, viscous
        assert e[1, part] < 0.3 * e[0, part] and e[2, part] < 0.3 * e[1, part], e
    assert e[2, 0] < 2e-2 and e[2, 1] < 5e-1, e


def test_w_momentum_second_order_on_tanh_grid():
    _w_pin(NS)


def _w_balance(ns):
    nz, ny, nx, dx, dy = 12, 6, 8, 0.4, 0.3
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    dzf, dzc = O.metrics(zf)
    u3 = np.random.default_rng(11).standard_normal((3, nz, ny, nx))
    u3[2, 0] = 0.0
    hdn = np.concatenate([[dzf[0]], dzc])[:, None, None]
    for nu in (0.0, 0.7):
        ad = ns.advection_diffusion(u3, nu, dx, dy, zf, ("P", "P", "NN"))
        s = (hdn[1:] * ad[2, 1:]).sum()
        wall = _wall_flux(ns, u3, 2, nu, dzf)
        assert abs(s - wall) < 1e-11 * np.abs(hdn * ad[2]).sum(), (nu, s, wall)


def test_w_momentum_balance_on_tanh_grid():
    _w_balance(NS)


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
        for c in (0, 1, 2):                  # periodic directions: momentum conserved,
            s = (vol[c] * ad[c]).sum()       # but for the fluxes through the walls
            wall = _wall_flux(NS, u3, c, nu, dzf) if bcs[2] != "P" else 0.0
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


def _mutant(old, new):
    """A copy of the oracle's substep module with one expression replaced."""
    src = inspect.getsource(NS)
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle._ns_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), "<oracle.navier_stokes mutant>", "exec"), mod.__dict__)
    return mod


W_SLIPS = [
    # viscous w flux below face k divided by Δz^f_k instead of Δz^f_{k−1}
    ("- (w - Z.fm(w)) / dzf_m) / hdn)", "- (w - Z.fm(w)) / dzf) / hdn)"),
    # flux difference of w² taken over the cell width instead of the centre distance
    ("np.roll(wcc ** 2, 1, axis=0)) / hdn", "np.roll(wcc ** 2, 1, axis=0)) / dzf"),
]


@pytest.mark.parametrize("old,new", W_SLIPS)
def test_planted_w_slips_are_caught(old, new):
    """Each slip in the w equation's stretched metrics fails a w pin."""
    ns = _mutant(old, new)
    caught = 0
    for pin in (_w_pin, _w_balance):
        try:
            pin(ns)
        except AssertionError:
            caught += 1
    assert caught >= 1


def test_unmutated_copy_passes_the_w_pins():
    """The copy mechanism itself changes nothing: a no-op replacement passes."""
    ns = _mutant(W_SLIPS[0][0], W_SLIPS[0][0])
    _w_pin(ns)
    _w_balance(ns)


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
