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
* Walls on x and y: ν∂²/∂x² of sin(πx) across x walls (and the same along y)
  converges at second order, and so do the advective and viscous parts of the
  normal component u = sin(πx) sin(2πz) between x walls.
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


def _faces(shape, dx, dy, zf):
    """Face coordinates per array axis (0 = z, 1 = y, 2 = x)."""
    nz, ny, nx = shape
    return {0: np.asarray(zf, dtype=np.float64), 1: np.arange(ny + 1) * dy, 2: np.arange(nx + 1) * dx}


def _bc(bcs, a):
    return {2: bcs[0], 1: bcs[1], 0: bcs[2]}[a]


def _widths(c, bcs, faces, shape):
    """Extent of component c's control volumes along each array axis, broadcast: the
    cell width across the other axes, the centre distance across its own face (the
    wall face, which carries no equation, gets 0)."""
    ca = (2, 1, 0)[c]
    out = {}
    for a in (0, 1, 2):
        dzf, dzc = O.metrics(faces[a])
        per = _bc(bcs, a) == "P"
        if a == ca:
            w = np.concatenate([[0.5 * (dzf[0] + dzf[-1]) if per else 0.0], dzc])
        else:
            w = dzf
        sh = [1, 1, 1]
        sh[a] = -1
        out[a] = w.reshape(sh)
    return out


def _volume(c, bcs, faces, shape):
    w = _widths(c, bcs, faces, shape)
    return w[0] * w[1] * w[2]


def _wall_flux(ns, u3, c, nu, bcs, faces):
    """What the fluxes of component c leave behind at the walls when its control
    volumes are summed (the interior faces telescope away), weighted by the face
    areas of the volumes:

    across the walls of another axis d: the viscous flux through the mirrored ghost,
    −2u/Δ^f at each wall (the advective edge products vanish there, u_d = 0);
    across the walls of its own axis (faces 1 … n−1): the flux of u_c² at the cell
    centres next to the walls (the centre value the mean of the two faces of the
    cell, the wall faces 0) and the viscous flux (u_1 − u_0)/Δ^f_0, (u_n − u_{n−1})/Δ^f_{n−1}.
    """
    ca = (2, 1, 0)[c]
    uc = np.asarray(u3[c], dtype=np.float64)
    w = _widths(c, bcs, faces, uc.shape)
    total = 0.0
    for d in (0, 1, 2):
        if _bc(bcs, d) == "P":
            continue
        dzf, _ = O.metrics(faces[d])
        others = [a for a in (0, 1, 2) if a != d]
        area = np.take(w[others[0]] * w[others[1]] * np.ones_like(uc), 0, axis=d)
        if d != ca:
            top, bot = np.take(uc, -1, axis=d), np.take(uc, 0, axis=d)
            total += (area * nu * (-2 * top / dzf[-1] - 2 * bot / dzf[0])).sum()
        else:
            top, first = np.take(uc, -1, axis=d), np.take(uc, 1, axis=d)
            flux = -((0.5 * top) ** 2 - (0.5 * first) ** 2) + nu * (-top / dzf[-1] - first / dzf[0])
            total += (area * flux).sum()
    return total


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
    bcs = ("P", "P", "NN")
    u3 = np.random.default_rng(11).standard_normal((3, nz, ny, nx))
    u3[2, 0] = 0.0
    faces = _faces((nz, ny, nx), dx, dy, zf)
    vol = _volume(2, bcs, faces, (nz, ny, nx))
    for nu in (0.0, 0.7):
        ad = ns.advection_diffusion(u3, nu, dx, dy, zf, bcs)
        s = (vol * ad[2]).sum()
        wall = _wall_flux(ns, u3, 2, nu, bcs, faces)
        assert abs(s - wall) < 1e-11 * np.abs(vol * ad[2]).sum(), (nu, s, wall)


def test_w_momentum_balance_on_tanh_grid():
    _w_balance(NS)


def _random_div_free(shape, zf, bcs, seed, dx, dy):
    u3 = np.random.default_rng(seed).standard_normal((3,) + shape)
    if bcs[0] != "P":
        u3[0, :, :, 0] = 0.0
    if bcs[1] != "P":
        u3[1, :, 0, :] = 0.0
    if bcs[2] != "P":
        u3[2, 0] = 0.0
    return AD.project(u3, dx, dy, zf, *bcs)


CONS = [(("P", "P", "P"), False), (("P", "P", "NN"), True), (("P", "P", "NN"), False),
        (("NN", "P", "NN"), True), (("NN", "NN", "P"), False), (("P", "NN", "NN"), False),
        (("NN", "NN", "NN"), True), (("NN", "NN", "NN"), False)]


@pytest.mark.parametrize("bcs,stretched", CONS, ids=["-".join(b) + ("-tanh" if st else "") for b, st in CONS])
def test_momentum_and_energy_conservation(bcs, stretched):
    nz, ny, nx, dx, dy = 10, 8, 12, 0.4, 0.3
    zf = synth.tanh_faces(nz, 1.0, 1.5) if stretched else O.uniform_faces(nz, 0.1)
    u3 = _random_div_free((nz, ny, nx), zf, bcs, 5, dx, dy)
    faces = _faces((nz, ny, nx), dx, dy, zf)
    vol = [_volume(c, bcs, faces, (nz, ny, nx)) for c in range(3)]
    for nu in (0.0, 0.7):
        ad = NS.advection_diffusion(u3, nu, dx, dy, zf, bcs)
        for c in (0, 1, 2):                  # periodic directions: momentum conserved,
            s = (vol[c] * ad[c]).sum()       # but for the fluxes through the walls
            wall = _wall_flux(NS, u3, c, nu, bcs, faces)
            assert abs(s - wall) < 1e-11 * np.abs(vol[c] * ad[c]).sum(), (c, nu, s, wall)
        if nu == 0.0 and not stretched:  # exact on uniform spacings only (arithmetic averages)
            work = sum((vol[c] * u3[c] * ad[c]).sum() for c in range(3))
            scale = sum(np.abs(vol[c] * u3[c] * ad[c]).sum() for c in range(3))
            assert abs(work) < 1e-11 * scale, (work, scale)


def test_wall_diffusion_along_x_and_y():
    """ν∂²v/∂x² of v = sin(πx) between walls on x (tangential to them: the mirrored
    ghost is exact), and ν∂²u/∂y² of u = sin(πy) between walls on y, converge at
    second order."""
    err = {"x": [], "y": []}
    for n in (16, 32, 64):
        h = 1.0 / n
        xc = (np.arange(n) + 0.5) * h
        zf = O.uniform_faces(4, 0.25)
        v = np.broadcast_to(np.sin(np.pi * xc)[None, None, :], (4, 4, n)).copy()
        u3 = np.stack([np.zeros_like(v), v, np.zeros_like(v)])
        ad = NS.advection_diffusion(u3, 1.0, h, 0.25, zf, ("NN", "P", "P"))
        err["x"].append(np.abs(ad[1, 0, 0] + np.pi ** 2 * np.sin(np.pi * xc)).max())
        u = np.broadcast_to(np.sin(np.pi * xc)[None, :, None], (4, n, 4)).copy()
        u3 = np.stack([u, np.zeros_like(u), np.zeros_like(u)])
        ad = NS.advection_diffusion(u3, 1.0, 0.25, h, zf, ("P", "NN", "P"))
        err["y"].append(np.abs(ad[0, 0, :, 0] + np.pi ** 2 * np.sin(np.pi * xc)).max())
    for e in err.values():
        assert e[1] < 0.3 * e[0] and e[2] < 0.3 * e[1], err


def _u_errors(ns, n):
    """AD_u's advective and viscous parts for u = sin(πx)·sin(2πz) on x faces between
    walls on x (zero on both), v = w = 0, periodic y and z: −∂(u²)/∂x and
    −ν(π² + 4π²)u."""
    h = 1.0 / n
    xf = np.arange(n) * h
    zc = (np.arange(n) + 0.5) * h
    Z, _, X = np.meshgrid(zc, np.arange(2), xf, indexing="ij")
    u = np.sin(np.pi * X) * np.sin(2 * np.pi * Z)
    u3 = np.stack([u, np.zeros_like(u), np.zeros_like(u)])
    zf = O.uniform_faces(n, h)
    bcs = ("NN", "P", "P")
    ad0 = ns.advection_diffusion(u3, 0.0, h, 0.5, zf, bcs)[0]
    ad1 = ns.advection_diffusion(u3, 1.0, h, 0.5, zf, bcs)[0]
    adv = -np.pi * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Z) ** 2
    lap = -(np.pi ** 2 + 4 * np.pi ** 2) * u
    inner = (slice(None), slice(None), slice(1, None))   # face 0 is the wall
    return np.abs(ad0 - adv)[inner].max(), np.abs((ad1 - ad0) - lap)[inner].max()


def test_u_momentum_between_x_walls_second_order():
    e = np.array([_u_errors(NS, n) for n in (16, 32, 64)])
    for part in (0, 1):
        assert e[1, part] < 0.3 * e[0, part] and e[2, part] < 0.3 * e[1, part], e


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
    # viscous flux below a face divided by the width of the cell above it, not below it
    ("(uc - A.fm(uc)) / A.col(dzf_m)", "(uc - A.fm(uc)) / A.col(A.dzf)"),
    # flux difference of u_c² taken over the cell width instead of the centre distance
    ("np.roll(cc ** 2, 1, axis=A.axis)) / A.col(A.hdn)", "np.roll(cc ** 2, 1, axis=A.axis)) / A.col(A.dzf)"),
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
    """A wall ghost with the wrong sign fails the wall-diffusion pins (z, and x/y);
    RK3 without its β_k terms fails the Taylor–Green pin."""
    orig_cm = NS._Axis.cm

    def cm_plus(self, a):
        out = orig_cm(self, a)
        if not self.per:
            out = out.copy()
            idx = [slice(None)] * out.ndim
            idx[self.axis] = 0
            out[tuple(idx)] = a[tuple(idx)]
        return out

    monkeypatch.setattr(NS._Axis, "cm", cm_plus)
    with pytest.raises(AssertionError):
        test_wall_diffusion_second_order_on_tanh_grid()
    with pytest.raises(AssertionError):
        test_wall_diffusion_along_x_and_y()
    monkeypatch.setattr(NS._Axis, "cm", orig_cm)
    monkeypatch.setattr(NS, "BETA", (0.0, 0.0, 0.0))
    with pytest.raises(AssertionError):
        test_rk3_taylor_green_decay_and_divergence()
