"""One RK3 substep of the fractional-step Navier–Stokes integration of §2 (Eqs. 2a–2d), FP64.

Oracle module (test infrastructure only; see ``oracle/__init__``).

Substep k (k = 1, 2, 3; α = 8/15, 5/12, 3/4; β = 0, −17/60, −5/12; γ = α + β):

    u* = u^k + Δt (α_k AD^k + β_k AD^{k−1} − γ_k G p^{k−1/2})        (2a)
    A Φ = D u* / (γ_k Δt)                                              (2b)
    u^{k+1} = u* − γ_k Δt G Φ                                          (2c)
    p^{k+1/2} = p^{k−1/2} + Φ                                          (2d)

with AD = −(u·∇)u + ν∇²u, and D, G, A the divergence, gradient and operator of
the projection (``oracle.adjoint``; D·G = A, Eq. 4). Layout as there: each
component has the cell array's shape [n_z][n_y][n_x], entry i along its own
axis being the face on the low side of cell i; the stack is (3, n_z, n_y, n_x).

Readings (the paper names second-order central differences on the staggered
grid and gives no stencil):

* x and y are periodic; z is periodic or bounded by no-slip walls (the
  Neumann pressure axis of the projection). On walls w = 0 on the wall faces
  (face 0 stored, the top face implicit), and the tangential components have a
  ghost cell mirrored across the wall with the opposite sign (zero on the wall).
* Advection in divergence form, ∂(u_i u_j)/∂x_j, with arithmetic averages for
  every interpolation (to cell centres for the normal products, to cell edges
  for the cross products); the derivative of a flux is the difference over the
  control volume of the face value: Δ (cell width) across a cell, the centre
  distance Δz^c across a z face.
* Viscous term: the finite-volume second differences of Eq. 4 applied to each
  component on its own control volume (for w: flux differences over Δz^f
  between z faces, divided by the centre distance).
* On a wall face AD is not formed: w there stays 0 (the predictor and the
  projection leave it unchanged).

With these choices the advective flux form conserves momentum exactly, and for a
discretely divergence-free field it does no work on uniform spacings; on the
stretched z the arithmetic averages leave an energy error of truncation size.
"""

import numpy as np

from .operator import metrics
from .adjoint import divergence_matrix, gradient_matrix
from .solve import solve

ALPHA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
BETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)


def _check(bcs):
    if bcs[0] != "P" or bcs[1] != "P" or bcs[2] not in ("P", "NN"):
        raise ValueError("the Navier–Stokes substep needs periodic x and y, and a periodic or wall z")


def _xm(a):
    return np.roll(a, 1, axis=2)


def _xp(a):
    return np.roll(a, -1, axis=2)


def _ym(a):
    return np.roll(a, 1, axis=1)


def _yp(a):
    return np.roll(a, -1, axis=1)


class _Z:
    """z neighbours of cell-centred and z-face arrays under the z boundary rule."""

    def __init__(self, zf, bcz):
        self.per = bcz == "P"
        self.dzf, dzc = metrics(zf)
        n = len(self.dzf)
        wrap = 0.5 * (self.dzf[0] + self.dzf[-1])
        # centre distance below cell k (k−1 to k) and above it (k to k+1)
        self.hdn = np.concatenate([[wrap if self.per else self.dzf[0]], dzc])
        self.hup = np.concatenate([dzc, [wrap if self.per else self.dzf[-1]]])
        self.n = n

    def cm(self, a):
        """Cell-centred quantity at k−1 (wall: the mirrored ghost −a_0)."""
        if self.per:
            return np.roll(a, 1, axis=0)
        return np.concatenate([-a[:1], a[:-1]], axis=0)

    def cp(self, a):
        """Cell-centred quantity at k+1 (wall: the ghost −a_{n−1})."""
        if self.per:
            return np.roll(a, -1, axis=0)
        return np.concatenate([a[1:], -a[-1:]], axis=0)

    def fp(self, w):
        """z-face quantity at face k+1 (wall: the implicit top face, 0)."""
        if self.per:
            return np.roll(w, -1, axis=0)
        return np.concatenate([w[1:], np.zeros_like(w[:1])], axis=0)

    def fm(self, w):
        """z-face quantity at face k−1 (used for faces k ≥ 1 only on walls)."""
        if self.per:
            return np.roll(w, 1, axis=0)
        return np.concatenate([np.zeros_like(w[:1]), w[:-1]], axis=0)


def advection_diffusion(u3, nu, dx, dy, zf, bcs):
    """AD = −∂(u_i u_j)/∂x_j + ν∇²u_i at the faces of each component (shape (3, n_z, n_y, n_x))."""
    _check(bcs)
    zf = np.asarray(zf, dtype=np.float64)
    Z = _Z(zf, bcs[2])
    u, v, w = (np.asarray(c, dtype=np.float64) for c in u3)
    if not Z.per:
        w = w.copy()
        w[0] = 0.0
    dzf = Z.dzf[:, None, None]
    hdn = Z.hdn[:, None, None]
    hup = Z.hup[:, None, None]

    # edge products (arithmetic averages of the two neighbours across the edge)
    uv = 0.5 * (u + _ym(u)) * 0.5 * (v + _xm(v))          # x face i, y face j
    uw = 0.5 * (u + Z.cm(u)) * 0.5 * (w + _xm(w))         # x face i, z face k
    vw = 0.5 * (v + Z.cm(v)) * 0.5 * (w + _ym(w))         # y face j, z face k

    # x momentum at x face i (cells j, k)
    ucc = 0.5 * (u + _xp(u))                               # u at the centre of cell i
    adv_u = (ucc ** 2 - _xm(ucc ** 2)) / dx + (_yp(uv) - uv) / dy + (Z.fp(uw) - uw) / dzf
    lap_u = ((_xp(u) - 2 * u + _xm(u)) / dx ** 2 + (_yp(u) - 2 * u + _ym(u)) / dy ** 2
             + ((Z.cp(u) - u) / hup - (u - Z.cm(u)) / hdn) / dzf)

    # y momentum at y face j
    vcc = 0.5 * (v + _yp(v))
    adv_v = (_xp(uv) - uv) / dx + (vcc ** 2 - _ym(vcc ** 2)) / dy + (Z.fp(vw) - vw) / dzf
    lap_v = ((_xp(v) - 2 * v + _xm(v)) / dx ** 2 + (_yp(v) - 2 * v + _ym(v)) / dy ** 2
             + ((Z.cp(v) - v) / hup - (v - Z.cm(v)) / hdn) / dzf)

    # z momentum at z face k: control volume between the centres of cells k−1 and k
    wcc = 0.5 * (w + Z.fp(w))                              # w at the centre of cell k
    dzf_m = np.roll(Z.dzf, 1)[:, None, None]               # Δz^f_{k−1} (k ≥ 1; periodic wraps)
    adv_w = (_xp(uw) - uw) / dx + (_yp(vw) - vw) / dy + (wcc ** 2 - np.roll(wcc ** 2, 1, axis=0)) / hdn
    lap_w = ((_xp(w) - 2 * w + _xm(w)) / dx ** 2 + (_yp(w) - 2 * w + _ym(w)) / dy ** 2
             + ((Z.fp(w) - w) / dzf - (w - Z.fm(w)) / dzf_m) / hdn)

    ad = np.stack([-adv_u + nu * lap_u, -adv_v + nu * lap_v, -adv_w + nu * lap_w])
    if not Z.per:
        ad[2, 0] = 0.0                                     # wall face: w stays 0
    return ad


def substep(u3, p, ad_prev, k, dt, nu, dx, dy, zf, bcs):
    """Substep k ∈ {1, 2, 3}: returns (u^{k+1}, p^{k+1/2}, AD^k, Φ)."""
    _check(bcs)
    u3 = np.asarray(u3, dtype=np.float64)
    _, nz, ny, nx = u3.shape
    al, be = ALPHA[k - 1], BETA[k - 1]
    ga = al + be
    D = divergence_matrix(nx, ny, dx, dy, zf, *bcs)
    G = gradient_matrix(nx, ny, dx, dy, zf, *bcs)
    ad = advection_diffusion(u3, nu, dx, dy, zf, bcs)
    gp = (G @ p.ravel()).reshape(u3.shape)
    ustar = u3 + dt * (al * ad + be * ad_prev - ga * gp)
    phi_s = solve((D @ ustar.ravel()).reshape(nz, ny, nx), dx, dy, zf, *bcs)   # = γΔt·Φ
    u_new = ustar - (G @ phi_s.ravel()).reshape(u3.shape)
    phi = phi_s / (ga * dt)
    return u_new, p + phi, ad, phi


def rk3_step(u3, p, dt, nu, dx, dy, zf, bcs):
    """One time step: the three substeps in order (AD^{k−1} carried between them)."""
    ad = np.zeros_like(u3)
    for k in (1, 2, 3):
        u3, p, ad, _ = substep(u3, p, ad, k, dt, nu, dx, dy, zf, bcs)
    return u3, p
