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

* Each axis is periodic or bounded by no-slip walls at both ends (the Neumann
  pressure axis of the projection; the paper's duct and cavity cases of Table 3
  have walls on x and y). On a wall axis the normal component is 0 on the wall
  faces (face 0 stored, the top face implicit), and the tangential components
  have a ghost cell mirrored across the wall with the opposite sign (zero on the
  wall), one cell width away. x and y are uniform, z may be stretched.
* Advection in divergence form, ∂(u_i u_j)/∂x_j, with arithmetic averages for
  every interpolation (to cell centres for the normal products, to cell edges
  for the cross products); the derivative of a flux is the difference over the
  control volume of the face value: Δ (cell width) across a cell, the centre
  distance Δz^c across a z face.
* Viscous term: the finite-volume second differences of Eq. 4 applied to each
  component on its own control volume (for w: flux differences over Δz^f
  between z faces, divided by the centre distance).
* On a wall face AD is not formed: the normal component there stays 0 (the
  predictor and the projection leave it unchanged).

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
    if any(b not in ("P", "NN") for b in bcs):
        raise ValueError("the Navier–Stokes substep needs each axis periodic or bounded by walls (NN)")


class _Axis:
    """Neighbours of cell-centred and face quantities along one axis of the
    [n_z][n_y][n_x] arrays, under that axis's rule: periodic (wrap), or no-slip walls
    at both ends (the normal component is 0 on the wall faces, face 0 stored and the
    top face implicit; a tangential component has a ghost cell mirrored across the
    wall with the opposite sign, one cell width away)."""

    def __init__(self, faces, bc, axis):
        self.per = bc == "P"
        self.axis = axis                     # array axis: 2 = x, 1 = y, 0 = z
        self.dzf, dzc = metrics(faces)
        n = len(self.dzf)
        wrap = 0.5 * (self.dzf[0] + self.dzf[-1])
        # centre distance below cell k (k−1 to k) and above it (k to k+1)
        self.hdn = np.concatenate([[wrap if self.per else self.dzf[0]], dzc])
        self.hup = np.concatenate([dzc, [wrap if self.per else self.dzf[-1]]])
        self.n = n

    def col(self, v):
        """A per-index vector broadcast along this axis."""
        shape = [1, 1, 1]
        shape[self.axis] = -1
        return np.reshape(v, shape)

    def _sl(self, a, s):
        idx = [slice(None)] * a.ndim
        idx[self.axis] = s
        return a[tuple(idx)]

    def cm(self, a):
        """Cell-centred quantity at index −1 (wall: the mirrored ghost −a_0)."""
        if self.per:
            return np.roll(a, 1, axis=self.axis)
        return np.concatenate([-self._sl(a, slice(0, 1)), self._sl(a, slice(0, -1))], axis=self.axis)

    def cp(self, a):
        """Cell-centred quantity at index +1 (wall: the ghost −a_{n−1})."""
        if self.per:
            return np.roll(a, -1, axis=self.axis)
        return np.concatenate([self._sl(a, slice(1, None)), -self._sl(a, slice(-1, None))], axis=self.axis)

    def fp(self, w):
        """Face quantity at face +1 (wall: the implicit top face, 0)."""
        if self.per:
            return np.roll(w, -1, axis=self.axis)
        return np.concatenate([self._sl(w, slice(1, None)), np.zeros_like(self._sl(w, slice(0, 1)))],
                              axis=self.axis)

    def fm(self, w):
        """Face quantity at face −1 (used for faces ≥ 1 only on walls)."""
        if self.per:
            return np.roll(w, 1, axis=self.axis)
        return np.concatenate([np.zeros_like(self._sl(w, slice(0, 1))), self._sl(w, slice(0, -1))],
                              axis=self.axis)

    def wall_face(self, a):
        """a with its face 0 set to 0 (the wall face of the normal component)."""
        if self.per:
            return a
        a = a.copy()
        idx = [slice(None)] * a.ndim
        idx[self.axis] = 0
        a[tuple(idx)] = 0.0
        return a


def advection_diffusion(u3, nu, dx, dy, zf, bcs):
    """AD = −∂(u_i u_j)/∂x_j + ν∇²u_i at the faces of each component (shape (3, n_z, n_y, n_x)).

    Component c sits on the faces normal to its axis; its control volume spans the
    cell widths along the other two axes and the centre distance across its own
    face. For each axis d the flux of u_c through the volume's d faces is
    differenced over the volume's extent along d: advection with arithmetic
    averages (the normal product u_c² at cell centres when d = c; the cross product
    on the (c, d) cell edge otherwise, the same product for u_d's equation),
    diffusion the finite-volume second difference of Eq. 4."""
    _check(bcs)
    zf = np.asarray(zf, dtype=np.float64)
    nx, ny = np.shape(u3)[3], np.shape(u3)[2]
    axes = {0: _Axis(zf, bcs[2], 0), 1: _Axis(np.arange(ny + 1) * dy, bcs[1], 1),
            2: _Axis(np.arange(nx + 1) * dx, bcs[0], 2)}
    comp_axis = (2, 1, 0)                              # u on x faces, v on y faces, w on z faces
    u = [axes[comp_axis[c]].wall_face(np.asarray(u3[c], dtype=np.float64)) for c in range(3)]
    ad = []
    for c in range(3):
        A = axes[comp_axis[c]]
        uc = u[c]
        adv = np.zeros_like(uc)
        lap = np.zeros_like(uc)
        for d in range(3):
            if d == c:
                cc = 0.5 * (uc + A.fp(uc))                                 # u_c at the cell centre above the face
                adv += (cc ** 2 - np.roll(cc ** 2, 1, axis=A.axis)) / A.col(A.hdn)
                dzf_m = np.roll(A.dzf, 1)                                  # width of the cell below the face
                lap += ((A.fp(uc) - uc) / A.col(A.dzf) - (uc - A.fm(uc)) / A.col(dzf_m)) / A.col(A.hdn)
            else:
                B = axes[comp_axis[d]]
                e = 0.5 * (uc + B.cm(uc)) * 0.5 * (u[d] + A.cm(u[d]))    # the (c, d) edge below, along d
                adv += (B.fp(e) - e) / B.col(B.dzf)
                lap += ((B.cp(uc) - uc) / B.col(B.hup) - (uc - B.cm(uc)) / B.col(B.hdn)) / B.col(B.dzf)
        ad.append(A.wall_face(-adv + nu * lap))         # on a wall face AD is not formed: u_c stays 0
    return np.stack(ad)


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
