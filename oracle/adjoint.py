"""Transpose solve and the staggered projection step (Eqs. 2b–2c), in FP64.

Oracle module (test infrastructure only; see ``oracle/__init__``).

Transpose solve. The operator of Eq. 4 on a stretched z is A = W⁻¹ S with
W = diag(Δz^f_k) (x and y are uniform) and S symmetric, so Aᵀ = W A W⁻¹ and
the transpose of the solve map M (including its singular-mode handling: the
projector that removes the weighted mean has transpose W·(projector)·W⁻¹) is
Mᵀ g = W · M(W⁻¹ g). ``solve_transpose`` is that formula; the tests pin it
against the explicit transpose of M built column by column on tiny grids.

Projection. On the staggered (MAC) grid of §2 the velocity component along an
axis lives on the cell faces normal to it. Storage used here: each component
has the cell array's shape, entry ``[…, i]`` being the face on the low side of
cell i. On a periodic axis face 0 is the wrap face; on a Neumann-pressure axis
(prescribed velocity, end of §2) face 0 is the wall, and the high wall is
implicit; the divergence gives wall faces zero weight and the gradient is zero
there. With these, D·G equals the operator of Eq. 4. The projection of
Eqs. 2b–2c (γΔt cancels) is u = u* − G M D u*.

Only P and NN axes are supported for the projection (the pressure BCs that go
with periodic and prescribed-velocity boundaries).
"""

import numpy as np
import scipy.sparse as sp

from .operator import metrics, uniform_faces
from .solve import solve


def solve_transpose(g, dx, dy, zf, bcx, bcy, bcz, alpha=0.0):
    """Mᵀ g = W · M(W⁻¹ g), W = diag(Δz^f) along z (A − α = W⁻¹(S − αW), S − αW symmetric)."""
    dzf, _ = metrics(zf)
    w = dzf[:, None, None]
    return w * solve(g / w, dx, dy, zf, bcx, bcy, bcz, alpha)


def _check(bcs):
    for b in bcs:
        if b not in ("P", "NN"):
            raise ValueError("projection supports P and NN axes only")


def _axis_faces(n, faces):
    """Centre distances used by the gradient at face i (low side of cell i)."""
    dzf, dzc = metrics(faces)
    h = np.empty(n)
    h[1:] = dzc
    h[0] = 0.5 * (dzf[0] + dzf[-1])
    return dzf, h


def divergence_matrix(nx, ny, dx, dy, zf, bcx, bcy, bcz):
    """Sparse N×3N matrix D: cell divergence of the stacked (u, v, w) face arrays."""
    _check((bcx, bcy, bcz))
    zf = np.asarray(zf, dtype=np.float64)
    nz = len(zf) - 1
    N = nx * ny * nz
    shape = (nz, ny, nx)
    rows, cols, vals = [], [], []
    axes = [(2, nx, uniform_faces(nx, dx), bcx), (1, ny, uniform_faces(ny, dy), bcy),
            (0, nz, zf, bcz)]
    for comp, (ax, n, faces, bc) in enumerate(axes):
        dzf, _ = metrics(faces)
        for c in range(N):
            idx = list(np.unravel_index(c, shape))
            i = idx[ax]
            h = dzf[i]
            # + flux out of the high face (face i+1), − flux in through face i
            hi = i + 1
            if hi < n:
                idh = idx.copy(); idh[ax] = hi
                rows.append(c); cols.append(comp * N + np.ravel_multi_index(idh, shape)); vals.append(1.0 / h)
            elif bc == "P":
                idh = idx.copy(); idh[ax] = 0
                rows.append(c); cols.append(comp * N + np.ravel_multi_index(idh, shape)); vals.append(1.0 / h)
            if i > 0 or bc == "P":
                rows.append(c); cols.append(comp * N + c); vals.append(-1.0 / h)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, 3 * N))


def gradient_matrix(nx, ny, dx, dy, zf, bcx, bcy, bcz):
    """Sparse 3N×N matrix G: face gradient of a cell array (zero on walls)."""
    _check((bcx, bcy, bcz))
    zf = np.asarray(zf, dtype=np.float64)
    nz = len(zf) - 1
    N = nx * ny * nz
    shape = (nz, ny, nx)
    rows, cols, vals = [], [], []
    axes = [(2, nx, uniform_faces(nx, dx), bcx), (1, ny, uniform_faces(ny, dy), bcy),
            (0, nz, zf, bcz)]
    for comp, (ax, n, faces, bc) in enumerate(axes):
        _, h = _axis_faces(n, faces)
        for c in range(N):
            idx = list(np.unravel_index(c, shape))
            i = idx[ax]
            if i == 0 and bc != "P":
                continue
            lo = idx.copy(); lo[ax] = (i - 1) % n
            rows.append(comp * N + c); cols.append(c); vals.append(1.0 / h[i])
            rows.append(comp * N + c); cols.append(np.ravel_multi_index(lo, shape)); vals.append(-1.0 / h[i])
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * N, N))


def project(ustar, dx, dy, zf, bcx, bcy, bcz):
    """u = u* − G M D u* for u* of shape (3, n_z, n_y, n_x)."""
    _, nz, ny, nx = ustar.shape
    D = divergence_matrix(nx, ny, dx, dy, zf, bcx, bcy, bcz)
    G = gradient_matrix(nx, ny, dx, dy, zf, bcx, bcy, bcz)
    f = (D @ ustar.ravel()).reshape(nz, ny, nx)
    phi = solve(f, dx, dy, zf, bcx, bcy, bcz)
    return ustar - (G @ phi.ravel()).reshape(ustar.shape)


def project_vjp(g, dx, dy, zf, bcx, bcy, bcz):
    """Pᵀ g = g − Dᵀ Mᵀ Gᵀ g (plain transposes of the sparse D and G)."""
    _, nz, ny, nx = g.shape
    D = divergence_matrix(nx, ny, dx, dy, zf, bcx, bcy, bcz)
    G = gradient_matrix(nx, ny, dx, dy, zf, bcx, bcy, bcz)
    h = (G.T @ g.ravel()).reshape(nz, ny, nx)
    s = solve_transpose(h, dx, dy, zf, bcx, bcy, bcz)
    return g - (D.T @ s.ravel()).reshape(g.shape)
