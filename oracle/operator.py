"""The second-order 7-point operator of Eq. 4, built from ghost-cell rules.

Oracle module (test infrastructure only; see ``oracle/__init__``).

Arrays are C-ordered ``[n_z][n_y][n_x]`` (x fastest), cell-centred. x and y are
uniform (§2.1 requires a constant spacing in the two transformed directions);
z may be non-uniform (footnote to Eq. 5), given by its n_z + 1 face
coordinates.

Readings (the paper gives the uniform stencil only):

* "Staggered" BCs (Table 1 caption, end of §2.1): the boundary sits on a cell
  face. Neumann: ghost Φ_{−1} = Φ_0 (zero flux). Dirichlet: ghost
  Φ_{−1} = −Φ_0 mirrored across the face (zero value on the face). Periodic:
  the ghost is the cell on the other end. ``"ND"`` is Neumann at the low end,
  Dirichlet at the high end; ``"DN"`` (not in Table 1) the reverse.
* Stretched z: finite-volume form ``(flux_{k+1/2} − flux_{k−1/2}) / Δz^f_k``
  with ``flux_{k+1/2} = (Φ_{k+1} − Φ_k) / Δz^c_k``; Δz^f_k is the width of
  cell k and Δz^c_k the distance between the centres of cells k and k+1. A
  Dirichlet ghost sits a distance Δz^f of the boundary cell away (its mirror
  image); a periodic ghost sits (Δz^f_0 + Δz^f_{n−1})/2 away. On a uniform grid
  this is exactly the z row of Eq. 4.

Face-centred x or y (``"FD"`` on a transformed axis; non-staggered unknowns for the
velocity normal to walls on that axis). Entry i of a line is x face i; entry 0 is
the low wall face and the high wall face n is implicit, both with value 0. Reading
taken (the transforms of §2.1 must diagonalise it): the interior faces 1 … n−1
carry the Dirichlet second difference (u_{i+1} − 2u_i + u_{i−1})/Δ² with the wall
values u_0 = u_n = 0 (the node of the wall is boundary data, not the stored entry),
and the wall entry's own row is −u_0/Δ². With f = 0 on the wall face (the caller's
contract, as for z) u_0 = 0 and this is the same solution as the z rule.

``operator_1d`` and ``apply`` are two separate codings of these rules (a matrix
assembled row by row, and a padded-array stencil); tests check they agree.

Helmholtz variant (§2: an implicit diffusion step needs one Helmholtz equation
per velocity component; §4: done with the same method): the operator of Eq. 4
minus α times the identity, α ≥ 0 (``alpha``; α = 0 is the Poisson problem).
For α > 0 the constants leave the null space, so no problem is singular.

Face-centred z (``"FD"``, z only; the velocity component normal to the walls in
an implicit diffusion step, §2 and the end of §2.1: non-staggered unknowns). The
unknown w_k sits on z face k; plane 0 is the bottom wall face and the top wall
face n is implicit, both with w = 0 (Dirichlet on the node). Row k ≥ 1 is the
finite-volume second difference on the control volume between the centres of
cells k−1 and k: ((w_{k+1} − w_k)/Δz^f_k − (w_k − w_{k−1})/Δz^f_{k−1}) / Δz^c_{k−1},
with w_n = 0; row 0 is −w_0 (so w_0 = 0 when the right-hand side is 0 there).
"""

import numpy as np
import scipy.sparse as sp

from .transforms import BCS


def uniform_faces(n, h):
    """Face coordinates 0, h, …, n·h of a uniform axis."""
    return np.arange(n + 1, dtype=np.float64) * h


def metrics(faces):
    """(Δz^f, Δz^c): cell widths (n) and centre-to-centre distances (n−1)."""
    faces = np.asarray(faces, dtype=np.float64)
    dzf = np.diff(faces)
    zc = 0.5 * (faces[:-1] + faces[1:])
    return dzf, np.diff(zc)


def _ends(bc):
    """BC kind at (low, high) end: 'N', 'D' or 'P'."""
    if bc not in BCS:
        raise ValueError(f"unknown BC {bc!r}")
    return {"P": ("P", "P"), "NN": ("N", "N"), "DD": ("D", "D"), "ND": ("N", "D"), "DN": ("D", "N")}[bc]


def operator_1d_faces(faces):
    """Dense n×n matrix of the face-centred ("FD") z operator, assembled row by row."""
    dzf, dzc = metrics(faces)
    n = len(dzf)
    L = np.zeros((n, n))
    L[0, 0] = -1.0
    for k in range(1, n):
        h = dzc[k - 1]                     # control volume: centres of cells k−1 and k
        up = 1.0 / (dzf[k] * h)            # flux to face k+1 (the top wall when k = n−1)
        dn = 1.0 / (dzf[k - 1] * h)        # flux to face k−1 (the stored bottom wall when k = 1)
        L[k, k] -= up + dn
        L[k, k - 1] += dn
        if k + 1 < n:
            L[k, k + 1] += up
    return L


def operator_1d_nodes(n, h):
    """Dense n×n matrix of the face-centred ("FD") x/y operator, assembled row by row."""
    L = np.zeros((n, n))
    L[0, 0] = -1.0 / h ** 2                 # the wall face's own row
    for i in range(1, n):
        L[i, i] = -2.0 / h ** 2
        if i > 1:                           # (i = 1: the low wall node carries 0)
            L[i, i - 1] = 1.0 / h ** 2
        if i < n - 1:                       # (i = n−1: the high wall node carries 0)
            L[i, i + 1] = 1.0 / h ** 2
    return L


def operator_1d(bc, faces, axis="z"):
    """Dense n×n matrix of the 1D operator on one axis, assembled row by row
    (``axis`` "xy" selects the transformed-axis rule for "FD")."""
    if bc == "FD":
        if axis == "xy":
            faces = np.asarray(faces, dtype=np.float64)
            return operator_1d_nodes(len(faces) - 1, faces[1] - faces[0])
        return operator_1d_faces(faces)
    dzf, dzc = metrics(faces)
    n = len(dzf)
    lo, hi = _ends(bc)
    L = np.zeros((n, n))
    hper = 0.5 * (dzf[0] + dzf[-1])
    for k in range(n):
        w = 1.0 / dzf[k]
        # flux through the upper face of cell k: (Φ_up − Φ_k)/h_up
        if k < n - 1:
            L[k, k + 1] += w / dzc[k]
            L[k, k] -= w / dzc[k]
        elif hi == "P":
            L[k, 0] += w / hper
            L[k, k] -= w / hper
        elif hi == "D":            # ghost −Φ_k at distance Δz^f_k
            L[k, k] -= 2.0 * w / dzf[k]
        # Neumann: zero flux, nothing added
        # minus the flux through the lower face: (Φ_k − Φ_down)/h_down
        if k > 0:
            L[k, k] -= w / dzc[k - 1]
            L[k, k - 1] += w / dzc[k - 1]
        elif lo == "P":
            L[k, k] -= w / hper
            L[k, n - 1] += w / hper
        elif lo == "D":
            L[k, k] -= 2.0 * w / dzf[k]
    return L


def operator_3d(nx, ny, dx, dy, zf, bcx, bcy, bcz, alpha=0.0):
    """Sparse (CSR) N×N matrix of Eq. 4 (minus α·I) on the [n_z][n_y][n_x] grid."""
    zf = np.asarray(zf, dtype=np.float64)
    nz = len(zf) - 1
    Lx = sp.csr_matrix(operator_1d(bcx, uniform_faces(nx, dx), axis="xy"))
    Ly = sp.csr_matrix(operator_1d(bcy, uniform_faces(ny, dy), axis="xy"))
    Lz = sp.csr_matrix(operator_1d(bcz, zf))
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    A = sp.kron(Lz, sp.kron(Iy, Ix)) + sp.kron(Iz, sp.kron(Ly, Ix)) + sp.kron(Iz, sp.kron(Iy, Lx))
    if alpha:
        A = A - alpha * sp.identity(nx * ny * nz)
    return A.tocsr()


def _faces_term(p, axis, faces):
    """The face-centred ("FD") z term from shifted copies (wall values 0)."""
    dzf, dzc = metrics(faces)
    w = np.moveaxis(p, axis, 0)
    n = w.shape[0]
    shape = (-1,) + (1,) * (w.ndim - 1)
    wp = np.concatenate([w[1:], np.zeros_like(w[:1])], axis=0)        # w_{k+1}, w_n = 0
    flux_up = (wp - w) / dzf.reshape(shape)                            # between faces k and k+1
    term = np.empty_like(w)
    term[1:] = (flux_up[1:] - flux_up[:-1]) / dzc.reshape(shape)       # rows k ≥ 1
    term[0] = -w[0]
    return np.moveaxis(term, 0, axis)


def _nodes_term(p, axis, h):
    """The face-centred ("FD") x/y term from shifted copies (wall nodes 0)."""
    u = np.moveaxis(p, axis, 0)
    z = np.zeros_like(u[:1])
    um = np.concatenate([z, z, u[1:-1]], axis=0)      # u_{i−1}; row 1 sees the wall node 0
    up = np.concatenate([u[1:], z], axis=0)           # u_{i+1}; the high wall node 0
    term = (um + up - 2.0 * u) / h ** 2
    term[0] = -u[0] / h ** 2                          # the wall face's own row
    return np.moveaxis(term, 0, axis)


def _axis_term(p, axis, faces, bc):
    """Second-difference term of one axis, from a padded copy (ghost rules above)."""
    if bc == "FD":
        if axis != 0:
            return _nodes_term(p, axis, faces[1] - faces[0])
        return _faces_term(p, axis, faces)
    dzf, dzc = metrics(faces)
    lo, hi = _ends(bc)
    x = np.moveaxis(p, axis, 0)
    if lo == "P":
        glo, ghi = x[-1], x[0]
        hlo = hhi = 0.5 * (dzf[0] + dzf[-1])
    else:
        glo = x[0] if lo == "N" else -x[0]
        ghi = x[-1] if hi == "N" else -x[-1]
        hlo, hhi = dzf[0], dzf[-1]
    ext = np.concatenate([glo[None], x, ghi[None]], axis=0)
    h = np.concatenate([[hlo], dzc, [hhi]])
    shape = (-1,) + (1,) * (x.ndim - 1)
    flux = (ext[1:] - ext[:-1]) / h.reshape(shape)
    term = (flux[1:] - flux[:-1]) / dzf.reshape(shape)
    return np.moveaxis(term, 0, axis)


def apply(p, dx, dy, zf, bcx, bcy, bcz, alpha=0.0):
    """A·p − α·p for a [n_z][n_y][n_x] FP64 array (stencil form of Eq. 4)."""
    p = np.asarray(p, dtype=np.float64)
    nz, ny, nx = p.shape
    ap = (_axis_term(p, 2, uniform_faces(nx, dx), bcx)
          + _axis_term(p, 1, uniform_faces(ny, dy), bcy)
          + _axis_term(p, 0, np.asarray(zf, dtype=np.float64), bcz))
    return ap - alpha * p if alpha else ap


def is_singular(bcx, bcy, bcz, alpha=0.0):
    """True when the constant is in the null space: every axis P or NN, and α = 0."""
    return alpha == 0 and all(b in ("P", "NN") for b in (bcx, bcy, bcz))


def cell_volumes(nx, ny, dx, dy, zf):
    """Cell volumes Δx·Δy·Δz^f_k broadcast to [n_z][n_y][n_x]."""
    dzf, _ = metrics(zf)
    return np.broadcast_to((dx * dy * dzf)[:, None, None], (len(dzf), ny, nx))


def compatible_part(f, dx, dy, zf, bcx, bcy, bcz, alpha=0.0):
    """f with its volume-weighted mean removed when the operator is singular."""
    if not is_singular(bcx, bcy, bcz, alpha):
        return np.array(f, dtype=np.float64, copy=True)
    nz, ny, nx = f.shape
    v = cell_volumes(nx, ny, dx, dy, zf)
    return f - (v * f).sum() / v.sum()


def relative_residual(p, f, dx, dy, zf, bcx, bcy, bcz, alpha=0.0):
    """‖f_c − (A − α) p‖∞ / ‖f_c‖∞ with f_c the compatible part of f."""
    fc = compatible_part(f, dx, dy, zf, bcx, bcy, bcz, alpha)
    r = fc - apply(p, dx, dy, zf, bcx, bcy, bcz, alpha)
    return np.abs(r).max() / np.abs(fc).max()
