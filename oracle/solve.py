"""The eigenfunction-expansion solve of §2.1 (three steps), in plain FP64.

Oracle module (test infrastructure only; see ``oracle/__init__``).

Steps, in the order of §2.1:

1. f̂ = F^y(F^x(f)): the Table 2 forward transform along x on every x-line,
   then along y on every y-line (dense matrices, one matmul per axis).
2. For every wavenumber pair (q_x, q_y) solve the z system of Eq. 5,
   ``a_k Φ̂_{k−1} + (b_k + λ_{q_x}/Δx² + λ_{q_y}/Δy²) Φ̂_k + c_k Φ̂_{k+1} = f̂_k``,
   by Gauss elimination (cyclic for a periodic z).
3. Φ = F^{−1,x}(F^{−1,y}(Φ̂)) with the Table 1 inverses.

Singular problems (every axis P or NN, so constants are in the null space):
the (q_x, q_y) = (0, 0) column is singular. Reading taken: remove the
Δz^f-weighted mean of f̂(0,0,:) (this is the volume-weighted mean of f, i.e.
the incompatible part), solve that column with Φ̂_0 = 0 pinned (row 0
dropped; it is implied by the others for a compatible right-hand side), then
subtract the Δz^f-weighted mean of the column. The result solves A p = f_c
(f_c = f minus its volume-weighted mean) with zero volume-weighted mean of p.

Helmholtz variant (``alpha`` = α ≥ 0, see ``oracle.operator``): the transforms
diagonalise the identity as well, so α only moves every diagonal of Eq. 5 by −α;
for α > 0 no column is singular.
"""

import numpy as np

from .transforms import forward_matrix, backward_matrix, eigenvalues, apply_along
from .operator import metrics, is_singular
from .tridiag import thomas, thomas_cyclic


def z_system(zf, bcz):
    """Coefficients (a, b, c) of the z rows of Eq. 4 on faces ``zf``.

    a_k = 1/(Δz^f_k Δz^c_{k−1}), c_k = 1/(Δz^f_k Δz^c_k), b_k = −(a_k + c_k)
    inside; at an end a Neumann face drops its term, a Dirichlet face adds
    −2/(Δz^f)² to b (ghost −Φ mirrored across the face), a periodic face couples
    to the other end at distance (Δz^f_0 + Δz^f_{n−1})/2 (a_0 and c_{n−1} then
    hold the wrap couplings).
    """
    dzf, dzc = metrics(zf)
    n = len(dzf)
    a = np.zeros(n)
    c = np.zeros(n)
    b = np.zeros(n)
    if bcz == "FD":  # face-centred unknowns between two walls (see oracle.operator)
        b[0] = -1.0
        a[1:] = 1.0 / (dzf[:-1] * dzc)     # to face k−1 (row 1: the stored wall face)
        c[1:-1] = 1.0 / (dzf[1:-1] * dzc[:-1])
        b[1:] = -(a[1:] + 1.0 / (dzf[1:] * dzc))
        return a, b, c
    a[1:] = 1.0 / (dzf[1:] * dzc)
    c[:-1] = 1.0 / (dzf[:-1] * dzc)
    b[1:] -= a[1:]
    b[:-1] -= c[:-1]
    if bcz == "P":
        hper = 0.5 * (dzf[0] + dzf[-1])
        a[0] = 1.0 / (dzf[0] * hper)
        c[-1] = 1.0 / (dzf[-1] * hper)
        b[0] -= a[0]
        b[-1] -= c[-1]
    else:
        lo_d = bcz in ("DD", "DN")
        hi_d = bcz in ("DD", "ND")
        if lo_d:
            b[0] -= 2.0 / dzf[0] ** 2
        if hi_d:
            b[-1] -= 2.0 / dzf[-1] ** 2
    return a, b, c


def shifts(nx, ny, dx, dy, bcx, bcy):
    """λ_{q_x}/Δx² + λ_{q_y}/Δy² as an [n_y][n_x] array (Eq. 5, Table 1)."""
    return eigenvalues(bcx, nx)[None, :] / dx ** 2 + eigenvalues(bcy, ny)[:, None] / dy ** 2


def forward_xy(f, bcx, bcy):
    """Step 1: f̂ = F^y(F^x(f)) for a [n_z][n_y][n_x] array."""
    nz, ny, nx = f.shape
    fh = apply_along(forward_matrix(bcx, nx), f, 2)
    return apply_along(forward_matrix(bcy, ny), fh, 1)


def backward_xy(ph, bcx, bcy):
    """Step 3: F^{−1,x}(F^{−1,y}(Φ̂))."""
    nz, ny, nx = ph.shape
    p = apply_along(backward_matrix(bcy, ny), ph, 1)
    return apply_along(backward_matrix(bcx, nx), p, 2)


def _singular_column(a, b, c, d, dzf):
    d = d - (dzf * d).sum() / dzf.sum()
    x = np.zeros_like(d)
    x[1:] = thomas(a[1:], b[1:], c[1:], d[1:])
    return x - (dzf * x).sum() / dzf.sum()


def solve_columns(fh, lam, zf, bcz, singular):
    """Step 2: the N_x·N_y z systems of Eq. 5 (spectral in x and y)."""
    a, b, c = z_system(zf, bcz)
    dzf, _ = metrics(zf)
    B = b[:, None, None] + lam[None, :, :]
    if singular:
        B = B.copy()
        B[:, 0, 0] -= 1.0          # placeholder; column (0,0) is replaced below
    solver = thomas_cyclic if bcz == "P" else thomas
    ph = solver(a, B, c, fh)
    if singular:
        ph[:, 0, 0] = _singular_column(a, b, c, fh[:, 0, 0], dzf)
    return ph


def solve(f, dx, dy, zf, bcx, bcy, bcz, alpha=0.0):
    """Φ with (A − α) Φ = f (f_c for singular problems), A the operator of Eq. 4."""
    f = np.asarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    zf = np.asarray(zf, dtype=np.float64)
    if len(zf) != nz + 1:
        raise ValueError("zf must hold n_z + 1 face coordinates")
    fh = forward_xy(f, bcx, bcy)
    lam = shifts(nx, ny, dx, dy, bcx, bcy) - alpha
    ph = solve_columns(fh, lam, zf, bcz, is_singular(bcx, bcy, bcz, alpha))
    return backward_xy(ph, bcx, bcy)
