"""Direct LU solve of the assembled 7-point system (no transform involved).

Oracle module (test infrastructure only; see ``oracle/__init__``).

The eigenfunction-expansion method reaches the exact discrete solution up to
rounding (§1: FFT direct solvers satisfy the solution to machine precision), so
a direct factorisation of the same assembled matrix must give the same answer.
This is the independent cross-check of ``oracle.solve``: it uses only
``operator.operator_3d`` (ghost-cell rules) and a library LU.

Singular problems use the bordered system [[A, 1], [vᵀ, 0]] [p; μ] = [f; 0]
with v the cell volumes: it returns the p with A p = f − μ·1 (μ the
volume-weighted mean of f) and vᵀ p = 0.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .operator import operator_3d, is_singular, cell_volumes


def solve_direct(f, dx, dy, zf, bcx, bcy, bcz, dense=False, alpha=0.0):
    f = np.asarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    A = operator_3d(nx, ny, dx, dy, zf, bcx, bcy, bcz, alpha)
    rhs = f.ravel()
    N = rhs.size
    if is_singular(bcx, bcy, bcz, alpha):
        v = np.ascontiguousarray(cell_volumes(nx, ny, dx, dy, zf)).ravel()
        A = sp.bmat([[A, sp.csr_matrix(np.ones((N, 1)))],
                     [sp.csr_matrix(v[None, :]), None]]).tocsr()
        rhs = np.concatenate([rhs, [0.0]])
    if dense:
        x = np.linalg.solve(A.toarray(), rhs)
    else:
        x = spla.spsolve(A.tocsc(), rhs)
    return x[:N].reshape(nz, ny, nx)
