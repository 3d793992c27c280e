"""Gauss elimination for the z systems of Eq. 5 (Thomas), and the cyclic case.

Oracle module (test infrastructure only; see ``oracle/__init__``).

The paper solves each of the N_x·N_y tridiagonal systems with LAPACK DGTSV
(§3), which pivots. Here the elimination is done without pivoting: every
non-singular column is weakly diagonally dominant with a strictly dominant
row (λ ≤ 0 on the diagonal, b_k = −(a_k + c_k) inside), so no pivot is needed
and the result equals DGTSV's up to rounding. For a periodic z the cyclic
system is reduced to two tridiagonal solves sharing one elimination
(Sherman–Morrison), as §3 says.

Row k reads ``a_k x_{k−1} + b_k x_k + c_k x_{k+1} = d_k``. All arrays have the
z index first; trailing dimensions are independent columns, solved together.
"""

import numpy as np


def thomas(a, b, c, d):
    """Solve one tridiagonal system per column; a_0 and c_{n−1} are ignored."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    b = np.broadcast_to(b, d.shape) if np.ndim(b) == d.ndim else np.broadcast_to(
        np.reshape(b, (n,) + (1,) * (d.ndim - 1)), d.shape)
    shp = (n,) + (1,) * (d.ndim - 1)
    a = np.reshape(np.asarray(a, dtype=np.float64), shp)
    c = np.reshape(np.asarray(c, dtype=np.float64), shp)
    cp = np.empty(d.shape)
    dp = np.empty(d.shape)
    m = b[0]
    cp[0] = c[0] / m
    dp[0] = d[0] / m
    for k in range(1, n):
        m = b[k] - a[k] * cp[k - 1]
        cp[k] = c[k] / m
        dp[k] = (d[k] - a[k] * dp[k - 1]) / m
    x = np.empty(d.shape)
    x[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return x


def thomas_cyclic(a, b, c, d):
    """Cyclic system: row 0 also has a_0·x_{n−1}, row n−1 also has c_{n−1}·x_0.

    Sherman–Morrison: A = B + u vᵀ with γ = −b_0,
    u = (γ, 0, …, 0, c_{n−1}), v = (1, 0, …, 0, a_0/γ); solve B y = d and
    B z = u, then x = y − (v·y)/(1 + v·z) z.
    """
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    shp = (n,) + (1,) * (d.ndim - 1)
    b = np.array(np.broadcast_to(b if np.ndim(b) == d.ndim else np.reshape(b, shp), d.shape))
    a = np.asarray(a, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    gamma = -b[0]
    bb = b.copy()
    bb[0] = b[0] - gamma
    bb[n - 1] = b[n - 1] - a[0] * c[n - 1] / gamma
    u = np.zeros(d.shape)
    u[0] = gamma
    u[n - 1] = c[n - 1]
    y = thomas(a, bb, c, d)
    z = thomas(a, bb, c, u)
    vy = y[0] + (a[0] / gamma) * y[n - 1]
    vz = z[0] + (a[0] / gamma) * z[n - 1]
    return y - (vy / (1.0 + vz)) * z
