"""Table 1 eigenvalues and Table 2 discrete transforms, as dense FP64 matrices.

Oracle module (test infrastructure only; see ``oracle/__init__``).

Boundary-condition names follow Table 1: ``"P"`` periodic (P-P), ``"NN"``
staggered Neumann at both ends, ``"DD"`` staggered Dirichlet at both ends,
``"ND"`` Neumann at the low end and Dirichlet at the high end. ``n`` is the
(even) number of cells along the axis (Table 1 caption).

``"DN"`` (Dirichlet at the low end, Neumann at the high end) is not in Table 1.
Reading taken: it is the ND problem on the reversed axis (a_p ↦ a_{n−1−p}), so
its forward transform is ND's applied to the reversed line, its inverse ND's
inverse followed by the reversal, and its θ_q (hence λ_q) are ND's.

Conventions
-----------
``forward_matrix(bc, n)[q, p]`` maps a physical line ``a_p`` to its spectral
coefficient ``â_q`` exactly as Table 2 writes it; ``backward_matrix(bc, n)``
is the inverse named in Table 1 (1/n IDFT, 1/(2n) DCT-III, 1/(2n) DST-III,
1/(2n) DCT-IV), so ``backward @ forward == I``.

Reading of the periodic rows (the DFT/IDFT rows of Table 2 are garbled: the
cosine row starts at ``q = 1`` with ``l = 0``, which repeats ``q = 0``, and the
IDFT row lacks the factor 2 of the paired terms). The reading taken here is the
half-complex layout of a real DFT of n reals (footnote of §3):

* ``q = 0``:        Σ a_p
* ``q = 2l − 1``:   Σ a_p cos(2π p l / n),   l = 1 … n/2 − 1
* ``q = 2l``:       Σ a_p sin(2π p l / n),   l = 1 … n/2 − 1
* ``q = n − 1``:    Σ a_p (−1)^p
* inverse:  a_p = (1/n)[â_0 + 2 Σ_l (â_{2l−1} cos + â_{2l} sin)(2π p l/n)
  + â_{n−1} (−1)^p].

With this layout Table 1's periodic θ reads θ_q = ⌈q/2⌉ π / n (its
``θ_{p−1}`` for even q is read as "the same θ as q − 1").

Non-staggered unknowns on x or y (``"FD"``; the velocity component normal to
walls on that axis in an implicit diffusion step: §2 and the end of §2.1 name
non-staggered transforms for it without stating them). Entry 0 of a line is the
low wall face (stored, value 0), entries 1 … n−1 the interior faces, the high
wall face n implicit. The interior faces are the nodes of the Dirichlet second
difference, diagonalised by the sine transform of type I: forward
â_0 = a_0, â_k = 2 Σ_{i=1}^{n−1} a_i sin(π k i / n), k = 1 … n−1; its inverse
a_0 = â_0, a_i = (1/n) Σ_k â_k sin(π k i / n) (the same transform divided by 2n);
eigenvalues λ_0 = −1 (the wall face's own row, see ``oracle.operator``) and
λ_k = −4 sin²(π k / 2n).
"""

import numpy as np

BCS = ("P", "NN", "DD", "ND", "DN")
XY_BCS = BCS + ("FD",)   # accepted on x and y (FD: non-staggered, see above)


def _check(bc, n):
    if bc not in XY_BCS:
        raise ValueError(f"unknown BC {bc!r}")
    if n < 2 or n % 2:
        raise ValueError("n must be even and >= 2 (Table 1 caption)")


def _cos_pi(num, den):
    """cos(π·num/den) for integer arrays, with the argument reduced mod 2π."""
    num = np.mod(num, 2 * den)
    return np.cos(np.pi * num / den)


def _sin_pi(num, den):
    num = np.mod(num, 2 * den)
    return np.sin(np.pi * num / den)


def theta(bc, n):
    """θ_q of Table 1, q = 0 … n−1 (FP64)."""
    _check(bc, n)
    q = np.arange(n)
    if bc == "P":
        return ((q + 1) // 2) * np.pi / n          # l(q) = ⌈q/2⌉, Nyquist l = n/2
    if bc == "NN":
        return q * np.pi / (2 * n)
    if bc == "DD":
        return (q + 1) * np.pi / (2 * n)
    if bc == "FD":                                 # interior faces: kπ/2n; q = 0 (wall) set below
        return q * np.pi / (2 * n)
    return (2 * q + 1) * np.pi / (4 * n)           # ND, and DN (the reversed ND axis)


def eigenvalues(bc, n):
    """λ_q = −4 sin²(θ_q), Table 1 (dimensionless; divide by Δ² for Eq. 5); for FD the
    wall face's row has λ_0 = −1."""
    lam = -4.0 * np.sin(theta(bc, n)) ** 2
    if bc == "FD":
        lam[0] = -1.0
    return lam


def forward_matrix(bc, n):
    """F with F[q, p] = coefficient of a_p in â_q, Table 2 (DFT rows as read above)."""
    _check(bc, n)
    p = np.arange(n)[None, :]
    q = np.arange(n)[:, None]
    if bc == "P":
        F = np.zeros((n, n))
        F[0, :] = 1.0
        for l in range(1, n // 2):
            F[2 * l - 1, :] = _cos_pi(2 * p[0] * l, n)
            F[2 * l, :] = _sin_pi(2 * p[0] * l, n)
        F[n - 1, :] = (-1.0) ** p[0]
        return F
    if bc == "NN":      # DCT-II: 2 Σ a_p cos(π (p+1/2) q / n)
        return 2.0 * _cos_pi((2 * p + 1) * q, 2 * n)
    if bc == "DD":      # DST-II: 2 Σ a_p sin(π (p+1/2)(q+1) / n)
        return 2.0 * _sin_pi((2 * p + 1) * (q + 1), 2 * n)
    if bc == "DN":      # the ND transform of the reversed line
        return forward_matrix("ND", n)[:, ::-1].copy()
    if bc == "FD":      # wall entry copied; DST-I of the interior faces: 2 Σ a_i sin(π k i / n)
        F = 2.0 * _sin_pi(q * p, n)
        F[0, :] = 0.0
        F[:, 0] = 0.0
        F[0, 0] = 1.0
        return F
    # ND, DCT-IV: 2 Σ a_p cos(π (p+1/2)(q+1/2) / n)
    return 2.0 * _cos_pi((2 * p + 1) * (2 * q + 1), 4 * n)


def backward_matrix(bc, n):
    """B with B[p, q] = weight of â_q in the reconstructed a_p (Table 1 inverse)."""
    _check(bc, n)
    p = np.arange(n)[:, None]
    q = np.arange(n)[None, :]
    if bc == "P":       # (1/n) IDFT, read as in the module docstring
        B = np.zeros((n, n))
        B[:, 0] = 1.0
        for l in range(1, n // 2):
            B[:, 2 * l - 1] = 2.0 * _cos_pi(2 * p[:, 0] * l, n)
            B[:, 2 * l] = 2.0 * _sin_pi(2 * p[:, 0] * l, n)
        B[:, n - 1] = (-1.0) ** p[:, 0]
        return B / n
    if bc == "NN":      # (1/2n) DCT-III: â_0 + 2 Σ_{q≥1} â_q cos(π q (p+1/2) / n)
        B = 2.0 * _cos_pi(q * (2 * p + 1), 2 * n)
        B[:, 0] = 1.0
        return B / (2 * n)
    if bc == "DD":      # (1/2n) DST-III: 2 Σ_{q≤n−2} â_q sin(π (q+1)(p+1/2) / n) + (−1)^p â_{n−1}
        B = 2.0 * _sin_pi((q + 1) * (2 * p + 1), 2 * n)
        B[:, n - 1] = (-1.0) ** p[:, 0]
        return B / (2 * n)
    if bc == "DN":      # ND's inverse, then the reversal
        return backward_matrix("ND", n)[::-1, :].copy()
    if bc == "FD":      # wall entry copied; (1/n) Σ_k â_k sin(π k i / n)
        B = _sin_pi(p * q, n) / n
        B[0, :] = 0.0
        B[:, 0] = 0.0
        B[0, 0] = 1.0
        return B
    # ND: (1/2n) DCT-IV
    return 2.0 * _cos_pi((2 * p + 1) * (2 * q + 1), 4 * n) / (2 * n)


def apply_along(M, a, axis):
    """Apply a matrix M (out×in) along one axis of an array (library matmul as one step)."""
    a = np.moveaxis(a, axis, -1)
    out = a @ M.T
    return np.moveaxis(out, -1, axis)
