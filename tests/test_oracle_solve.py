"""Pins for the oracle's solve (no GPU).

Independent references used:
* dense / sparse LU of the assembled operator (``oracle.direct``) — no transform;
* the dense matrix of a tridiagonal or cyclic system (numpy.linalg.solve);
* closed form for a single eigenmode on a uniform grid (Eq. 5 with Table 1 λ);
* second-order convergence toward analytic solutions (§2: second order in space);
* the stencil apply vs the sparse matrix (two codings of the ghost rules).
"""

import itertools

import numpy as np
import pytest
import scipy.fft as sfft
import scipy.sparse as sp

from oracle import transforms as T
from oracle import operator as O
from oracle import solve as S
from oracle import direct as D
from oracle import tridiag as TD
from paper_1802_10323_gb300 import synth

ALL = list(itertools.product(T.BCS, repeat=3))


def _stretched(n, seed=0):
    rng = np.random.default_rng(seed)
    return np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 1.5, n))])


@pytest.mark.parametrize("bcs", ALL, ids=["-".join(b) for b in ALL])
def test_eigen_solve_equals_dense_lu(bcs):
    zf = _stretched(6, seed=1)
    f = np.random.default_rng(2).uniform(-1, 1, (6, 4, 8))
    p = S.solve(f, 0.3, 0.7, zf, *bcs)
    q = D.solve_direct(f, 0.3, 0.7, zf, *bcs, dense=True)
    assert np.abs(p - q).max() <= 1e-12 * np.abs(q).max()
    assert O.relative_residual(p, f, 0.3, 0.7, zf, *bcs) < 1e-12


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("DD", "ND", "P"), ("NN", "NN", "NN")])
def test_stencil_equals_sparse_matrix(bcs):
    zf = _stretched(5, seed=3)
    x = np.random.default_rng(4).standard_normal((5, 6, 4))
    A = O.operator_3d(4, 6, 0.2, 0.9, zf, *bcs)
    assert np.abs(A @ x.ravel() - O.apply(x, 0.2, 0.9, zf, *bcs).ravel()).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("bcz", T.BCS)
@pytest.mark.parametrize("n", [2, 4, 7, 10])
def test_z_system_is_the_operator(bcz, n):
    zf = _stretched(n, seed=n)
    a, b, c = S.z_system(zf, bcz)
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    if bcz == "P":
        M[0, n - 1] += a[0]
        M[n - 1, 0] += c[n - 1]
    assert np.allclose(M, O.operator_1d(bcz, zf), rtol=0, atol=1e-12 * np.abs(M).max())


@pytest.mark.parametrize("n", [1, 2, 3, 17])
def test_thomas_vs_dense(n):
    rng = np.random.default_rng(n)
    a, c = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    b = -(a + c) - rng.uniform(0.01, 1, n)
    d = rng.standard_normal((n, 3))
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    assert np.allclose(TD.thomas(a, b, c, d), np.linalg.solve(M, d), atol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 16])
def test_cyclic_vs_dense(n):
    rng = np.random.default_rng(n)
    a, c = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    b = -(a + c) - rng.uniform(0.01, 1, n)
    d = rng.standard_normal((n, 2))
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    M[0, n - 1] += a[0]
    M[n - 1, 0] += c[n - 1]
    assert np.allclose(TD.thomas_cyclic(a, b, c, d), np.linalg.solve(M, d), atol=1e-12)


@pytest.mark.parametrize("bcs", [("P", "NN", "DD"), ("ND", "P", "NN"), ("DD", "DD", "ND"), ("P", "P", "P")])
def test_single_mode_closed_form(bcs):
    """f = product of eigenvectors ⇒ Φ = f / (λx/Δx² + λy/Δy² + λz/Δz²)."""
    nx, ny, nz, dx, dy, dz = 8, 6, 10, 0.25, 0.5, 0.1
    qx, qy, qz = 3, 1, 2
    if bcs == ("P", "P", "P"):
        qx = 5
    ex = T.backward_matrix(bcs[0], nx)[:, qx]
    ey = T.backward_matrix(bcs[1], ny)[:, qy]
    ez = T.backward_matrix(bcs[2], nz)[:, qz]
    f = ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    lam = (T.eigenvalues(bcs[0], nx)[qx] / dx ** 2 + T.eigenvalues(bcs[1], ny)[qy] / dy ** 2
           + T.eigenvalues(bcs[2], nz)[qz] / dz ** 2)
    p = S.solve(f, dx, dy, O.uniform_faces(nz, dz), *bcs)
    assert np.abs(p - f / lam).max() < 1e-13 * np.abs(f / lam).max()


@pytest.mark.parametrize("bcs", [("P", "NN", "DD"), ("ND", "DD", "NN"), ("NN", "P", "ND"), ("P", "P", "NN"),
                                 ("DN", "P", "DN"), ("NN", "DN", "ND")])
def test_second_order_convergence(bcs):
    errs, hs = [], []
    for n in (16, 32, 64):
        zf = synth.tanh_faces(n, 1.0, 1.5)
        p_ex, f = synth.manufactured(n, n, 1.0, 2.0, zf, bcs)
        p = S.solve(f, 1.0 / n, 2.0 / n, zf, *bcs)
        if O.is_singular(*bcs):
            v = O.cell_volumes(n, n, 1.0 / n, 2.0 / n, zf)
            p_ex = p_ex - (v * p_ex).sum() / v.sum()
        errs.append(np.abs(p - p_ex).max())
        hs.append(1.0 / n)
    orders = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(2.0)
    assert orders.min() >= 1.9, orders


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("NN", "NN", "NN"), ("P", "NN", "P"), ("P", "P", "P")])
def test_singular_zero_mean_and_compatible_part(bcs):
    zf = synth.tanh_faces(8, 1.0, 1.5) if bcs[2] != "P" else O.uniform_faces(8, 0.125)
    f = np.random.default_rng(7).uniform(-1, 1, (8, 6, 4)) + 0.3   # has a mean
    p = S.solve(f, 0.25, 0.2, zf, *bcs)
    v = O.cell_volumes(4, 6, 0.25, 0.2, zf)
    assert abs((v * p).sum()) < 1e-13 * np.abs(p).max() * v.sum()
    fc = O.compatible_part(f, 0.25, 0.2, zf, *bcs)
    assert abs((v * fc).sum()) < 1e-13 * v.sum()
    assert O.relative_residual(p, f, 0.25, 0.2, zf, *bcs) < 1e-12


def test_small_channel_32_cubed_vs_sparse_lu():
    """32³, P/P/NN, uniform unit cube, U[−1,1] mean-removed (the small FP64 case)."""
    n = 32
    f = synth.uniform_noise((n, n, n), seed=0)
    zf = O.uniform_faces(n, 1.0 / n)
    p = S.solve(f, 1.0 / n, 1.0 / n, zf, "P", "P", "NN")
    q = D.solve_direct(f, 1.0 / n, 1.0 / n, zf, "P", "P", "NN")
    assert np.abs(p - q).max() <= 1e-12 * np.abs(q).max()


@pytest.mark.parametrize("n", [2, 4])
def test_tiny_grids(n):
    for bcs in [("P", "P", "P"), ("DD", "ND", "NN"), ("NN", "NN", "P")]:
        zf = _stretched(n, seed=9)
        f = np.random.default_rng(n).standard_normal((n, n, n))
        p = S.solve(f, 0.5, 0.5, zf, *bcs)
        q = D.solve_direct(f, 0.5, 0.5, zf, *bcs, dense=True)
        assert np.abs(p - q).max() <= 1e-12 * max(np.abs(q).max(), 1e-300)


def test_golden_nonuniform_operator():
    """Hand-worked 1D operator rows on faces 0, 1, 3, 6 (tests/golden)."""
    import os
    from fractions import Fraction
    path = os.path.join(os.path.dirname(__file__), "golden", "operator_faces_0_1_3_6.txt")
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        bc, *vals = line.split()
        expect = np.array([float(Fraction(v)) for v in vals]).reshape(3, 3)
        got = O.operator_1d(bc, np.array([0.0, 1.0, 3.0, 6.0]))
        assert np.abs(got - expect).max() < 1e-15, bc
        a, b, c = S.z_system(np.array([0.0, 1.0, 3.0, 6.0]), bc)
        M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        if bc == "P":
            M[0, 2] += a[0]
            M[2, 0] += c[2]
        assert np.abs(M - expect).max() < 1e-15, bc


# ---- Helmholtz variant: (A − α) p = f, α > 0 (§2: implicit diffusion; §4) ----

HELM = [("P", "P", "NN"), ("NN", "NN", "NN"), ("P", "P", "P"), ("DD", "ND", "P"), ("ND", "NN", "DD")]


@pytest.mark.parametrize("alpha", [0.37, 25.0])
@pytest.mark.parametrize("bcs", HELM, ids=["-".join(b) for b in HELM])
def test_helmholtz_eigen_solve_equals_dense_lu(bcs, alpha):
    """The shift enters the eigen-expansion as −α on every Eq. 5 diagonal and the
    assembled matrix as −α·I: two codings that must agree. With α > 0 the all-P/NN
    triples are regular: the LU is unbordered and f keeps its mean."""
    zf = _stretched(6, seed=11)
    f = np.random.default_rng(12).uniform(-1, 1, (6, 4, 8)) + 0.3
    p = S.solve(f, 0.3, 0.7, zf, *bcs, alpha=alpha)
    q = D.solve_direct(f, 0.3, 0.7, zf, *bcs, dense=True, alpha=alpha)
    assert np.abs(p - q).max() <= 1e-12 * np.abs(q).max()
    r = f - O.apply(p, 0.3, 0.7, zf, *bcs, alpha=alpha)
    assert np.abs(r).max() < 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("bcs", [("P", "NN", "DD"), ("ND", "P", "NN"), ("P", "P", "P")])
def test_helmholtz_single_mode_closed_form(bcs):
    """f = product of eigenvectors ⇒ p = f / (λx/Δx² + λy/Δy² + λz/Δz² − α)."""
    nx, ny, nz, dx, dy, dz, alpha = 8, 6, 10, 0.25, 0.5, 0.1, 7.5
    qx, qy, qz = 3, 1, 2
    ex = T.backward_matrix(bcs[0], nx)[:, qx]
    ey = T.backward_matrix(bcs[1], ny)[:, qy]
    ez = T.backward_matrix(bcs[2], nz)[:, qz]
    f = ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    lam = (T.eigenvalues(bcs[0], nx)[qx] / dx ** 2 + T.eigenvalues(bcs[1], ny)[qy] / dy ** 2
           + T.eigenvalues(bcs[2], nz)[qz] / dz ** 2) - alpha
    p = S.solve(f, dx, dy, O.uniform_faces(nz, dz), *bcs, alpha=alpha)
    assert np.abs(p - f / lam).max() < 1e-13 * np.abs(f / lam).max()


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("NN", "P", "P"), ("NN", "NN", "NN")])
def test_helmholtz_constant_closed_form(bcs):
    """Constants are harmonic under P/NN ends (stretched z too), so f ≡ c gives p ≡ −c/α."""
    zf = _stretched(7, seed=13)
    f = np.full((7, 6, 4), 2.5)
    p = S.solve(f, 0.4, 0.2, zf, *bcs, alpha=3.0)
    assert np.abs(p + 2.5 / 3.0).max() < 1e-14


def test_helmholtz_stencil_equals_sparse_matrix():
    zf = _stretched(5, seed=14)
    x = np.random.default_rng(15).standard_normal((5, 6, 4))
    bcs = ("DD", "P", "ND")
    A = O.operator_3d(4, 6, 0.2, 0.9, zf, *bcs, alpha=4.25)
    assert np.abs(A @ x.ravel() - O.apply(x, 0.2, 0.9, zf, *bcs, alpha=4.25).ravel()).max() < 1e-12


# ---- face-centred z ("FD"): the wall-normal velocity of an implicit diffusion step ----

@pytest.mark.parametrize("bcxy", [("P", "P"), ("DD", "NN"), ("ND", "DN")])
@pytest.mark.parametrize("alpha", [0.0, 12.0])
def test_fd_eigen_solve_equals_dense_lu_and_codings(bcxy, alpha):
    zf = _stretched(7, seed=21)
    f = np.random.default_rng(22).uniform(-1, 1, (7, 4, 6))
    f[0] = 0.0                                   # the bottom wall face carries no equation
    bcs = (bcxy[0], bcxy[1], "FD")
    p = S.solve(f, 0.3, 0.7, zf, *bcs, alpha=alpha)
    q = D.solve_direct(f, 0.3, 0.7, zf, *bcs, dense=True, alpha=alpha)
    assert np.abs(p - q).max() <= 1e-12 * np.abs(q).max()
    assert np.abs(p[0]).max() <= 1e-12 * np.abs(q).max()
    r = f - O.apply(p, 0.3, 0.7, zf, *bcs, alpha=alpha)
    assert np.abs(r).max() < 1e-11 * np.abs(f).max()
    a, b, c = S.z_system(zf, "FD")
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    assert np.abs(O.operator_1d("FD", zf) - M).max() < 1e-12 * np.abs(M).max()


def test_fd_single_mode_closed_form():
    """Uniform z: the face system with zero wall nodes has the sine modes sin(πqk/n)
    (a DST-I basis) with λ_z = −4 sin²(πq/2n)/Δz², so p = f/(λ_x + λ_y + λ_z − α)."""
    nx, ny, nz, dx, dy, dz, alpha = 8, 6, 10, 0.25, 0.5, 0.1, 2.0
    qx, qy, qz = 3, 2, 4
    ex = T.backward_matrix("P", nx)[:, qx]
    ey = T.backward_matrix("NN", ny)[:, qy]
    ez = np.sin(np.pi * qz * np.arange(nz) / nz)
    f = ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    lam = (T.eigenvalues("P", nx)[qx] / dx ** 2 + T.eigenvalues("NN", ny)[qy] / dy ** 2
           - 4 * np.sin(np.pi * qz / (2 * nz)) ** 2 / dz ** 2) - alpha
    p = S.solve(f, dx, dy, O.uniform_faces(nz, dz), "P", "NN", "FD", alpha=alpha)
    assert np.abs(p - f / lam).max() < 1e-13 * np.abs(f / lam).max()


def test_fd_planted_control_volume_mistake_is_caught(monkeypatch):
    """Dividing the face rows by the cell width instead of the centre distance: the
    dense LU of the assembled operator no longer matches the eigen-expansion solve."""
    orig = O.operator_1d_faces

    def wrong(faces):
        L = orig(faces)
        dzf, dzc = O.metrics(faces)
        L[1:] *= (dzc / dzf[1:])[:, None]
        return L

    monkeypatch.setattr(O, "operator_1d_faces", wrong)
    with pytest.raises(AssertionError):
        test_fd_eigen_solve_equals_dense_lu_and_codings(("P", "P"), 12.0)


# ---- face-centred x and y ("FD" on a transformed axis): DST-I-type transforms ----

@pytest.mark.parametrize("n", [2, 4, 8, 12, 18])
def test_fd_xy_transform_is_dst1(n):
    """The interior block of the forward FD transform is scipy's DST type I (a library
    special case); the wall entry is copied; backward · forward = I."""
    F, B = T.forward_matrix("FD", n), T.backward_matrix("FD", n)
    assert np.abs(F[1:, 1:] - sfft.dst(np.eye(n - 1), type=1, axis=0)).max() < 1e-13 * n
    assert F[0, 0] == 1.0 and not F[0, 1:].any() and not F[1:, 0].any()
    assert np.abs(B @ F - np.eye(n)).max() < 1e-13


@pytest.mark.parametrize("n,h", [(4, 0.5), (10, 0.13), (16, 1.0)])
def test_fd_xy_eigen_identity(n, h):
    """F·L·F⁻¹ = diag(λ/h²) for the node operator with λ_0 = −1, λ_k = −4 sin²(πk/2n)."""
    L = O.operator_1d("FD", O.uniform_faces(n, h), axis="xy")
    M = T.forward_matrix("FD", n) @ L @ T.backward_matrix("FD", n)
    lam = T.eigenvalues("FD", n) / h ** 2
    assert np.abs(M - np.diag(lam)).max() < 1e-12 * np.abs(lam).max()
    k = np.arange(1, n)
    assert np.allclose(lam[1:], -4 * np.sin(np.pi * k / (2 * n)) ** 2 / h ** 2, rtol=1e-14, atol=0)


FDXY = [("FD", "P", "NN"), ("NN", "FD", "DD"), ("FD", "FD", "P"), ("FD", "DN", "FD"),
        ("DD", "FD", "ND"), ("FD", "FD", "FD")]


@pytest.mark.parametrize("bcs", FDXY)
@pytest.mark.parametrize("alpha", [0.0, 7.5])
def test_fd_xy_eigen_solve_equals_dense_lu_and_codings(bcs, alpha):
    zf = _stretched(6, seed=31)
    f = np.random.default_rng(32).uniform(-1, 1, (6, 8, 10))
    p = S.solve(f, 0.3, 0.7, zf, *bcs, alpha=alpha)
    q = D.solve_direct(f, 0.3, 0.7, zf, *bcs, dense=True, alpha=alpha)
    assert np.abs(p - q).max() <= 1e-12 * np.abs(q).max()
    r = f - O.apply(p, 0.3, 0.7, zf, *bcs, alpha=alpha)
    assert np.abs(r).max() < 1e-11 * np.abs(f).max()
    A = O.operator_3d(10, 8, 0.3, 0.7, zf, *bcs, alpha=alpha)
    if bcs[2] != "FD":  # the x/y parts are symmetric (the z part is under the Δz^f weight)
        W = sp.diags(np.repeat(np.diff(zf), 80))
        assert abs(W @ A - (W @ A).T).max() < 1e-9 * abs(W @ A).max()


def test_fd_xy_wall_contract():
    """f = 0 on the wall faces gives u = 0 there, and then the first interior row
    seeing the stored wall entry (the z rule) or the wall node 0 is the same."""
    zf = O.uniform_faces(6, 0.2)
    f = np.random.default_rng(33).uniform(-1, 1, (6, 8, 10))
    f[:, :, 0] = 0.0
    f[:, 0, :] = 0.0
    p = S.solve(f, 0.3, 0.7, zf, "FD", "FD", "NN")
    assert np.abs(p[:, :, 0]).max() == 0.0 and np.abs(p[:, 0, :]).max() == 0.0


def test_fd_xy_second_order_convergence():
    """u = sin(πx) sin(2πy)·cos(πz) with x and y on faces (walls at 0 and 1 on both)
    and z cell-centred Neumann: the discrete solution converges at second order."""
    err = []
    for n in (8, 16, 32):
        h = 1.0 / n
        xf = np.arange(n) * h                        # faces 0 … n−1 (face 0 the wall)
        zc = (np.arange(n) + 0.5) * h
        Z, Y, X = np.meshgrid(zc, xf, xf, indexing="ij")
        u = np.sin(np.pi * X) * np.sin(2 * np.pi * Y) * np.cos(np.pi * Z)
        f = -(np.pi ** 2 + 4 * np.pi ** 2 + np.pi ** 2) * u
        p = S.solve(f, h, h, O.uniform_faces(n, h), "FD", "FD", "NN")
        err.append(np.abs(p - u).max())
    assert err[1] < 0.3 * err[0] and err[2] < 0.3 * err[1], err


def test_fd_xy_planted_mistakes_are_caught(monkeypatch):
    """A sine index off by one in the FD eigenvalues fails the eigen identity; the wall
    row coupled into the first interior row (the z rule) in the matrix but not in the
    stencil fails the agreement of the two codings."""
    orig = T.eigenvalues

    def shifted(bc, n):
        lam = orig(bc, n)
        if bc == "FD":
            k = np.arange(1, n) + 1
            lam = lam.copy()
            lam[1:] = -4 * np.sin(np.pi * k / (2 * n)) ** 2
        return lam

    monkeypatch.setattr(T, "eigenvalues", shifted)
    with pytest.raises(AssertionError):
        test_fd_xy_eigen_identity(10, 0.13)
    monkeypatch.setattr(T, "eigenvalues", orig)
    orig_nodes = O.operator_1d_nodes

    def coupled(n, h):
        L = orig_nodes(n, h)
        L[1, 0] = 1.0 / h ** 2
        return L

    monkeypatch.setattr(O, "operator_1d_nodes", coupled)
    with pytest.raises(AssertionError):
        test_fd_xy_eigen_solve_equals_dense_lu_and_codings(("FD", "P", "NN"), 0.0)
