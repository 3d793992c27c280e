"""Pins for the oracle's transpose solve and projection (no GPU).

* The transpose solve (W·M·W⁻¹) is checked against the explicit transpose of the
  solve map M, built column by column on tiny grids (brute force).
* D·G equals the assembled operator (A = D G on the MAC grid).
* The projection leaves a divergence-free field and is idempotent.
* The vector–Jacobian product passes the dot-product test and matches central
  finite differences of a scalar loss.
"""

import itertools

import numpy as np
import pytest

from oracle import operator as O
from oracle import solve as S
from oracle import adjoint as AD
from paper_1802_10323_gb300 import synth

PN = list(itertools.product(("P", "NN"), repeat=3))


def _dense_solve_map(nx, ny, zf, dx, dy, bcs):
    nz = len(zf) - 1
    N = nx * ny * nz
    M = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        M[:, c] = S.solve(e.reshape(nz, ny, nx), dx, dy, zf, *bcs).ravel()
    return M


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("DD", "ND", "NN"), ("NN", "NN", "NN"), ("P", "DD", "ND")])
def test_transpose_solve_is_explicit_transpose(bcs):
    zf = synth.tanh_faces(4, 1.0, 1.5)
    M = _dense_solve_map(4, 2, zf, 0.3, 0.6, bcs)
    g = np.random.default_rng(0).standard_normal((4, 2, 4))
    got = AD.solve_transpose(g, 0.3, 0.6, zf, *bcs)
    assert np.abs(got.ravel() - M.T @ g.ravel()).max() < 1e-12 * np.abs(M).max() * np.abs(g).max() * 10


@pytest.mark.parametrize("bcs", PN, ids=["-".join(b) for b in PN])
def test_divergence_of_gradient_is_operator(bcs):
    zf = synth.tanh_faces(4, 1.0, 1.5) if bcs[2] != "P" else O.uniform_faces(4, 0.25)
    Dm = AD.divergence_matrix(4, 6, 0.3, 0.2, zf, *bcs)
    Gm = AD.gradient_matrix(4, 6, 0.3, 0.2, zf, *bcs)
    A = O.operator_3d(4, 6, 0.3, 0.2, zf, *bcs)
    assert abs(Dm @ Gm - A).max() < 1e-10 * abs(A).max()


def _field(nx, ny, nz, seed, bcs):
    u = np.random.default_rng(seed).standard_normal((3, nz, ny, nx))
    for comp, ax in enumerate((2, 1, 0)):
        if bcs[comp] != "P":
            sl = [slice(None)] * 3
            sl[ax] = 0
            u[comp][tuple(sl)] = 0.0       # wall faces carry no flux
    return u


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("NN", "NN", "NN"), ("P", "NN", "P")])
def test_projection_divergence_free_and_idempotent(bcs):
    nx, ny, nz = 6, 4, 8
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else O.uniform_faces(nz, 1.0 / nz)
    u = _field(nx, ny, nz, 1, bcs)
    pu = AD.project(u, 0.2, 0.3, zf, *bcs)
    Dm = AD.divergence_matrix(nx, ny, 0.2, 0.3, zf, *bcs)
    assert np.abs(Dm @ pu.ravel()).max() < 1e-11 * np.abs(Dm @ u.ravel()).max()
    assert np.abs(AD.project(pu, 0.2, 0.3, zf, *bcs) - pu).max() < 1e-12 * np.abs(pu).max()


def test_projection_vjp_dot_product_and_fd():
    bcs = ("P", "P", "NN")
    nx, ny, nz = 4, 4, 6
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    rng = np.random.default_rng(3)
    u = _field(nx, ny, nz, 4, bcs)
    g = rng.standard_normal(u.shape)
    lhs = (AD.project(u, 0.25, 0.25, zf, *bcs) * g).sum()
    rhs = (u * AD.project_vjp(g, 0.25, 0.25, zf, *bcs)).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # central differences of L(u) = Σ g ⊙ P(u) along a random direction
    d = rng.standard_normal(u.shape)
    h = 1e-6
    fd = ((AD.project(u + h * d, 0.25, 0.25, zf, *bcs) * g).sum()
          - (AD.project(u - h * d, 0.25, 0.25, zf, *bcs) * g).sum()) / (2 * h)
    an = (AD.project_vjp(g, 0.25, 0.25, zf, *bcs) * d).sum()
    assert abs(fd - an) < 1e-6 * abs(an)


@pytest.mark.parametrize("bcs", [("P", "P", "NN"), ("DD", "ND", "NN")])
def test_helmholtz_transpose_solve_is_explicit_transpose(bcs):
    """A − α = W⁻¹(S − αW) with S − αW symmetric: the same W·M·W⁻¹ rule holds."""
    zf = synth.tanh_faces(4, 1.0, 1.5)
    nz, ny, nx, alpha = 4, 2, 4, 6.0
    N = nx * ny * nz
    M = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        M[:, c] = S.solve(e.reshape(nz, ny, nx), 0.3, 0.6, zf, *bcs, alpha=alpha).ravel()
    g = np.random.default_rng(1).standard_normal((nz, ny, nx))
    got = AD.solve_transpose(g, 0.3, 0.6, zf, *bcs, alpha=alpha)
    assert np.abs(got.ravel() - M.T @ g.ravel()).max() < 1e-12 * np.abs(M).max() * np.abs(g).max() * 10
