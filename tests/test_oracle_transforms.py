"""Pins for the oracle's Table 1 / Table 2 code (no GPU).

What fixes each value independently of the oracle's own formulas:
* scipy.fft's DCT/DST types II, III, IV (norm=None) are Table 2's transforms;
* numpy's rfft gives the periodic rows in the half-complex layout;
* hand-derived n = 4 values (tests/golden, trig identities);
* the 1D operator, built from ghost-cell rules with no transform, must be
  diagonalised by F with Table 1's eigenvalues.
"""

import math
import os

import numpy as np
import pytest
import scipy.fft as sfft

from oracle import transforms as T
from oracle import operator as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SIZES = [2, 4, 6, 8, 12, 16, 24, 48]


def _expr(s):
    return float(eval(s, {"sqrt": math.sqrt, "__builtins__": {}}))


def _golden_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line)
    return rows


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("bc,kind,typ", [("NN", "dct", 2), ("DD", "dst", 2), ("ND", "dct", 4)])
def test_forward_is_scipy(bc, kind, typ, n):
    F = T.forward_matrix(bc, n)
    ref = getattr(sfft, kind)(np.eye(n), type=typ, axis=0)
    assert np.abs(F - ref).max() < 1e-13 * n


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("bc,kind,typ", [("NN", "dct", 3), ("DD", "dst", 3), ("ND", "dct", 4)])
def test_backward_is_scaled_scipy(bc, kind, typ, n):
    B = T.backward_matrix(bc, n)
    ref = getattr(sfft, kind)(np.eye(n), type=typ, axis=0) / (2 * n)
    assert np.abs(B - ref).max() < 1e-14 * n


@pytest.mark.parametrize("n", SIZES)
def test_dn_is_signed_scipy_dst4(n):
    """DN (not in Table 1, read as ND on the reversed axis): reversing a DCT-IV's input
    gives (−1)^q times the DST-IV, so F_DN = diag((−1)^q)·DST-IV and B_DN = DST-IV·diag((−1)^q)/2n."""
    sgn = (-1.0) ** np.arange(n)
    dst4 = sfft.dst(np.eye(n), type=4, axis=0)
    assert np.abs(T.forward_matrix("DN", n) - sgn[:, None] * dst4).max() < 1e-13 * n
    assert np.abs(T.backward_matrix("DN", n) - dst4 * sgn[None, :] / (2 * n)).max() < 1e-14 * n


@pytest.mark.parametrize("n", SIZES)
def test_periodic_rows_are_rfft(n):
    X = np.fft.rfft(np.eye(n), axis=0)
    ref = np.zeros((n, n))
    ref[0] = X[0].real
    for l in range(1, n // 2):
        ref[2 * l - 1] = X[l].real
        ref[2 * l] = -X[l].imag
    ref[n - 1] = X[n // 2].real
    assert np.abs(T.forward_matrix("P", n) - ref).max() < 1e-13 * n


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("bc", T.BCS)
def test_round_trip(bc, n):
    assert np.abs(T.backward_matrix(bc, n) @ T.forward_matrix(bc, n) - np.eye(n)).max() < 1e-13 * n


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("bc", T.BCS)
def test_eigen_identity(bc, n):
    """F · L · F⁻¹ = diag(λ): the ghost-cell operator is diagonalised (Eq. 5)."""
    L = O.operator_1d(bc, O.uniform_faces(n, 1.0))
    M = T.forward_matrix(bc, n) @ L @ T.backward_matrix(bc, n)
    assert np.abs(M - np.diag(T.eigenvalues(bc, n))).max() < 1e-12 * n


def test_golden_eigenvalues_n4():
    for row in _golden_rows("eigenvalues_n4.txt"):
        bc, *vals = row.split()
        expect = np.array([_expr(v) for v in vals])
        assert np.abs(T.eigenvalues(bc, 4) - expect).max() < 1e-14, bc


def test_golden_transforms_n4():
    for row in _golden_rows("dct2_n4.txt"):
        bc, inp, out = row.split(None, 2)
        a = np.array([float(x) for x in inp.split(",")])
        expect = np.array([_expr(x) for x in out.split(",")])
        assert np.abs(T.forward_matrix(bc, 4) @ a - expect).max() < 1e-14, bc


@pytest.mark.parametrize("bc", T.BCS)
def test_odd_or_tiny_n_rejected(bc):
    for n in (0, 1, 3, 7):
        with pytest.raises(ValueError):
            T.forward_matrix(bc, n)
