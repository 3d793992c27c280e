"""Planted mistakes: each plausible slip in the oracle must fail one of its pins.

Every case monkeypatches one oracle function with a realistic error (dropped
term, wrong sign, wrong index, transposed operand) and checks that at least one
independent reference (scipy transforms, dense LU, closed forms) catches it.
This runs on the CPU only and touches nothing outside ``oracle``.
"""

import numpy as np
import pytest
import scipy.fft as sfft

from oracle import transforms as T
from oracle import operator as O
from oracle import solve as S
from oracle import direct as D
from oracle import tridiag as TD


def _pins_fail():
    """Compact re-run of the pins; returns True when any of them fails."""
    n = 8
    for bc, kind, typ in (("NN", "dct", 2), ("DD", "dst", 2), ("ND", "dct", 4)):
        if np.abs(T.forward_matrix(bc, n) - getattr(sfft, kind)(np.eye(n), type=typ, axis=0)).max() > 1e-12:
            return True
    for bc in T.BCS:
        if np.abs(T.backward_matrix(bc, n) @ T.forward_matrix(bc, n) - np.eye(n)).max() > 1e-12:
            return True
        L = O.operator_1d(bc, O.uniform_faces(n, 1.0))
        M = T.forward_matrix(bc, n) @ L @ T.backward_matrix(bc, n)
        if np.abs(M - np.diag(T.eigenvalues(bc, n))).max() > 1e-10:
            return True
    rng = np.random.default_rng(0)
    zf = np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 1.5, 6))])
    for bcs in (("P", "NN", "DD"), ("ND", "DD", "P"), ("P", "P", "NN"), ("NN", "DD", "ND")):
        f = rng.uniform(-1, 1, (6, 4, 8))
        p = S.solve(f, 0.3, 0.7, zf, *bcs)
        q = D.solve_direct(f, 0.3, 0.7, zf, *bcs, dense=True)
        if not np.all(np.isfinite(p)) or np.abs(p - q).max() > 1e-10 * np.abs(q).max():
            return True
    for bcs in (("P", "NN", "NN"), ("DD", "P", "ND")):  # Helmholtz: α > 0
        f = rng.uniform(-1, 1, (6, 4, 8)) + 0.3
        p = S.solve(f, 0.3, 0.7, zf, *bcs, alpha=2.5)
        q = D.solve_direct(f, 0.3, 0.7, zf, *bcs, dense=True, alpha=2.5)
        if not np.all(np.isfinite(p)) or np.abs(p - q).max() > 1e-10 * np.abs(q).max():
            return True
        if np.abs(O.apply(p, 0.3, 0.7, zf, *bcs, alpha=2.5) - f).max() > 1e-10 * np.abs(f).max():
            return True
    from fractions import Fraction
    exp = {"NN": "-2/3 2/3 0 1/3 -8/15 1/5 0 2/15 -2/15", "DD": "-8/3 2/3 0 1/3 -8/15 1/5 0 2/15 -16/45"}
    for bc, row in exp.items():
        e = np.array([float(Fraction(v)) for v in row.split()]).reshape(3, 3)
        if np.abs(O.operator_1d(bc, np.array([0.0, 1.0, 3.0, 6.0])) - e).max() > 1e-14:
            return True
    return False


def test_unmutated_oracle_passes():
    assert not _pins_fail()


def _transposed_forward(orig):
    return lambda bc, n: orig(bc, n).T


def _flip_sin_rows(orig):
    def f(bc, n):
        B = orig(bc, n).copy()
        if bc == "P":
            B[:, 2:n - 1:2] *= -1.0
        return B
    return f


def _shift_theta(orig):
    def f(bc, n):
        th = orig(bc, n)
        return th + (np.pi / (2 * n) if bc == "DD" else 0.0)
    return f


def _drop_dirichlet_term(orig):
    def f(zf, bcz):
        a, b, c = orig(zf, bcz)
        dzf = np.diff(zf)
        b = b.copy()
        if bcz in ("DD", "ND"):
            b[-1] += 2.0 / dzf[-1] ** 2
        return a, b, c
    return f


def _wrong_backsub(orig):
    def f(a, b, c, d):
        x = orig(a, b, c, d)
        return x + 1e-6 * np.roll(x, 1, axis=0)
    return f


def _no_mean_removal(orig):
    def f(a, b, c, d, dzf):
        x = np.zeros_like(d)
        x[1:] = TD.thomas(a[1:], b[1:], c[1:], d[1:])
        return x
    return f


def _swap_metric(orig):
    def f(faces):
        dzf, dzc = orig(faces)
        return dzf[::-1].copy(), dzc
    return f


def _dn_ends_swapped(orig):
    def f(bc):
        return ("N", "D") if bc == "DN" else orig(bc)
    return f


def _flip_alpha(orig):
    def f(nx, ny, dx, dy, zf, bcx, bcy, bcz, alpha=0.0):
        return orig(nx, ny, dx, dy, zf, bcx, bcy, bcz, -alpha)
    return f


def _drop_alpha(orig):
    def f(p, dx, dy, zf, bcx, bcy, bcz, alpha=0.0):
        return orig(p, dx, dy, zf, bcx, bcy, bcz, 0.0)
    return f


def _singular_ignores_alpha(orig):
    def f(bcx, bcy, bcz, alpha=0.0):
        return orig(bcx, bcy, bcz, 0.0)
    return f


MUTATIONS = [
    ("transposed forward matrix", T, "forward_matrix", _transposed_forward),
    ("wrong sign of periodic sine rows", T, "backward_matrix", _flip_sin_rows),
    ("DD eigenvalue index off by one", T, "theta", _shift_theta),
    ("dropped Dirichlet ghost term in z", S, "z_system", _drop_dirichlet_term),
    ("perturbed back substitution", S, "thomas", _wrong_backsub),
    ("singular column mean not removed", S, "_singular_column", _no_mean_removal),
    ("reversed cell widths", O, "metrics", _swap_metric),
    ("DN ends swapped (read as ND) in the ghost rules", O, "_ends", _dn_ends_swapped),
    ("Helmholtz shift with the wrong sign in the assembled operator", O, "operator_3d", _flip_alpha),
    ("Helmholtz shift dropped from the stencil", O, "apply", _drop_alpha),
    ("singular-mode treatment kept for a Helmholtz shift", O, "is_singular", _singular_ignores_alpha),
]


@pytest.mark.parametrize("name,mod,attr,mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, mod, attr, mut):
    orig = getattr(mod, attr)
    monkeypatch.setattr(mod, attr, mut(orig))
    # modules that imported the name directly see the mutation too
    for other in (T, O, S, D, TD):
        if getattr(other, attr, None) is orig:
            monkeypatch.setattr(other, attr, mut(orig))
    if attr == "_singular_column":
        zf = O.uniform_faces(6, 1.0 / 6)
        f = np.random.default_rng(1).uniform(-1, 1, (6, 4, 4)) + 0.5
        p = S.solve(f, 0.25, 0.25, zf, "P", "NN", "NN")
        v = O.cell_volumes(4, 4, 0.25, 0.25, zf)
        assert abs((v * p).sum()) > 1e-10 or _pins_fail()
    else:
        assert _pins_fail(), name
