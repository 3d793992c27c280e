"""FP64 CPU oracle for the eigenfunction-expansion Poisson solve (Costa 2018, §2.1).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it. It
shares no code with the CUDA library (no kernels, tables, constants or helpers);
the only thing both sides use is the seeded input generator module, which holds
none of the method's arithmetic.

Everything here is plain NumPy in float64, written to be checked against the
paper by eye:

* ``transforms``  – Table 1 eigenvalues and the Table 2 forward/backward
  transforms as dense n×n matrices (with the reading of the garbled DFT rows
  stated there).
* ``operator``    – the 7-point operator of Eq. 4 built from ghost-cell rules
  (staggered BCs, finite-volume stretched z), as 1D matrices, a sparse 3D
  matrix and a stencil apply.
* ``tridiag``     – Gauss elimination (Thomas) per column and the cyclic variant
  reduced to two tridiagonal solves (§3).
* ``solve``       – the 3-step solve of §2.1: transform x and y, N_x·N_y
  tridiagonal solves of Eq. 5, inverse transforms; singular-mode handling.
* ``direct``      – the same discrete system solved directly by (sparse or
  dense) LU of the assembled operator, with no transform involved.
* ``adjoint``     – transpose solve and the staggered divergence/gradient of the
  projection step (Eqs. 2b–2c).

Parity status of every function is stated in its docstring; each is pinned by
a ``-m "not gpu"`` test against closed forms, library special cases or brute
force.
"""

from . import transforms, operator, tridiag, solve, direct, adjoint  # noqa: F401
