"""The C-ABI library loads, exports every symbol its header declares, and
rejects invalid plans on the host (no GPU needed for any of this)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            names |= set(re.findall(r"^(?:ps_status|const char\*|int)\s+(ps_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def binding():
    from paper_1802_10323_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1802_10323_gb300 import binding as b
    return b


def test_every_declared_symbol_is_exported(binding):
    declared = _declared()
    assert len(declared) >= 12
    lib = ctypes.CDLL(binding.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(binding.EXPORTS)


@pytest.mark.parametrize("n,status", [(0, 2), (3, 2), (7, 2), (16384, 2), (10, 2), (14, 2), (5120, 2)])
def test_unsupported_sizes_rejected(binding, n, status):
    h = ctypes.c_void_p()
    st = binding.ps_plan_create(ctypes.byref(h), n, 8, 8, 1.0, 1.0, None, 1.0, 0, 0, 1, 0, 1e-10, 3)
    assert st == status
    assert not h.value
    assert b"n/2" in binding.ps_last_error(None) or b"nx" in binding.ps_last_error(None)


@pytest.mark.parametrize("kw", [dict(dx=0.0), dict(dz=-1.0), dict(bcx=7), dict(prec=9),
                                dict(prec=2, rtol=0.0), dict(prec=2, max_iter=-1)])
def test_invalid_arguments_rejected(binding, kw):
    a = dict(nx=8, ny=8, nz=8, dx=1.0, dy=1.0, dz=1.0, bcx=0, bcy=0, bcz=1, prec=0, rtol=1e-10, max_iter=3)
    a.update(kw)
    h = ctypes.c_void_p()
    st = binding.ps_plan_create(ctypes.byref(h), a["nx"], a["ny"], a["nz"], a["dx"], a["dy"], None,
                                a["dz"], a["bcx"], a["bcy"], a["bcz"], a["prec"], a["rtol"], a["max_iter"])
    assert st == binding.PS_INVALID_ARG
    assert not h.value


def test_non_increasing_faces_rejected(binding):
    zf = (ctypes.c_double * 5)(0.0, 1.0, 1.0, 2.0, 3.0)
    h = ctypes.c_void_p()
    st = binding.ps_plan_create(ctypes.byref(h), 8, 8, 4, 1.0, 1.0, ctypes.cast(zf, ctypes.c_void_p),
                                0.0, 0, 0, 1, 0, 1e-10, 3)
    assert st == binding.PS_INVALID_ARG


def test_null_arguments(binding):
    assert binding.ps_plan_create(None, 8, 8, 8, 1.0, 1.0, None, 1.0, 0, 0, 1, 0, 1e-10, 3) == binding.PS_INVALID_ARG
    assert binding.ps_solve(None, None, None, None, None, None) == binding.PS_INVALID_ARG
    assert binding.ps_plan_destroy(None) == binding.PS_OK
    n = ctypes.c_size_t()
    assert binding.ps_workspace_bytes(None, ctypes.byref(n)) == binding.PS_INVALID_ARG


@pytest.mark.parametrize("alpha", [-1.0, float("inf"), float("nan")])
def test_helmholtz_shift_validated(binding, alpha):
    h = ctypes.c_void_p()
    st = binding.ps_plan_create_helmholtz(ctypes.byref(h), 8, 8, 8, 1.0, 1.0, None, 1.0, 0, 0, 1, 0,
                                          1e-10, 3, alpha)
    assert st == binding.PS_INVALID_ARG
    assert not h.value
    assert b"alpha" in binding.ps_last_error(None)


def test_ns_substep_null_plan(binding):
    assert binding.ps_ns_substep(None, 1, 1e-3, 0.0, None, None, None, None, None, None, None, None,
                                 None) == binding.PS_INVALID_ARG


def test_host_sequence_null_plan(binding):
    """ps_solve_host_seq checks its plan before touching any stream or buffer."""
    assert binding.ps_solve_host_seq(None, 0, None, None, None, None, None, None, None) == binding.PS_INVALID_ARG
    assert binding.ps_solve_host_seq(None, 3, None, None, None, None, None, None, None) == binding.PS_INVALID_ARG


def test_injected_allocation_failure(binding):
    """A host-injected allocation failure (the stand-in for an out-of-memory device)
    makes ps_plan_create return PS_OUT_OF_MEMORY cleanly: a NULL plan and a message,
    one injection consumed per create; a negative count is refused. No device is
    touched, so this runs without a GPU."""
    assert binding.ps_inject_alloc_failures(-1) == binding.PS_INVALID_ARG
    assert binding.ps_inject_alloc_failures(2) == binding.PS_OK
    for prec in (0, 2):
        h = ctypes.c_void_p(12345)
        st = binding.ps_plan_create(ctypes.byref(h), 8, 8, 8, 1.0, 1.0, None, 1.0, 0, 0, 1, prec, 1e-10, 3)
        assert st == binding.PS_OUT_OF_MEMORY and not h.value
        assert b"cudaMalloc" in binding.ps_last_error(None)
    assert binding.ps_inject_alloc_failures(0) == binding.PS_OK
