"""ps_solve_static: the solve for callers that cannot allocate device memory.

Some callers cannot hand the library a workspace at solve time (for example
code that runs under another framework's memory pool, or behind an interface
that has no slot for one). ps_solve_static runs the same kernels as ps_solve
with the workspace in a fixed 8 MiB device array compiled into the library.
These tests call it twice in a row through the C ABI, each time against
ps_solve on the same input, and check that an oversized plan is refused with
a clear error instead of touching memory it does not have.

This file is collected last on purpose (tests/test_zz_*), so that a run that
stops at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu


def _static_solve(lib, plan, f, p, info):
    import torch
    st = torch.cuda.current_stream().cuda_stream
    return lib.ps_solve_static(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                               ctypes.c_void_p(st), ctypes.c_void_p(info.data_ptr()))


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_static_scratch_matches_workspace_solve_twice(lib, precision):
    import torch
    nz, ny, nx = 24, 48, 64
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    plan = lib.Plan(nx, ny, nz, 6.0 / nx, 3.0 / ny, zf=zf, bcs=("P", "P", "NN"), precision=precision,
                    rtol=1e-10, max_iter=5)
    assert plan.workspace_bytes <= 8 << 20
    for seed in (21, 22):  # two calls in a row, different right-hand sides
        f = torch.as_tensor(synth.uniform_noise((nz, ny, nx), seed=seed), device="cuda")
        ref = plan.solve(f, info=lib.info_tensor())
        p = torch.empty_like(f)
        info = lib.info_tensor()
        assert _static_solve(lib, plan, f, p, info) == lib.PS_OK, lib.ps_last_error(plan.handle)
        torch.cuda.synchronize()
        a, b = p.cpu().numpy(), ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
        inf = lib.read_info(info)
        assert inf.status == 0
        if precision == "fp32_refine":
            assert inf.rel_residual <= 1e-10
    plan.close()


def test_static_scratch_refuses_oversized_plan(lib):
    plan = lib.Plan(256, 256, 256, 1.0 / 256, 1.0 / 256, dz=1.0 / 256, bcs=("P", "P", "NN"))
    assert plan.workspace_bytes > 8 << 20
    import torch
    f = torch.zeros((1, 1, 1), dtype=torch.float64, device="cuda")   # never read: refused first
    info = lib.info_tensor()
    st = _static_solve(lib, plan, f, f, info)
    assert st == lib.PS_UNSUPPORTED_SIZE
    assert b"static scratch" in lib.ps_last_error(plan.handle)
    plan.close()
