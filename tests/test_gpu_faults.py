"""Stand-ins for a memory checker on the GPU, and host-injected failures.

* Canary-padded buffers: f, p and the workspace of every solve mode sit inside one
  larger device allocation whose guard regions (before and after each buffer) hold
  a bit pattern; after the solve every guard must be intact and the result must
  match the FP64 oracle. Sizes are tiny and of odd factors (lines of 6, 12, 48 and
  18; z of 3 and 7) so that every ragged-tile and tail path of the kernels runs.
  Each plane, line and column count is small, so an out-of-bounds write of any
  kernel would land in a guard.
* A host-injected allocation failure (ps_inject_alloc_failures) makes the plan and
  batch constructors return PS_OUT_OF_MEMORY cleanly, and the library stays
  usable: the next create on the same device succeeds and solves.
"""

import ctypes

import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import solve as S
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes of canary on each side of every buffer
CANARY = 0x5A


class Padded:
    """Device buffers carved out of one allocation with canary guards around each."""

    def __init__(self, sizes):
        import torch
        self.sizes = [int(s) for s in sizes]
        self.offs = []
        off = GUARD
        for s in self.sizes:
            self.offs.append(off)
            off += (s + 255) // 256 * 256 + GUARD
        self.buf = torch.full((off,), CANARY, dtype=torch.uint8, device="cuda")

    def view(self, i, dtype, shape=None):
        import torch
        n = self.sizes[i] // torch.empty((), dtype=dtype).element_size()
        t = self.buf[self.offs[i]:self.offs[i] + self.sizes[i]].view(dtype)
        return t.view(shape) if shape is not None else t

    def intact(self):
        b = self.buf.cpu().numpy()
        mask = np.ones(len(b), dtype=bool)
        for o, s in zip(self.offs, self.sizes):
            mask[o:o + s] = False
        return bool((b[mask] == CANARY).all())


CASES = [((3, 12, 6), ("P", "NN", "DD")), ((7, 6, 12), ("ND", "P", "NN")), ((3, 48, 18), ("DN", "DD", "P")),
         ((7, 18, 48), ("NN", "NN", "NN")), ((3, 12, 6), ("FD", "DD", "FD"))]
IDS = ["x".join(map(str, s)) + "-" + "-".join(b) for s, b in CASES]


@pytest.mark.parametrize("shape,bcs", CASES, ids=IDS)
@pytest.mark.parametrize("mode", ["fp64", "fp32", "fp32_refine", "transpose"])
def test_canary_guards_stay_intact(lib, shape, bcs, mode):
    import torch
    if mode == "transpose" and bcs[2] == "FD":
        pytest.skip("face-centred z has no transpose solve")
    nz, ny, nx = shape
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    dx, dy = 1.0 / nx, 2.0 / ny
    f = np.random.default_rng(nx * ny + nz).uniform(-1, 1, shape)
    if bcs[2] == "FD":
        f[0] = 0.0
    prec = "fp64" if mode == "transpose" else mode
    plan = lib.Plan(nx, ny, nz, dx, dy, zf=zf, bcs=bcs, precision=prec, rtol=1e-10, max_iter=8)
    dt = torch.float32 if prec == "fp32" else torch.float64
    es = 4 if prec == "fp32" else 8
    ws_bytes = ctypes.c_size_t()
    lib._check(lib.ps_workspace_bytes(plan.handle, ctypes.byref(ws_bytes)), plan.handle)
    N = nx * ny * nz
    pad = Padded([N * es, N * es, max(int(ws_bytes.value), 256), 32])
    fd, pd = pad.view(0, dt, shape), pad.view(1, dt, shape)
    ws, info = pad.view(2, torch.uint8), pad.view(3, torch.float64)
    fd.copy_(torch.as_tensor(f, dtype=dt))
    fn = {"fp64": lib.ps_solve, "fp32_refine": lib.ps_solve, "fp32": lib.ps_solve_f32,
          "transpose": lib.ps_solve_transpose}[mode]
    st = fn(plan.handle, ctypes.c_void_p(fd.data_ptr()), ctypes.c_void_p(pd.data_ptr()),
            ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
            ctypes.c_void_p(info.data_ptr()))
    lib._check(st, plan.handle)
    torch.cuda.synchronize()
    assert pad.intact(), "a kernel wrote outside its buffers"
    if mode == "transpose":
        q = AD.solve_transpose(f, dx, dy, zf, *bcs)
    else:
        q = S.solve(f, dx, dy, zf, *bcs)
    tol = {"fp64": 1e-12, "fp32": 3e-5, "fp32_refine": 1e-8, "transpose": 1e-12}[mode]
    p = pd.double().cpu().numpy()
    assert np.abs(p - q).max() <= tol * np.abs(q).max()
    plan.close()


def test_injected_allocation_failure_then_recovery(lib):
    import torch
    zf = synth.uniform_faces(8, 1.0)
    lib.inject_alloc_failures(1)
    with pytest.raises(lib.PoissonError) as ei:
        lib.Plan(16, 16, 8, 0.1, 0.1, zf=zf, bcs=("P", "P", "NN"), precision="fp64")
    assert ei.value.status == lib.PS_OUT_OF_MEMORY
    grids = [dict(nx=16, ny=16, nz=8, dx=1 / 16, dy=1 / 16, zf=zf, bcs=("P", "NN", "DD"))] * 2
    lib.inject_alloc_failures(2)  # the second grid's plan
    with pytest.raises(Exception):
        lib.Batch(grids, rtol=1e-10, max_iter=4)
    lib.inject_alloc_failures(0)
    plan = lib.Plan(16, 16, 8, 0.1, 0.1, zf=zf, bcs=("P", "P", "NN"), precision="fp64")
    f = np.random.default_rng(1).uniform(-1, 1, (8, 16, 16))
    f -= f.mean()
    p = plan.solve(torch.as_tensor(f, device="cuda"))
    torch.cuda.synchronize()
    q = S.solve(f, 0.1, 0.1, zf, "P", "P", "NN")
    assert np.abs(p.cpu().numpy() - q).max() <= 1e-12 * np.abs(q).max()
    plan.close()


def test_misaligned_fields_are_refused(lib):
    """f or p off a 16-byte boundary (the transforms move lines with 16-byte accesses) is
    refused on the host with PS_INVALID_ARG before anything is launched; the plan then
    solves aligned fields as before."""
    import torch
    zf = synth.uniform_faces(8, 1.0)
    plan = lib.Plan(32, 32, 8, 1 / 32, 1 / 32, zf=zf, bcs=("P", "P", "NN"), precision="fp64")
    N = 32 * 32 * 8
    big = torch.zeros(N + 2, dtype=torch.float64, device="cuda")
    ws = plan.workspace()
    s = torch.cuda.current_stream().cuda_stream
    for f_off, p_off in ((1, 0), (0, 1)):
        fp = ctypes.c_void_p(big.data_ptr() + 8 * f_off)
        pp = torch.empty(N + 2, dtype=torch.float64, device="cuda")
        st = lib.ps_solve(plan.handle, fp, ctypes.c_void_p(pp.data_ptr() + 8 * p_off),
                          ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(s), None)
        assert st == lib.PS_INVALID_ARG
    f = np.random.default_rng(3).uniform(-1, 1, (8, 32, 32))
    f -= f.mean()
    p = plan.solve(torch.as_tensor(f, device="cuda"))
    torch.cuda.synchronize()
    q = S.solve(f, 1 / 32, 1 / 32, zf, "P", "P", "NN")
    assert np.abs(p.cpu().numpy() - q).max() <= 1e-12 * np.abs(q).max()
    plan.close()
