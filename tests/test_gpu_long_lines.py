"""GPU parity for x and y lines longer than 1024 cells (up to 8192; n/2 = 2^a·3^b).

Lines of n ≤ 1024 run in the register-resident transform kernels; longer ones
run in the shared-memory kernel, one line per CTA (two buffers of n/2 + 1
complex values, 131 KB for an FP64 line of 8192), with radix-4/2/3 stages.
Checked against the FP64 oracle (dense Table 2 matrices) in FP64, FP32 and the
refined mode, for each BC family including D-N, along x and along y.
"""

import numpy as np
import pytest

from oracle import solve as S
from oracle import operator as O
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(lib, f, dx, dy, zf, bcs, precision="fp64", **kw):
    import torch
    nz, ny, nx = f.shape
    plan = lib.Plan(nx, ny, nz, dx, dy, zf=zf, bcs=bcs, precision=precision, **kw)
    dt = torch.float32 if precision == "fp32" else torch.float64
    ft = torch.as_tensor(f, dtype=dt, device="cuda").contiguous()
    info = lib.info_tensor()
    out = plan.solve(ft, info=info)
    torch.cuda.synchronize()
    res = out.double().cpu().numpy(), lib.read_info(info)
    plan.close()
    return res


def _relerr(p, q):
    return np.abs(p - q).max() / max(np.abs(q).max(), 1e-300)


CASES = [((2, 6, 2048), ("P", "NN", "DD")), ((2, 2048, 8), ("DD", "P", "NN")),
         ((3, 4, 1536), ("ND", "DD", "NN")), ((2, 1536, 16), ("NN", "DN", "ND")),
         ((2, 4, 4096), ("DN", "P", "P")), ((2, 4096, 4), ("P", "ND", "DD")),
         ((2, 2, 8192), ("P", "NN", "NN")), ((2, 8192, 2), ("NN", "DD", "DN"))]
IDS = ["x".join(map(str, s)) + "-" + "-".join(b) for s, b in CASES]


@pytest.mark.parametrize("shape,bcs", CASES, ids=IDS)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_long_lines(lib, shape, bcs, precision, tol):
    nz, ny, nx = shape
    zf = synth.tanh_faces(nz, 1.0, 1.5) if bcs[2] != "P" else synth.uniform_faces(nz, 1.0)
    f = np.random.default_rng(nx + ny).uniform(-1, 1, shape)
    p, _ = _run(lib, f, 4.0 / nx, 4.0 / ny, zf, bcs, precision=precision)
    q = S.solve(f, 4.0 / nx, 4.0 / ny, zf, *bcs)
    assert _relerr(p, q) <= tol


REFINE = [((4, 8, 8192), ("P", "P", "NN")), ((4, 8192, 8), ("DD", "NN", "ND")),
          ((3, 2048, 1536), ("P", "DN", "NN"))]


@pytest.mark.parametrize("shape,bcs", REFINE, ids=["x".join(map(str, s)) + "-" + "-".join(b) for s, b in REFINE])
def test_long_lines_refine(lib, shape, bcs):
    nz, ny, nx = shape
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = np.random.default_rng(nx * 3 + ny).uniform(-1, 1, shape)
    lx, ly = 6.0 * nx / 1024, 3.0 * ny / 1024
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs)
    assert info.status == 0 and info.rel_residual <= 1e-10, (info.status, info.rel_residual, rr)
    assert rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)
