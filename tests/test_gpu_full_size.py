"""Parity at the benchmark's full sizes, in the benchmark's own configuration.

The refined solve of the 1024³ channel (6×3×1 box, P/P/NN, tanh z, f = the divergence
of a seeded Gaussian staggered velocity, rtol 1e-10, max_iter 4) and of the same
workload on 8192×8192×16 (lines of 8192) runs with the plan and input bench.py times
(its make_input and constants). The oracle cannot solve these sizes, but it can
evaluate the residual f_c − A·p at any point from the rows of its own 1D operators
(the x line, the y line and the z column through the point): at 20,000 sampled points
(5,000 for the 8192 lines) the residual of the returned p must stay within the
refinement tolerance and below the residual the device reported for the whole field.
"""

import os
import sys

import numpy as np
import pytest

from oracle import operator as O
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


@pytest.mark.parametrize("shape,samples", [((1024, 1024, 1024), 20000), ((8192, 8192, 16), 5000)],
                         ids=["channel-1024^3", "long-lines-8192x8192x16"])
def test_full_size_refined_solve_sampled_residual(lib, shape, samples):
    import torch
    B = _bench()
    dev = torch.device("cuda", 0)
    f, zf, dx, dy = B.make_input(shape, B.GRID["seed"], dev)
    plan = lib.Plan(*shape, dx, dy, zf=zf, bcs=B.BCS, precision="fp32_refine", rtol=B.RTOL, max_iter=B.MAX_ITER)
    info = lib.info_tensor(dev)
    p = plan.solve(f, info=info)
    torch.cuda.synchronize()
    inf = lib.read_info(info)
    plan.close()
    assert inf.status == 0 and inf.rel_residual <= B.RTOL, (inf.status, inf.rel_residual)
    fh = f.cpu().numpy()
    del f
    ph = p.cpu().numpy()
    del p
    torch.cuda.empty_cache()
    nx, ny, nz = shape
    fc_scale = np.abs(fh).max()
    # the volume-weighted mean of f (the singular problem's compatible part)
    dzf, _ = O.metrics(zf)
    mean = float((fh.sum(axis=(1, 2)) * dzf).sum() / (dzf.sum() * nx * ny))
    lx = O.operator_1d(B.BCS[0], synth.uniform_faces(nx, dx * nx), axis="xy")
    ly = O.operator_1d(B.BCS[1], synth.uniform_faces(ny, dy * ny), axis="xy")
    lz = O.operator_1d(B.BCS[2], zf)
    rng = np.random.default_rng(17)
    zs, ys, xs = rng.integers(0, nz, samples), rng.integers(0, ny, samples), rng.integers(0, nx, samples)
    ax = np.einsum("ij,ij->i", lx[xs], ph[zs, ys, :])
    ay = np.einsum("ij,ij->i", ly[ys], ph[zs, :, xs])
    az = np.einsum("ij,ij->i", lz[zs], ph[:, ys, xs].T)
    r = (fh[zs, ys, xs] - mean) - (ax + ay + az)
    rel = np.abs(r).max() / fc_scale
    assert rel <= B.RTOL, rel
    # the sampled points cannot exceed the device's residual over the whole field
    # (both relative to max|f_c| ≈ max|f|; slack for the two evaluations' rounding)
    assert rel <= inf.rel_residual * (1 + 1e-3) + 1e-13, (rel, inf.rel_residual)
