"""GPU parity for face-centred z unknowns between two walls (PS_BC_FACE_DIRICHLET,
"FD"): the wall-normal velocity of an implicit diffusion step (§2). Plane k is z face
k; plane 0 is the bottom wall (f's plane 0 kept zero, p's comes out zero) and the top
wall is implicit. Checked against the FP64 oracle with the same operator, with and
without a Helmholtz shift, in FP64, FP32 and the refined mode, on stretched z.
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


def _rhs(shape, seed):
    f = np.random.default_rng(seed).uniform(-1, 1, shape)
    f[0] = 0.0
    return f


CASES = [((12, 16, 24), ("P", "P"), 0.0), ((12, 16, 24), ("P", "P"), 80.0), ((10, 24, 12), ("DD", "NN"), 0.0),
         ((16, 12, 18), ("DN", "ND"), 5.0)]
IDS = [f"{'x'.join(map(str, s))}-{b[0]}-{b[1]}-a{a:g}" for s, b, a in CASES]


@pytest.mark.parametrize("shape,bcxy,alpha", CASES, ids=IDS)
def test_fp64_and_fp32_face_z(lib, shape, bcxy, alpha):
    nz, ny, nx = shape
    bcs = (bcxy[0], bcxy[1], "FD")
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = _rhs(shape, nx + nz)
    q = S.solve(f, 1.0 / nx, 2.0 / ny, zf, *bcs, alpha=alpha)
    p, _ = _run(lib, f, 1.0 / nx, 2.0 / ny, zf, bcs, alpha=alpha)
    assert _relerr(p, q) <= 1e-12 and np.abs(p[0]).max() <= 1e-13 * np.abs(q).max()
    p32, _ = _run(lib, f, 1.0 / nx, 2.0 / ny, zf, bcs, precision="fp32", alpha=alpha)
    assert _relerr(p32, q) <= 2e-5


REFINE = [((12, 16, 24), ("P", "P"), 0.0), ((16, 128, 256), ("P", "P"), 40.0), ((6, 512, 512), ("P", "NN"), 0.0),
          ((10, 24, 72), ("DD", "DN"), 3.0)]


@pytest.mark.parametrize("shape,bcxy,alpha", REFINE,
                         ids=[f"{'x'.join(map(str, s))}-{b[0]}-{b[1]}-a{a:g}" for s, b, a in REFINE])
def test_refine_face_z(lib, shape, bcxy, alpha):
    nz, ny, nx = shape
    bcs = (bcxy[0], bcxy[1], "FD")
    lx, ly = 6.0, 3.0
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    f = _rhs(shape, nx * 3 + ny)
    p, info = _run(lib, f, lx / nx, ly / ny, zf, bcs, precision="fp32_refine", rtol=1e-10, max_iter=6,
                   alpha=alpha)
    rr = O.relative_residual(p, f, lx / nx, ly / ny, zf, *bcs, alpha=alpha)
    assert info.status == 0 and info.rel_residual <= 1e-10, (info.status, info.rel_residual, rr)
    assert rr <= 1e-10 and abs(info.rel_residual - rr) <= 1e-11, (info.rel_residual, rr)
    q = S.solve(f, lx / nx, ly / ny, zf, *bcs, alpha=alpha)
    assert _relerr(p, q) <= 1e-8


def test_face_z_has_no_transpose(lib):
    import torch
    zf = synth.tanh_faces(8, 1.0, 1.5)
    plan = lib.Plan(8, 8, 8, 0.1, 0.1, zf=zf, bcs=("P", "P", "FD"), precision="fp64")
    g = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.PoissonError):
        plan.solve_transpose(g)
    plan.close()


def test_batch_face_z_grids(lib):
    import torch
    grids = [dict(nx=32, ny=24, nz=20, dx=1 / 32, dy=2 / 24, zf=synth.tanh_faces(20, 1.0, 1.5), bcs=("P", "P", "FD")),
             dict(nx=24, ny=48, nz=16, dx=1 / 24, dy=2 / 48, zf=synth.tanh_faces(16, 1.0, 1.5), bcs=("DD", "P", "FD"),
                  alpha=30.0),
             dict(nx=48, ny=16, nz=12, dx=1 / 48, dy=2 / 16, zf=synth.tanh_faces(12, 1.0, 1.5), bcs=("P", "NN", "NN"))]
    b = lib.Batch(grids, rtol=1e-10, max_iter=6)
    fs = []
    for g, d in enumerate(grids):
        f = np.random.default_rng(90 + g).uniform(-1, 1, (d["nz"], d["ny"], d["nx"]))
        if d["bcs"][2] == "FD":
            f[0] = 0.0
        fs.append(torch.as_tensor(f, device="cuda").contiguous())
    ps = [torch.zeros_like(f) for f in fs]
    fptr, pptr = b.pointers(fs, ps)
    infos = lib.infos_tensor(len(grids))
    b.solve(fptr, pptr, infos)
    torch.cuda.synchronize()
    for g, (d, inf) in enumerate(zip(grids, lib.read_infos(infos, len(grids)))):
        f, p = fs[g].cpu().numpy(), ps[g].cpu().numpy()
        al = d.get("alpha", 0.0)
        rr = O.relative_residual(p, f, d["dx"], d["dy"], d["zf"], *d["bcs"], alpha=al)
        assert inf.status == 0 and rr <= 1e-10, (g, inf.status, inf.rel_residual, rr)
        q = S.solve(f, d["dx"], d["dy"], d["zf"], *d["bcs"], alpha=al)
        assert np.abs(p - q).max() <= 1e-8 * np.abs(q).max(), g
    b.close()
