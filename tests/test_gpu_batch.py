"""GPU tests of the batched persistent solve (ps_batch_*).

* uneven grids of every BC kind (radix-2/3 sizes, stretched and periodic z,
  singular and non-singular) against the FP64 oracle, residual ≤ 1e-10;
* the 64-grid workload (sizes 32…192) under a captured CUDA graph, replayed
  twice: every grid converges and its residual, re-measured by the oracle's
  stencil, is ≤ 1e-10;
* the bounded wait: an unsatisfiable dependency (host-side test hook) ends
  with PS_TIMEOUT in the infos instead of a hang, and the context stays usable;
* the autotuner picks one of its candidate tile scales and the solve still
  agrees; a second batch of the same grids reads the choice back from the
  cache file, and a batch with another z stretching is a new cache key.
"""

import json

import numpy as np
import pytest

from oracle import operator as O
from oracle import solve as S
from paper_1802_10323_gb300 import synth, workloads

pytestmark = pytest.mark.gpu

SMALL = [
    dict(nx=32, ny=48, nz=20, bcs=("P", "P", "NN"), stretched=True),
    dict(nx=48, ny=32, nz=24, bcs=("NN", "DD", "ND"), stretched=True),
    dict(nx=64, ny=24, nz=16, bcs=("DD", "ND", "P"), stretched=False),
    dict(nx=24, ny=64, nz=30, bcs=("ND", "NN", "DD"), stretched=True),
    dict(nx=96, ny=16, nz=12, bcs=("NN", "NN", "NN"), stretched=True),
    dict(nx=16, ny=96, nz=8, bcs=("P", "NN", "P"), stretched=False),
    dict(nx=48, ny=24, nz=18, bcs=("DN", "ND", "DN"), stretched=True),
]


def _grids(spec):
    out = []
    for d in spec:
        zf = synth.tanh_faces(d["nz"], 1.0, 1.5) if d["stretched"] else synth.uniform_faces(d["nz"], 1.0)
        out.append(dict(nx=d["nx"], ny=d["ny"], nz=d["nz"], dx=1.0 / d["nx"], dy=2.0 / d["ny"], zf=zf,
                        bcs=d["bcs"]))
    return out


def _fields(lib, grids, seed):
    import torch
    fs, ps = [], []
    for g, d in enumerate(grids):
        f = np.random.default_rng(seed + g).uniform(-1, 1, (d["nz"], d["ny"], d["nx"]))
        fs.append(torch.as_tensor(f, device="cuda").contiguous())
        ps.append(torch.zeros_like(fs[-1]))
    return fs, ps


def test_batch_matches_oracle_every_bc_kind(lib):
    import torch
    grids = _grids(SMALL)
    b = lib.Batch(grids, rtol=1e-10, max_iter=6)
    fs, ps = _fields(lib, grids, 50)
    fptr, pptr = b.pointers(fs, ps)
    infos = lib.infos_tensor(len(grids))
    b.solve(fptr, pptr, infos)
    torch.cuda.synchronize()
    for g, (d, inf) in enumerate(zip(grids, lib.read_infos(infos, len(grids)))):
        f, p = fs[g].cpu().numpy(), ps[g].cpu().numpy()
        assert inf.status == 0 and inf.rel_residual <= 1e-10, (g, inf.status, inf.rel_residual)
        assert O.relative_residual(p, f, d["dx"], d["dy"], d["zf"], *d["bcs"]) <= 1e-10
        q = S.solve(f, d["dx"], d["dy"], d["zf"], *d["bcs"])
        assert np.abs(p - q).max() <= 1e-8 * np.abs(q).max(), g
    b.close()


def test_batch_64_grids_graph_capture(lib):
    import torch
    grids = workloads.batch_grids(64, seed=4)
    rhs = workloads.batch_rhs(grids, seed=4)
    b = lib.Batch(grids, rtol=1e-10, max_iter=4)
    fs = [torch.as_tensor(f, device="cuda").contiguous() for f in rhs]
    ps = [torch.zeros_like(f) for f in fs]
    fptr, pptr = b.pointers(fs, ps)
    infos = lib.infos_tensor(len(grids))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.solve(fptr, pptr, infos, stream=s)  # warm (loads the module, sets attributes)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.solve(fptr, pptr, infos, stream=s)
    for _ in range(2):
        for p in ps:
            p.zero_()
        graph.replay()
        torch.cuda.synchronize()
        got = lib.read_infos(infos, len(grids))
        for g, (d, inf) in enumerate(zip(grids, got)):
            assert inf.status == 0 and inf.rel_residual <= 1e-10, (g, inf.status, inf.rel_residual)
    for g in range(0, 64, 9):
        d = grids[g]
        assert O.relative_residual(ps[g].cpu().numpy(), rhs[g], d["dx"], d["dy"], d["zf"], *d["bcs"]) <= 1e-10
    b.close()


def test_batch_bounded_wait_reports_timeout(lib):
    import torch
    grids = _grids(SMALL[:3])
    b = lib.Batch(grids, rtol=1e-10, max_iter=3)
    fs, ps = _fields(lib, grids, 60)
    fptr, pptr = b.pointers(fs, ps)
    infos = lib.infos_tensor(len(grids))
    b.configure(wait_limit_seconds=0.02, inject_unsatisfiable_wait=True)
    b.solve(fptr, pptr, infos)
    torch.cuda.synchronize()
    got = lib.read_infos(infos, len(grids))
    assert got[0].status == lib.PS_TIMEOUT
    # the context is still usable: the same batch without the hook converges
    b.configure(wait_limit_seconds=2.0, inject_unsatisfiable_wait=False)
    b.solve(fptr, pptr, infos)
    torch.cuda.synchronize()
    assert all(i.status == 0 for i in lib.read_infos(infos, len(grids)))
    b.close()


def test_batch_autotune(lib, tmp_path, monkeypatch):
    import torch
    monkeypatch.setenv("PS_AUTOTUNE_CACHE", str(tmp_path / "tune.jsonl"))
    grids = _grids(SMALL)
    b = lib.Batch(grids, rtol=1e-10, max_iter=6)
    fs, ps = _fields(lib, grids, 70)
    fptr, pptr = b.pointers(fs, ps)
    scale, ms = b.autotune(fptr, pptr)
    assert scale in (1, 2, 4, 8, 16, 32, 64) and ms > 0
    cache = tmp_path / "tune.jsonl"
    assert cache.read_text().count("scale") == 1
    stored = json.loads(cache.read_text().splitlines()[0])
    assert stored["scale"] == scale
    infos = lib.infos_tensor(len(grids))
    for p in ps:
        p.zero_()
    b.solve(fptr, pptr, infos)
    torch.cuda.synchronize()
    assert all(i.status == 0 for i in lib.read_infos(infos, len(grids)))
    b.close()
    # a new batch of the same grids reads the cached choice back without timing:
    # the returned time is the stored one and nothing is appended
    b2 = lib.Batch(grids, rtol=1e-10, max_iter=6)
    fptr2, pptr2 = b2.pointers(fs, ps)
    scale2, ms2 = b2.autotune(fptr2, pptr2)
    assert scale2 == scale and ms2 == stored["ms"]
    assert cache.read_text().count("scale") == 1
    b2.close()
    # a different z stretching (or shift) is another key: it is timed and appended
    grids3 = _grids(SMALL)
    grids3[0]["zf"] = synth.tanh_faces(SMALL[0]["nz"], 1.0, 1.2)
    b3 = lib.Batch(grids3, rtol=1e-10, max_iter=6)
    fs3, ps3 = _fields(lib, grids3, 70)
    fptr3, pptr3 = b3.pointers(fs3, ps3)
    b3.autotune(fptr3, pptr3)
    assert cache.read_text().count("scale") == 2
    b3.close()


def test_batch_helmholtz_grids(lib):
    """Per-grid Helmholtz shifts (ps_batch_create_helmholtz): each grid solves
    (A − α_g·I)·p = f; a zero shift leaves its grid a Poisson grid (singular ones keep
    the mean handling), a positive one makes the all-P/NN grids regular."""
    import torch
    spec = [dict(SMALL[0], alpha=3.0), dict(SMALL[1], alpha=0.0), dict(SMALL[4], alpha=250.0),
            dict(SMALL[6], alpha=0.5)]
    grids = _grids(spec)
    for g, d in enumerate(grids):
        d["alpha"] = spec[g]["alpha"]
    b = lib.Batch(grids, rtol=1e-10, max_iter=6)
    fs, ps = _fields(lib, grids, 70)
    fptr, pptr = b.pointers(fs, ps)
    infos = lib.infos_tensor(len(grids))
    b.solve(fptr, pptr, infos)
    torch.cuda.synchronize()
    for g, (d, inf) in enumerate(zip(grids, lib.read_infos(infos, len(grids)))):
        f, p = fs[g].cpu().numpy(), ps[g].cpu().numpy()
        al = d["alpha"]
        rr = O.relative_residual(p, f, d["dx"], d["dy"], d["zf"], *d["bcs"], alpha=al)
        assert inf.status == 0 and inf.rel_residual <= 1e-10 and rr <= 1e-10, (g, inf.status, inf.rel_residual, rr)
        q = S.solve(f, d["dx"], d["dy"], d["zf"], *d["bcs"], alpha=al)
        assert np.abs(p - q).max() <= 1e-8 * np.abs(q).max(), g
    b.close()
