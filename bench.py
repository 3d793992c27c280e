#!/usr/bin/env python
"""Throughput of the eigenfunction-expansion Poisson solve on the channel workload.

Workload (one step = one complete solve): 1024 × 1024 × 1024 cells on a
6 × 3 × 1 box, periodic x and y, Neumann–Neumann z on a tanh grid (α = 1.5);
right-hand side f = discrete divergence of a seeded Gaussian staggered
velocity field (w = 0 on the walls). The timed path is the FP32 bulk solve
with FP64 iterative refinement to a relative residual of 1e-10 (checked on
the device every step); the plain FP64 GPU solve of the same input is timed
beside it. Inputs are resident in HBM (8.6 GB per field, far above the
126 MB L2, so no flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent replica per GPU (torchrun; weak scaling, no
collective on the data path). ``--impl reference`` times the FP64 CPU oracle
(test infrastructure) on a bounded sample of the same workload.

Printed: one JSON line on rank 0.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson solve Mpts/s at 1024^3 (FP32+refine vs FP64) and % of HBM roofline"
GRID = dict(nx=1024, ny=1024, nz=1024, lx=6.0, ly=3.0, lz=1.0, alpha=1.5, seed=3)
BCS = ("P", "P", "NN")
RTOL = 1e-10
MAX_ITER = 4

# Algorithmic bytes per grid point of each kernel kind (compulsory reads + writes
# of the fields it must touch; scratch traffic is not counted).
BYTES_PER_POINT = {
    # x backward: reads the FP32 line, stores (or adds into) the FP64 p and keeps
    # the FP32 values for the next residual pass; residual pass 0 reads f (FP64)
    # and Φ_0 (FP32), later passes r = rh + rl and the correction, and both write
    # rh + rl (the check pass writes nothing); the exact pass reads p and f.
    # The first x backward keeps only the FP32 Φ_0; the first correction writes
    # p = Φ_0 + e (and e in FP32), later ones add into p.
    "refine": {"x_fwd_f64in": 8 + 4, "x_fwd": 4 + 4, "y_fwd": 4 + 4, "z_solve": 4 + 4,
               "y_bwd": 4 + 4, "x_bwd_f64store": 4 + 4, "x_bwd_f64base": 4 + 4 + 8 + 4,
               "x_bwd_f64acc": 4 + 8 + 8 + 4, "materialize": 4 + 8,
               "residual_first": 8 + 4 + 8, "residual_first3": 8 + 4 + 8, "residual": 8 + 4 + 8,
               "residual_check": 8 + 4, "residual_out": 8 + 4 + 8, "residual_exact": 8 + 8 + 4,
               # plane transposes of long y lines (read and write FP32; traffic beyond the
               # five-pass model, measured as its own kind)
               "transpose": 4 + 4},
    "fp64": {"x_fwd": 16, "y_fwd": 16, "z_solve": 16, "y_bwd": 16, "x_bwd": 16},
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash(unit):
    """Hash of one kernel's translation unit (csrc/<unit>, whose launcher sets the launch
    shape) and the csrc headers it includes (the public C header, which declares the ABI
    and generates no kernel code, is not followed)."""
    csrc = os.path.join(ROOT, "paper_1802_10323_gb300", "csrc")
    seen, todo = [], [os.path.join(csrc, unit)]
    while todo:
        fn = os.path.normpath(todo.pop())
        if fn in seen or not os.path.exists(fn) or os.path.dirname(fn) != os.path.normpath(csrc):
            continue
        seen.append(fn)
        for line in open(fn, encoding="utf-8"):
            if line.startswith('#include "'):
                todo.append(os.path.join(os.path.dirname(fn), line.split('"')[1]))
    h = hashlib.sha256()
    for fn in sorted(seen):
        h.update(os.path.relpath(fn, ROOT).encode())
        h.update(open(fn, "rb").read())
    return h.hexdigest()[:16]


FP64_FLOPS_PER_POINT = 126      # plain FP64 solve at n = 1024 (see the fp64_solve roofline)
# Algorithmic FP64 flops per cell of the RK3 predictor (AD^k of the three components and
# the predictor update, counted from the stencils of the substep, not from a kernel):
#   advection: u·u, v·v, w·w at the cell centre (average, square) 3 × 3; their differences
#     3 × 2; the three edge products (two averages, a product, the ¼) 3 × 4; the six
#     edge-product differences 6 × 2; three terms summed per component 3 × 2      = 45
#   diffusion: per component x and y second differences 2 × 3, the stretched z one 6,
#     summed 2                                                       3 × 14      = 42
#   AD = −adv + ν·lap: 3; predictor u* = u + Δt(α AD + β AD' − γ G p) with the
#     pressure gradient difference: 3 × 6                              3 + 18      = 21
NS_FLOPS_PER_CELL = 108
# The predictor on FP64 fields runs in double-float (pairs of floats) on the FP32 pipe, so
# its binding unit is FP32 instruction issue: thread instructions per cell from ncu
# (smsp__inst_executed.sum × 32 / cells of one launch, ns_predict_kernel<double, 1, 1, 0>
# on 512x256x64, profiles/kernels_rk3_512x256x64.md), against the issue peak of
# 152 SMs × 4 schedulers × 32 lanes per clock.
NS_PRED_INST_PER_CELL = 1647
FP32_LANES_PER_SM = 128
NUM_SMS_GB300 = 152
FP64_NOMINAL_TFLOPS = 1.25      # GB300 dense FP64


def recorded_traffic(kernel, n_points):
    """DRAM bytes per launch of a kernel kind of the channel solve, from the committed ncu
    counters (a small case, per grid point), if its sources still match."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    ent = rec.get(kernel)
    if not ent or not ent.get("source") or ent.get("source_hash") != source_hash(ent["source"]):
        return None
    return ent["dram_bytes_per_point"] * n_points


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_input(n, seed, device):
    """Channel right-hand side on the device (seeded Philox), FP64, and the z faces."""
    from paper_1802_10323_gb300 import synth
    zf = synth.tanh_faces(n[2], GRID["lz"], GRID["alpha"])
    dx, dy = GRID["lx"] / n[0], GRID["ly"] / n[1]
    u, v, w = synth.staggered_velocity_torch(n[0], n[1], n[2], seed, device=device)
    f = synth.divergence_rhs_torch(u, v, w, dx, dy, zf)
    del u, v, w
    return f.contiguous(), zf, dx, dy


def cpu_oracle_rate(nz_sample=None, target_s=15.0, keep=None):
    """Mpts/s of the FP64 oracle solve on a 1024 × 1024 × nz_sample slab of the workload.
    keep: a dict that receives the slab's f, the oracle's solution and the grid."""
    import numpy as np
    from oracle import solve as S
    from paper_1802_10323_gb300 import synth

    def run(nzs):
        zf = synth.tanh_faces(nzs, GRID["lz"], GRID["alpha"])
        dx, dy = GRID["lx"] / GRID["nx"], GRID["ly"] / GRID["ny"]
        u, v, w = synth.staggered_velocity(GRID["nx"], GRID["ny"], nzs, GRID["seed"])
        f = synth.divergence_rhs(u, v, w, dx, dy, zf)
        del u, v, w
        t0 = time.perf_counter()
        q = S.solve(f, dx, dy, zf, *BCS)
        dt = time.perf_counter() - t0
        if keep is not None:
            keep.update(f=f, q=q, zf=zf, dx=dx, dy=dy, nz=nzs)
        return dt

    if nz_sample is None:
        t8 = run(8)
        nz_sample = int(min(256, max(16, 8 * target_s / max(t8, 1e-3))) // 8 * 8)
    t = run(nz_sample)
    pts = GRID["nx"] * GRID["ny"] * nz_sample
    cores = len(os.sched_getaffinity(0))
    try:
        blas = np.__config__.CONFIG["Build Dependencies"]["blas"]["name"]
    except Exception:
        blas = "unknown"
    return {"value": pts / t / 1e6, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
            "sample": f"one FP64 oracle solve (dense Table 2 matmuls + Thomas) of a "
                      f"1024x1024x{nz_sample} slab of the channel workload "
                      f"(same x/y sizes, BCs, tanh z), {t:.1f} s; BLAS={blas}, "
                      f"threads={cores}"}


def scipy_cpu_rate(slab):
    """A library CPU solve of the oracle's slab for context ("library CPU", not the
    oracle): scipy.fft real FFTs along the periodic x and y (the same eigenvalues
    of Table 1 in the standard complex layout) and a vectorised Thomas sweep along
    the Neumann z, FP64, on the host's cores. Returns Mpts/s and its error against
    the oracle's solution."""
    import numpy as np
    import scipy.fft as sfft
    f, q, zf, dx, dy = slab["f"], slab["q"], slab["zf"], slab["dx"], slab["dy"]
    nz, ny, nx = f.shape
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    fh = sfft.rfft2(f, axes=(1, 2), workers=cores)             # [nz][ny][nx/2+1] complex
    kx = np.arange(nx // 2 + 1)
    ky = np.concatenate([np.arange(ny // 2 + 1), np.arange(ny // 2 + 1 - ny, 0)])
    lam = (-4 * np.sin(np.pi * kx / nx) ** 2 / dx ** 2)[None, :] + (-4 * np.sin(np.pi * ky / ny) ** 2 / dy ** 2)[:, None]
    dzf = np.diff(zf)
    dzc = 0.5 * (dzf[1:] + dzf[:-1])
    a = np.zeros(nz)
    c = np.zeros(nz)
    a[1:] = 1.0 / (dzf[1:] * dzc)
    c[:-1] = 1.0 / (dzf[:-1] * dzc)
    b = -(a + c)
    # (0, 0): the singular column, pinned and mean-free (Δz^f-weighted), as the oracle
    d = fh[:, 0, 0].real.copy()
    d -= (dzf * d).sum() / dzf.sum()
    lam00 = lam[0, 0]
    lam[0, 0] = 1.0                                            # any nonzero value; replaced below
    cp = np.zeros((nz,) + lam.shape)
    dp = np.zeros_like(fh)
    den = b[0] + lam
    cp[0] = c[0] / den
    dp[0] = fh[0] / den
    for k in range(1, nz):
        den = b[k] + lam - a[k] * cp[k - 1]
        cp[k] = c[k] / den
        dp[k] = (fh[k] - a[k] * dp[k - 1]) / den
    x = np.empty_like(fh)
    x[-1] = dp[-1]
    for k in range(nz - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    s = np.zeros(nz)                                           # the singular column
    cc, dd = np.zeros(nz), np.zeros(nz)
    den = b[1] + lam00
    cc[1], dd[1] = c[1] / den, d[1] / den
    for k in range(2, nz):
        den = b[k] + lam00 - a[k] * cc[k - 1]
        cc[k], dd[k] = c[k] / den, (d[k] - a[k] * dd[k - 1]) / den
    s[-1] = dd[-1]
    for k in range(nz - 2, 0, -1):
        s[k] = dd[k] - cc[k] * s[k + 1]
    s -= (dzf * s).sum() / dzf.sum()
    x[:, 0, 0] = s
    p = sfft.irfft2(x, s=(ny, nx), axes=(1, 2), workers=cores)
    t = time.perf_counter() - t0
    return {"value": nx * ny * nz / t / 1e6, "unit": "Mpts/s", "cores": cores, "kind": "library CPU (scipy.fft)",
            "max_rel_err_vs_oracle": float(np.abs(p - q).max() / np.abs(q).max()),
            "sample": f"the oracle's {nx}x{ny}x{nz} slab: scipy.fft rfft2/irfft2 in x and y, vectorised "
                      f"Thomas in z, FP64, {t:.2f} s"}


class Ranks:
    """The replica world of a multi-GPU run: one process per GPU, each solving its own
    copy of the workload (weak scaling, no collective on the data path). Only the
    timing uses the process group: a barrier around the timed region and the
    maximum of the per-rank times. The backend is NCCL on GPUs; the same code runs
    over gloo on the CPU (tests)."""

    def __init__(self, backend="nccl", device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.device = device
        if self.world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group(backend, device_id=device)
            else:
                dist.init_process_group(backend)

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x):
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


def _count_lines(path):
    try:
        with open(path) as fh:
            return sum(1 for ln in fh if ln.strip())
    except OSError:
        return 0


def job_rate(world, points_per_rank, ms_max):
    """Whole-job Mpts/s: the points all ranks solved over the slowest rank's time."""
    return world * points_per_rank / (ms_max * 1e-3) / 1e6


def bench_reference(args):
    """The FP64 CPU oracle, as it stands, on a bounded slab of the workload per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    nzs = 16
    for _ in range(args.warmup):
        cpu_oracle_rate(nz_sample=nzs)
    runs = [cpu_oracle_rate(nz_sample=nzs) for _ in range(args.steps)]
    v = statistics.median(r["value"] for r in runs)
    cpu = dict(runs[0])
    cpu["value"] = v
    pts = GRID["nx"] * GRID["ny"] * nzs
    line = {"metric": METRIC, "value": v, "unit": "Mpts/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": pts / v / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"channel 1024x1024x{nzs} slab (bounded CPU sample of the 1024^3 "
                                   "workload), P/P/NN, tanh z 1.5", "parallelism": "none (host cores)"},
            "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def bench_ours(args):
    import torch
    from paper_1802_10323_gb300 import binding as lib

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ranks = Ranks("nccl", dev)
    world, rank = ranks.world, ranks.rank
    barrier, max_over_ranks = ranks.barrier, ranks.max

    n = (args.n, args.n, args.nz or args.n)
    N = n[0] * n[1] * n[2]
    f, zf, dx, dy = make_input(n, GRID["seed"], dev)
    plan = lib.Plan(n[0], n[1], n[2], dx, dy, zf=zf, bcs=BCS, precision="fp32_refine",
                    rtol=RTOL, max_iter=MAX_ITER)
    p = torch.empty_like(f)
    info = lib.info_tensor(dev)
    ws = plan.workspace(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        plan.solve(f, p, info=info)
    torch.cuda.synchronize()
    inf = lib.read_info(info)
    if inf.status != 0:
        raise SystemExit(f"refined solve did not converge: status {inf.status}, rel {inf.rel_residual}")

    # ---- timed region: K refined solves ----
    plan.profile(True)
    clk = Clocks(local)
    time.sleep(0.4)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.solve(f, p, info=info)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms)
    prof = plan.profile_read()
    plan.profile(False)
    inf = lib.read_info(info)
    value = job_rate(world, N, ms_max)

    # dominant kernel and its roofline
    bpp = BYTES_PER_POINT["refine"]
    dom, dom_ms = None, -1.0
    for k, (launches, active, tot, act_ms) in prof.items():
        if k in bpp and act_ms > dom_ms:
            dom, dom_ms = k, act_ms
    launches, active, tot, act_ms = prof[dom]
    avg_ms = act_ms / max(active, 1)
    bytes_launch = bpp[dom] * N
    achieved = bytes_launch / (avg_ms * 1e-3) / 1e9
    peak, peak_src = peaks()
    gpu_launches = sum(v[0] for v in prof.values()) + sum(
        prof.get(k, (0,))[0] for k in ("residual_first", "residual_first3", "residual", "residual_check",
                                       "residual_out", "residual_exact"))
    kernels = {k: {"launches": v[0], "active": v[1], "active_ms_per_step": v[3] / args.steps,
                   "share": v[3] / max(sum(x[3] for x in prof.values()), 1e-9)}
               for k, v in prof.items() if v[0]}

    # ---- end to end through the public host-buffer call ----
    e2e = None
    if not args.no_e2e:
        fh = f.cpu().pin_memory()
        ph = torch.empty_like(fh).pin_memory()
        f2, p2 = torch.empty_like(f), torch.empty_like(p)  # the second device slot
        for _ in range(2):  # warm (the first calls on fresh pinned buffers run slower)
            plan.solve_host(fh, ph, f, p)
        plan.solve_host_seq([fh] * 2, [ph] * 2, [f, f2], [p, p2])
        k_e2e = max(4, min(args.steps, 10))
        # K problems through the sequence call: each one's f copied in from pinned host
        # memory and its p copied out, the copies of neighbouring problems overlapping.
        # The host link is shared with other work on the machine and its speed varies
        # from second to second, so the sequence runs three times and the median counts.
        barrier()
        seq_ms = []
        for _ in range(3):
            t0 = time.perf_counter()
            ies = plan.solve_host_seq([fh] * k_e2e, [ph] * k_e2e, [f, f2], [p, p2])
            seq_ms.append(max_over_ranks((time.perf_counter() - t0) / k_e2e) * 1e3)
        t_e2e = statistics.median(seq_ms) * 1e-3
        ie = ies[-1]
        del f2, p2
        # the same problem through the one-call-per-solve path (nothing overlaps across calls)
        per_call = []
        for _ in range(k_e2e):
            tc = time.perf_counter()
            plan.solve_host(fh, ph, f, p)
            per_call.append(time.perf_counter() - tc)
        # the host link alone: the same pinned buffers copied in and out (no solve), as many
        # times, so that the spread of the calls can be set against the spread of the copies
        per_copy = []
        for _ in range(k_e2e):
            tc = time.perf_counter()
            f.copy_(fh, non_blocking=True)
            ph.copy_(p, non_blocking=True)
            torch.cuda.synchronize()
            per_copy.append(time.perf_counter() - tc)
        # both directions at once (two streams): the link's bound for a sequence whose
        # copies overlap across problems
        per_both = []
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        for _ in range(k_e2e):
            torch.cuda.synchronize()
            tc = time.perf_counter()
            with torch.cuda.stream(s_in):
                f.copy_(fh, non_blocking=True)
            with torch.cuda.stream(s_out):
                ph.copy_(p, non_blocking=True)
            torch.cuda.synchronize()
            per_both.append(time.perf_counter() - tc)
        e2e = {"value": job_rate(world, N, t_e2e * 1e3), "unit": "Mpts/s",
               "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8 + 32,
               "ms_per_step": t_e2e * 1e3, "problems": k_e2e, "sequences_ms_per_problem": seq_ms,
               "api": "ps_solve_host_seq (copies of neighbouring problems overlap)",
               "statuses": sorted({i.status for i in ies}), "status": ie.status,
               "single_calls": {"api": "ps_solve_host, one call per problem", "calls": k_e2e,
                                "ms_min": min(per_call) * 1e3, "ms_max": max(per_call) * 1e3,
                                "ms_median": statistics.median(per_call) * 1e3},
               "copies_only": {"what": "f host->device then p device->host, pinned, no solve",
                               "ms_min": min(per_copy) * 1e3, "ms_median": statistics.median(per_copy) * 1e3,
                               "ms_max": max(per_copy) * 1e3},
               "copies_both_directions": {"what": "f host->device and p device->host at once, two streams",
                                          "ms_min": min(per_both) * 1e3,
                                          "ms_median": statistics.median(per_both) * 1e3,
                                          "ms_max": max(per_both) * 1e3}}
        del fh, ph

    # ---- plain FP64 GPU solve of the same input (the comparison) ----
    plan64 = lib.Plan(n[0], n[1], n[2], dx, dy, zf=zf, bcs=BCS, precision="fp64")
    p64 = torch.empty_like(f)
    plan64.solve(f, p64)
    torch.cuda.synchronize()
    # the FP64 pipe's measured rate (the FP64 solve and the RK3 predictor are bound by it),
    # with the SM clocks sampled while the probe runs
    ck = Clocks(torch.cuda.current_device()) if rank == 0 else None
    time.sleep(0.25)
    tfl, pms = lib.probe_fp64(iters=400000)
    time.sleep(0.25)
    pclk = ck.stop() if ck else None
    fp64_peak = {"tflops": tfl, "probe_ms": pms, "clocks": pclk,
                 "source": f"measured: ps_probe_fp64 (FP64 FMA chains on every SM, {pms:.0f} ms, "
                           f"SM clock median {pclk['sm_mhz'] if pclk else None} MHz)",
                 "nominal_tflops": FP64_NOMINAL_TFLOPS}
    k64 = max(1, args.fp64_steps)
    plan64.profile(True)
    e0.record(stream)
    for _ in range(k64):
        plan64.solve(f, p64)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = max_over_ranks(e0.elapsed_time(e1) / k64)
    prof64 = plan64.profile_read()
    diff = (p - p64).abs().max().item() / p64.abs().max().item()
    del p64
    plan64.close()

    # ---- Helmholtz plan on the same grid and input: (A − α·I)·p = f, α = 2/(ν·Δt) of a
    # Crank–Nicolson diffusion step of the channel (bulk Reynolds number 5600, unit bulk
    # velocity and height; Δt at convective CFL 0.5 with u_max = 1.5) ----
    helm = None
    if not args.no_helmholtz:
        nu = 1.0 / 5600.0
        dt = 0.5 * dx / 1.5
        alpha = 2.0 / (nu * dt)
        planh = lib.Plan(n[0], n[1], n[2], dx, dy, zf=zf, bcs=BCS, precision="fp32_refine",
                         rtol=RTOL, max_iter=MAX_ITER, alpha=alpha)
        infh = lib.info_tensor(dev)
        for _ in range(args.warmup):
            planh.solve(f, p, info=infh)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            planh.solve(f, p, info=infh)
        e1.record(stream)
        torch.cuda.synchronize()
        msh = max_over_ranks(e0.elapsed_time(e1) / args.steps)
        ih = lib.read_info(infh)
        helm = {"value": job_rate(world, N, msh), "unit": "Mpts/s", "ms_per_step": msh, "alpha": alpha,
                "iterations": ih.iterations, "rel_residual": ih.rel_residual, "status": ih.status,
                "workload": "the same grid and f, Helmholtz shift of a Crank-Nicolson diffusion step "
                            "(Re_b 5600, CFL 0.5), FP32+refine to 1e-10"}
        planh.close()
        plan.solve(f, p, info=info)  # p again holds the Poisson solution (e2e below reuses it)

    # ---- the D-N pair (not in Table 1) on x and z of the same grid and input ----
    dn = None
    if not args.no_dn:
        bcs_dn = ("DN", BCS[1], "DN")
        pland = lib.Plan(n[0], n[1], n[2], dx, dy, zf=zf, bcs=bcs_dn, precision="fp32_refine",
                         rtol=RTOL, max_iter=MAX_ITER)
        infd = lib.info_tensor(dev)
        for _ in range(args.warmup):
            pland.solve(f, p, info=infd)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            pland.solve(f, p, info=infd)
        e1.record(stream)
        torch.cuda.synchronize()
        msd = max_over_ranks(e0.elapsed_time(e1) / args.steps)
        idn = lib.read_info(infd)
        dn = {"value": job_rate(world, N, msd), "unit": "Mpts/s", "ms_per_step": msd, "bcs": list(bcs_dn),
              "iterations": idn.iterations, "rel_residual": idn.rel_residual, "status": idn.status,
              "workload": "the same grid and f with Dirichlet-Neumann pairs on x and z, FP32+refine to 1e-10"}
        pland.close()
        plan.solve(f, p, info=info)

    # ---- lines longer than 1024: the same number of points as 8192 x 8192 x 16 ----
    longl = None
    if not args.no_long and args.n == 1024 and not args.nz:
        from paper_1802_10323_gb300 import synth
        nl = (8192, 8192, 16)
        # the headline's right-hand side (divergence of a Gaussian staggered velocity) on
        # the same 6 x 3 x 1 channel box with 8192 x 8192 x 16 cells
        fl, zl, dxl, dyl = make_input(nl, GRID["seed"], dev)
        planl = lib.Plan(nl[0], nl[1], nl[2], dxl, dyl, zf=zl, bcs=BCS,
                         precision="fp32_refine", rtol=RTOL, max_iter=MAX_ITER)
        pl_ = torch.empty_like(fl)
        infl = lib.info_tensor(dev)
        for _ in range(2):
            planl.solve(fl, pl_, info=infl)
        torch.cuda.synchronize()
        barrier()
        kl = max(1, min(args.steps, 3))
        planl.profile(True)
        e0.record(stream)
        for _ in range(kl):
            planl.solve(fl, pl_, info=infl)
        e1.record(stream)
        torch.cuda.synchronize()
        msl = max_over_ranks(e0.elapsed_time(e1) / kl)
        profl = planl.profile_read()
        planl.profile(False)
        il = lib.read_info(infl)
        ptsl = nl[0] * nl[1] * nl[2]
        doml = max((k for k in profl if k in bpp and profl[k][1]), key=lambda k: profl[k][3])
        avgl = profl[doml][3] / profl[doml][1]
        achl = bpp[doml] * ptsl / (avgl * 1e-3) / 1e9
        longl = {"value": job_rate(world, nl[0] * nl[1] * nl[2], msl), "unit": "Mpts/s",
                 "ms_per_step": msl, "grid": list(nl), "iterations": il.iterations,
                 "roofline": {"bound": "hbm", "kernel": doml, "achieved": achl, "peak": peak,
                              "unit": "GB/s", "frac": achl / peak, "avg_launch_ms": avgl,
                              "algorithmic_bytes_per_launch": bpp[doml] * ptsl},
                 "rel_residual": il.rel_residual, "status": il.status,
                 "kernels_ms_per_step": {k: v[3] / kl for k, v in profl.items() if v[1]},
                 "workload": "8192x8192x16 (x and y lines of 8192: the one-line-per-CTA transform kernel, "
                             "y lines through plane transposes), 6x3x1 box, P/P/NN tanh z, "
                             "f = div(Gaussian staggered velocity) (Philox seed 3), FP32+refine to 1e-10"}
        planl.close()
        del fl, pl_, planl
        torch.cuda.empty_cache()

    # ---- one RK3 time step of the fractional-step integration around the solve (§2):
    # the 512 x 256 x 256 channel (6x3x1, P/P/NN, tanh z), FP64 fields, refined solves ----
    ns = None
    if not args.no_ns and args.n == 1024 and not args.nz:
        from paper_1802_10323_gb300 import synth
        n5 = (512, 256, 256)
        z5 = synth.tanh_faces(n5[2], 1.0, 1.5)
        plan5 = lib.Plan(n5[0], n5[1], n5[2], 6.0 / n5[0], 3.0 / n5[1], zf=z5, bcs=BCS,
                         precision="fp32_refine", rtol=RTOL, max_iter=MAX_ITER)
        uu, vv, ww = synth.staggered_velocity_torch(n5[0], n5[1], n5[2], 5, device=dev)
        u5 = torch.stack([uu, vv, ww]).contiguous()
        del uu, vv, ww
        us5, ad5 = torch.empty_like(u5), torch.zeros_like(u5)
        p5 = torch.zeros((n5[2], n5[1], n5[0]), dtype=torch.float64, device=dev)
        phi5, rhs5 = torch.empty_like(p5), torch.empty_like(p5)
        inf5 = lib.info_tensor(dev)
        dt5, nu5 = 1e-3, 1.0 / 5600.0

        def rk3():
            for kk in (1, 2, 3):
                plan5.ns_substep(kk, dt5, nu5, u5, us5, ad5, p5, phi5, rhs5, info=inf5)

        for _ in range(2):
            rk3()
        torch.cuda.synchronize()
        barrier()
        k5 = max(1, min(args.steps, 5))
        # the step time without per-kernel events (a step launches ~170 kernels, whose
        # bracketing event records would add ~4 %), then the same steps again with them
        # for the per-kernel times and the predictor's roofline
        e0.record(stream)
        for _ in range(k5):
            rk3()
        e1.record(stream)
        torch.cuda.synchronize()
        ms5 = max_over_ranks(e0.elapsed_time(e1) / k5)
        plan5.profile(True)
        e0.record(stream)
        for _ in range(k5):
            rk3()
        e1.record(stream)
        torch.cuda.synchronize()
        ms5_prof = max_over_ranks(e0.elapsed_time(e1) / k5)
        prof5 = plan5.profile_read()
        plan5.profile(False)
        i5 = lib.read_info(inf5)
        cells5 = n5[0] * n5[1] * n5[2]
        pl5, pa5, _, pm5 = prof5["ns_predict"]
        pred_ms = pm5 / max(pa5, 1)
        sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
        issue_peak = NUM_SMS_GB300 * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12  # T thread-inst/s
        inst_rate = NS_PRED_INST_PER_CELL * cells5 / (pred_ms * 1e-3) / 1e12
        f64eq = NS_FLOPS_PER_CELL * cells5 / (pred_ms * 1e-3) / 1e12
        ns = {"value": job_rate(world, n5[0] * n5[1] * n5[2], ms5), "unit": "Mpts/s (cells x RK3 steps)",
              "ms_per_rk3_step": ms5, "ms_per_rk3_step_profiled": ms5_prof, "grid": list(n5),
              "last_solve_status": i5.status,
              # the fused predictor (double-float arithmetic on FP64 fields) is bound by FP32
              # instruction issue: ncu's instructions per cell against the issue peak
              "roofline": {"bound": "alu", "kernel": "ns_predict", "avg_launch_ms": pred_ms,
                           "inst_per_cell": NS_PRED_INST_PER_CELL, "achieved": inst_rate,
                           "peak": issue_peak, "unit": "T thread-inst/s",
                           "peak_source": f"{NUM_SMS_GB300} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz "
                                          "(median SM clock of the main timed region)",
                           "frac": inst_rate / issue_peak,
                           # the same launch as FP64-accurate flops (the stencils' count)
                           "fp64_equivalent": {"flops_per_cell": NS_FLOPS_PER_CELL, "tflops": f64eq,
                                               "native_fp64_peak_tflops": fp64_peak["tflops"],
                                               "frac_of_native_fp64": f64eq / fp64_peak["tflops"]}},
              "kernels_ms_per_step": {k: v[3] / k5 for k, v in prof5.items() if v[0]},
              "last_solve_rel_residual": i5.rel_residual,
              "workload": "3 substeps of ps_ns_substep (predictor, divergence, refined solve to 1e-10, "
                          "projection, pressure update) per step; FP64 fields; Gaussian staggered velocity "
                          "(seed 5), nu = 1/5600, dt = 1e-3"}
        plan5.close()
        del u5, us5, ad5, p5, phi5, rhs5, plan5
        torch.cuda.empty_cache()

    # ---- batched persistent solve: 64 uneven grids, one captured CUDA graph ----
    batch = None
    if not args.no_batch:
        from paper_1802_10323_gb300 import workloads
        grids = workloads.batch_grids(64, seed=4)
        rhs = workloads.batch_rhs(grids, seed=4)
        bt = lib.Batch(grids, rtol=RTOL, max_iter=MAX_ITER)
        bf = [torch.as_tensor(x, device=dev).contiguous() for x in rhs]
        bp = [torch.zeros_like(x) for x in bf]
        fptr, pptr = bt.pointers(bf, bp)
        # the autotuner's cache file: the first call times the candidate scales (or
        # reads an entry a previous run left), a second batch of the same grids must
        # read the entry back without timing
        if not os.environ.get("PS_AUTOTUNE_CACHE"):
            os.environ["PS_AUTOTUNE_CACHE"] = os.path.join(tempfile.gettempdir(),
                                                           f"ps_autotune_{os.getpid()}.jsonl")
        cache_file = os.environ["PS_AUTOTUNE_CACHE"]
        lines0 = _count_lines(cache_file)
        t_tune = time.perf_counter()
        scale, tune_ms = bt.autotune(fptr, pptr)
        t_tune = time.perf_counter() - t_tune
        lines1 = _count_lines(cache_file)
        bt2 = lib.Batch(grids, rtol=RTOL, max_iter=MAX_ITER)
        t_hit = time.perf_counter()
        scale2, _ = bt2.autotune(*bt2.pointers(bf, bp))
        t_hit = time.perf_counter() - t_hit
        bt2.close()
        autotune = {"scale": scale, "batch_ms_at_scale": tune_ms, "first_call_s": t_tune,
                    "entries_before": lines0, "entries_after_first": lines1,
                    "second_batch_scale": scale2, "second_call_s": t_hit,
                    "second_call_hit_cache": scale2 == scale and _count_lines(cache_file) == lines1}
        binfo = lib.infos_tensor(len(grids), dev)
        sb = torch.cuda.Stream(dev)
        sb.wait_stream(stream)
        with torch.cuda.stream(sb):
            bt.solve(fptr, pptr, binfo, stream=sb)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=sb):
            bt.solve(fptr, pptr, binfo, stream=sb)
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        kb = 10
        e0.record(stream)
        for _ in range(kb):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1) / kb
        infos_b = lib.read_infos(binfo, len(grids))
        npts = sum(d["nx"] * d["ny"] * d["nz"] for d in grids)
        batch = {"value": npts / (bms * 1e-3) / 1e6, "unit": "Mpts/s", "ms_per_replay": bms,
                 "grids": len(grids), "points": npts, "tile_scale": scale, "autotune": autotune,
                 "all_converged": all(i.status == 0 for i in infos_b),
                 "max_rel_residual": max(i.rel_residual for i in infos_b),
                 "workload": "64 grids, sizes {32..192} (x<=192, y<=128, z<=96), random BC pairs, "
                             "uniform or tanh z, FP32+refine to 1e-10, one persistent launch per graph replay"}
        bt.close()

    cpu = None
    vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu:
        slab = {}
        cpu = cpu_oracle_rate(keep=slab)
        cpu["library_cpu"] = scipy_cpu_rate(slab)
        # the FP64 and refined GPU solves of the same slab (same x/y lines, BCs, tanh z)
        # against the oracle's solution, element by element
        import numpy as np
        fs = torch.as_tensor(slab["f"], device=dev).contiguous()
        vs_oracle = {"slab": [GRID["nx"], GRID["ny"], slab["nz"]],
                     "input": "f = div(Gaussian staggered velocity) (PCG64 seed 3) on the slab's own tanh z"}
        for prec in ("fp64", "fp32_refine"):
            pls = lib.Plan(GRID["nx"], GRID["ny"], slab["nz"], slab["dx"], slab["dy"], zf=slab["zf"], bcs=BCS,
                           precision=prec, rtol=RTOL, max_iter=MAX_ITER)
            infs = lib.info_tensor(dev)
            ps_ = pls.solve(fs, info=infs)
            torch.cuda.synchronize()
            got = ps_.cpu().numpy()
            vs_oracle[prec] = {"max_rel_err": float(np.abs(got - slab["q"]).max() / np.abs(slab["q"]).max()),
                               "status": lib.read_info(infs).status}
            pls.close()
            del ps_
        del fs
        torch.cuda.empty_cache()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (bulk) + double-float residual", "data": "synthetic",
            "config": {"workload": f"channel {n[0]}x{n[1]}x{n[2]}, 6x3x1 box, P/P/NN, tanh z alpha=1.5, "
                                   "f = div(Gaussian staggered velocity), seed 3",
                       "grid": list(n), "precision": "fp32_refine", "rtol": RTOL, "max_iter": MAX_ITER,
                       "l2": "no flush: every field (8.6 GB at 1024^3) exceeds the 126 MB L2",
                       "parallelism": f"replicas x{world}"},
            "refine": {"iterations": inf.iterations, "rel_residual": inf.rel_residual,
                       "status": inf.status,
                       "max_rel_err_vs_oracle": vs_oracle["fp32_refine"]["max_rel_err"] if vs_oracle else None},
            "fp64_solve": {"value": job_rate(world, N, ms64), "unit": "Mpts/s",
                           "ms_per_step": ms64, "max_rel_diff_vs_refined": diff,
                           "max_rel_err_vs_oracle": vs_oracle["fp64"]["max_rel_err"] if vs_oracle else None,
                           "vs_oracle": vs_oracle,
                           # FP64-ALU bound on this part: four transforms (≈ 2.5·log2 n + 4 flops
                           # per point each) and the Thomas sweep (≈ 9), ≈ 126 flops per point at
                           # n = 1024, against the nominal FP64 rate; and its 80 B/pt against HBM
                           "roofline_fp64": {"bound": "fp64", "flops_per_point": FP64_FLOPS_PER_POINT,
                                             "achieved": FP64_FLOPS_PER_POINT * N / (ms64 * 1e-3) / 1e12,
                                             "peak": fp64_peak["tflops"], "unit": "TFLOP/s",
                                             "peak_source": fp64_peak["source"],
                                             "frac": FP64_FLOPS_PER_POINT * N / (ms64 * 1e-3) / 1e12
                                             / fp64_peak["tflops"],
                                             "hbm_frac": 80 * N / (ms64 * 1e-3) / 1e9 / peak},
                           "kernels": {k: v[3] / k64 for k, v in prof64.items() if v[0]}},
            "speedup_vs_fp64": ms64 / ms_max,
            "fp64_peak": fp64_peak,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                         "algorithmic_bytes_per_launch": bytes_launch,
                         "avg_launch_ms": avg_ms, "traffic": recorded_traffic(dom, N)},
            "kernels": kernels,
            "gpu_launches": int(gpu_launches),
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "batch_64": batch,
            "helmholtz": helm,
            "dirichlet_neumann": dn,
            "long_lines": longl,
            "rk3_step": ns,
        }
        print(json.dumps(line))
    plan.close()
    ranks.close()
    return 0


def _time_ms(fn, warmup, steps):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def bench_configs(args, dev):
    """The small configurations beside the 1024^3 channel (timing only; their parity
    against the oracle is asserted by the GPU tests):
      C1  32^3 unit cube, P/P/NN uniform z, f ~ U[-1,1] (PCG64 seed 0), FP64;
      C2  256^3 unit cube, x, y in {P, NN, DD, ND} (16 pairs), NN tanh z, manufactured
          f + 10 % noise (seed 100 + pair), FP64 and FP32+refine to 1e-10;
      C5  512x256x256 channel box, P/P/NN tanh z, FP32 projection forward + backward
          (u* ~ N(0,1) on faces, seed 5; loss = sum(weights * P(u*)), weights seed 6)."""
    import itertools
    import torch
    from paper_1802_10323_gb300 import autograd, binding as lib, synth
    w_, k_ = max(args.warmup, 3), max(args.steps, 10)
    out = {"case": "configs"}
    zf1 = synth.uniform_faces(32, 1.0)
    f1 = torch.as_tensor(synth.uniform_noise((32, 32, 32), 0), device=dev)
    plan1 = lib.Plan(32, 32, 32, 1 / 32, 1 / 32, zf=zf1, bcs=("P", "P", "NN"), precision="fp64")
    p1 = torch.empty_like(f1)
    ms1 = _time_ms(lambda: plan1.solve(f1, p1), w_, 20 * k_)
    plan1.close()
    out["C1"] = {"ms_per_solve": ms1, "mpts_s": 32 ** 3 / (ms1 * 1e-3) / 1e6, "precision": "fp64"}
    n = 256
    zf2 = synth.tanh_faces(n, 1.0, 1.5)
    c2 = {}
    for prec in ("fp64", "fp32_refine"):
        tot = 0.0
        worst = 0.0
        for idx, bxy in enumerate(itertools.product(("P", "NN", "DD", "ND"), repeat=2)):
            bcs = (bxy[0], bxy[1], "NN")
            _, f = synth.manufactured(n, n, 1.0, 1.0, zf2, bcs, noise=0.1, seed=100 + idx)
            ft = torch.as_tensor(f, device=dev).contiguous()
            pl = lib.Plan(n, n, n, 1 / n, 1 / n, zf=zf2, bcs=bcs, precision=prec, rtol=RTOL, max_iter=MAX_ITER)
            pt, info = torch.empty_like(ft), lib.info_tensor(dev)
            ms = _time_ms(lambda: pl.solve(ft, pt, info=info), w_, k_)
            tot += ms
            if prec == "fp32_refine":
                worst = max(worst, lib.read_info(info).rel_residual)
            pl.close()
        c2[prec] = {"ms_per_solve_mean": tot / 16, "mpts_s": 16 * n ** 3 / (tot * 1e-3) / 1e6}
        if prec == "fp32_refine":
            c2[prec]["max_rel_residual"] = worst
    out["C2"] = c2
    n5 = (512, 256, 256)
    z5 = synth.tanh_faces(n5[2], 1.0, 1.5)
    proj = autograd.Projection(*n5, 6.0 / n5[0], 3.0 / n5[1], zf=z5, bcs=("P", "P", "NN"), precision="fp32")
    us = torch.stack(synth.staggered_velocity_torch(*n5, 5, device=dev)).float().contiguous().requires_grad_(True)
    wts = torch.randn(us.shape, generator=torch.Generator(device=dev).manual_seed(6), device=dev, dtype=torch.float32)

    def step():
        us.grad = None
        (wts * proj(us)).sum().backward()
    ms5 = _time_ms(step, w_, k_)
    proj.close()
    cells = n5[0] * n5[1] * n5[2]
    out["C5"] = {"ms_per_fwd_bwd": ms5, "mcells_s": cells / (ms5 * 1e-3) / 1e6, "precision": "fp32"}
    print(json.dumps(out))
    return 0


def bench_case(args):
    """One small workload for per-kernel ncu captures (not the benchmark line).

    --case solve: the channel right-hand side on an --shape NX,NY,NZ grid of the same
    6 x 3 x 1 box (P/P/NN, tanh z), solved --warmup + --steps times at --precision;
    --case ns: RK3 steps (three ps_ns_substep calls each) on --shape, FP64 fields;
    --case batch: the 64-grid batch, one persistent launch per solve.
    Prints one JSON line with the mean milliseconds per step.
    """
    import torch
    from paper_1802_10323_gb300 import binding as lib, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    shape = tuple(int(x) for x in args.shape.split(",")) if args.shape else (1024, 1024, 64)
    out = {"case": args.case}
    if args.case == "solve":
        f, zf, dx, dy = make_input(shape, GRID["seed"], dev)
        if args.precision == "fp32":
            f = f.float()
        plan = lib.Plan(*shape, dx, dy, zf=zf, bcs=BCS, precision=args.precision, rtol=RTOL, max_iter=MAX_ITER)
        p, info = torch.empty_like(f), lib.info_tensor(dev)
        step = lambda: plan.solve(f, p, info=info)  # noqa: E731
        out.update(shape=list(shape), precision=args.precision)
    elif args.case == "ns":
        zf = synth.tanh_faces(shape[2], 1.0, 1.5)
        plan = lib.Plan(*shape, 6.0 / shape[0], 3.0 / shape[1], zf=zf, bcs=BCS, precision="fp32_refine",
                        rtol=RTOL, max_iter=MAX_ITER)
        u = torch.stack(synth.staggered_velocity_torch(*shape, 5, device=dev)).contiguous()
        us, ad = torch.empty_like(u), torch.zeros_like(u)
        p = torch.zeros((shape[2], shape[1], shape[0]), dtype=torch.float64, device=dev)
        phi, rhs, info = torch.empty_like(p), torch.empty_like(p), lib.info_tensor(dev)

        def step():
            for kk in (1, 2, 3):
                plan.ns_substep(kk, 1e-3, 1.0 / 5600.0, u, us, ad, p, phi, rhs, info=info)
        out.update(shape=list(shape))
    elif args.case == "configs":
        return bench_configs(args, dev)
    elif args.case == "batch":
        from paper_1802_10323_gb300 import workloads
        grids = workloads.batch_grids(64, seed=4)
        plan = lib.Batch(grids, rtol=RTOL, max_iter=MAX_ITER)
        bf = [torch.as_tensor(x, device=dev).contiguous() for x in workloads.batch_rhs(grids, seed=4)]
        bp = [torch.zeros_like(x) for x in bf]
        fptr, pptr = plan.pointers(bf, bp)
        infos = lib.infos_tensor(len(grids), dev)
        step = lambda: plan.solve(fptr, pptr, infos)  # noqa: E731
    else:
        raise SystemExit(f"unknown case {args.case}")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    out["ms_per_step"] = e0.elapsed_time(e1) / max(args.steps, 1)
    plan.close()
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024, help="cells per axis (default: the 1024^3 workload)")
    ap.add_argument("--nz", type=int, default=0,
                    help="cells along z if not --n (an n x n x nz slab of the workload, e.g. for profiling)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-helmholtz", action="store_true")
    ap.add_argument("--no-dn", action="store_true")
    ap.add_argument("--no-long", action="store_true")
    ap.add_argument("--no-ns", action="store_true")
    ap.add_argument("--case", choices=["solve", "ns", "batch", "configs"],
                    help="run one small workload for an ncu capture instead of the benchmark")
    ap.add_argument("--shape", default="", help="NX,NY,NZ of --case solve / ns")
    ap.add_argument("--precision", default="fp32_refine", choices=["fp32_refine", "fp64", "fp32"])
    args = ap.parse_args()
    if args.case:
        return bench_case(args)
    if args.impl == "reference":
        return bench_reference(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
