"""Batched workload description: 64 independent grids of uneven sizes and BCs.

Per-axis sizes are drawn from {32, 48, 64, 96, 128, 192} with caps x ≤ 192,
y ≤ 128, z ≤ 96; each axis gets a BC pair from {P, NN, DD, ND}; z is uniform,
or tanh-stretched (α = 1.5) when it is not periodic; Δ = 1/n per axis (unit
box). Right-hand sides are U[−1, 1] (PCG64), mean removed for singular grids.
"""

import numpy as np

from . import synth

SIZES = (32, 48, 64, 96, 128, 192)
BCS = ("P", "NN", "DD", "ND")


def batch_grids(count=64, seed=4):
    rng = np.random.default_rng(seed)
    grids = []
    for _ in range(count):
        nx = int(rng.choice([s for s in SIZES if s <= 192]))
        ny = int(rng.choice([s for s in SIZES if s <= 128]))
        nz = int(rng.choice([s for s in SIZES if s <= 96]))
        bcs = tuple(str(b) for b in rng.choice(BCS, 3))
        stretched = bcs[2] != "P" and bool(rng.integers(0, 2))
        zf = synth.tanh_faces(nz, 1.0, 1.5) if stretched else synth.uniform_faces(nz, 1.0)
        grids.append(dict(nx=nx, ny=ny, nz=nz, dx=1.0 / nx, dy=1.0 / ny, zf=zf, bcs=bcs))
    return grids


def batch_rhs(grids, seed=4):
    out = []
    for g, d in enumerate(grids):
        singular = all(b in ("P", "NN") for b in d["bcs"])
        out.append(synth.uniform_noise((d["nz"], d["ny"], d["nx"]), seed=1000 * seed + g,
                                       remove_mean=singular))
    return out
