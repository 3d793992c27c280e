"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the only code shared by the CUDA path's tests/benchmarks and the
CPU oracle. It holds grid construction and random right-hand sides, none of
the solver's arithmetic (no transform, eigenvalue, tridiagonal or Laplacian).

Workloads (domain sizes follow Table 3; the channel box is 6 × 3 × 1):

* ``tanh_faces``: a wall-clustered z grid. The paper allows a non-uniform z
  (footnote to Eq. 5) without giving a stretching law; the one used here is
  z_k = (L/2)(1 + tanh(α(2k/n − 1)) / tanh α), k = 0…n, α = 1.5.
* ``uniform_noise``: i.i.d. U[−1, 1] right-hand side, arithmetic mean removed.
* ``manufactured``: a product of per-axis eigenfunction-like profiles that
  satisfy each BC (P: cos 2πx/L, NN: cos πx/L, DD: sin πx/L, ND: cos πx/2L, DN: sin πx/2L)
  with its analytic Laplacian at the cell centres, plus seeded noise.
* ``staggered_velocity`` / ``divergence_rhs``: a Gaussian random velocity on
  the faces of a staggered grid that is periodic in x and y with walls in z
  (w = 0 on both walls), and its discrete divergence — the right-hand side of
  the pressure equation in a projection step (Eq. 2b), used here only as a
  realistic, compatible input.

NumPy (PCG64) serves the small cases; the 1024³ channel input is drawn on the
GPU with a seeded torch Philox generator (``*_torch`` variants).
"""

import numpy as np


def tanh_faces(n, length=1.0, alpha=1.5):
    """n + 1 face coordinates on [0, length], clustered toward both ends."""
    k = np.arange(n + 1, dtype=np.float64)
    z = 0.5 * length * (1.0 + np.tanh(alpha * (2.0 * k / n - 1.0)) / np.tanh(alpha))
    z[0], z[-1] = 0.0, length
    return z


def uniform_faces(n, length=1.0):
    return np.linspace(0.0, length, n + 1)


def uniform_noise(shape, seed, remove_mean=True):
    """i.i.d. U[−1, 1] in FP64 (PCG64), arithmetic mean removed."""
    f = np.random.default_rng(seed).uniform(-1.0, 1.0, shape)
    if remove_mean:
        f -= f.mean()
    return f


_PROFILE = {
    "P": lambda x, L: (np.cos(2 * np.pi * x / L), (2 * np.pi / L) ** 2),
    "NN": lambda x, L: (np.cos(np.pi * x / L), (np.pi / L) ** 2),
    "DD": lambda x, L: (np.sin(np.pi * x / L), (np.pi / L) ** 2),
    "ND": lambda x, L: (np.cos(0.5 * np.pi * x / L), (0.5 * np.pi / L) ** 2),
    "DN": lambda x, L: (np.sin(0.5 * np.pi * x / L), (0.5 * np.pi / L) ** 2),
}


def manufactured(nx, ny, lx, ly, zf, bcs, noise=0.0, seed=0):
    """(p_exact, f) at cell centres; f = ∇²p_exact (+ noise·max|f|·U[−1,1])."""
    zf = np.asarray(zf, dtype=np.float64)
    xc = (np.arange(nx) + 0.5) * lx / nx
    yc = (np.arange(ny) + 0.5) * ly / ny
    zc = 0.5 * (zf[:-1] + zf[1:])
    lz = zf[-1] - zf[0]
    px, kx = _PROFILE[bcs[0]](xc, lx)
    py, ky = _PROFILE[bcs[1]](yc, ly)
    pz, kz = _PROFILE[bcs[2]](zc - zf[0], lz)
    p = pz[:, None, None] * py[None, :, None] * px[None, None, :]
    f = -(kx + ky + kz) * p
    if noise:
        f = f + noise * np.abs(f).max() * np.random.default_rng(seed).uniform(-1.0, 1.0, f.shape)
    return p, f


def staggered_velocity(nx, ny, nz, seed):
    """(u, v, w) ~ N(0,1) on faces, each [n_z][n_y][n_x]; w = 0 on the bottom wall.

    Face i of a component is the face on the low side of cell i; x and y are
    periodic, the top wall face of w is implicit (zero).
    """
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((nz, ny, nx))
    v = rng.standard_normal((nz, ny, nx))
    w = rng.standard_normal((nz, ny, nx))
    w[0] = 0.0
    return u, v, w


def divergence_rhs(u, v, w, dx, dy, zf):
    """Cell divergence of the staggered field above (periodic x, y; walls in z)."""
    dzf = np.diff(np.asarray(zf, dtype=np.float64))
    f = (np.roll(u, -1, axis=2) - u) / dx + (np.roll(v, -1, axis=1) - v) / dy
    wt = np.concatenate([w[1:], np.zeros_like(w[:1])], axis=0)   # top wall: w = 0
    return f + (wt - w) / dzf[:, None, None]


def staggered_velocity_torch(nx, ny, nz, seed, device="cuda"):
    """Same recipe drawn with a seeded torch (Philox on CUDA) generator, FP64."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    shape = (nz, ny, nx)
    u = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
    v = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
    w = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
    w[0].zero_()
    return u, v, w


def divergence_rhs_torch(u, v, w, dx, dy, zf):
    """torch version of ``divergence_rhs`` (input construction only)."""
    import torch
    dzf = torch.as_tensor(np.diff(np.asarray(zf, dtype=np.float64)), device=u.device)
    f = (torch.roll(u, -1, dims=2) - u) / dx
    f += (torch.roll(v, -1, dims=1) - v) / dy
    f[:-1] += (w[1:] - w[:-1]) / dzf[:-1, None, None]
    f[-1] += (0.0 - w[-1]) / dzf[-1]
    return f
