"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds random numbers and workload parameters only: it does none
of the lattice Boltzmann arithmetic.  Both the GPU path's tests and the
oracle's tests draw their inputs here, so the two sides see the same data.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out from its published
definition.  The base seed of every workload is 1904117920.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1904117920
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of SplitMix64 started from state `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# Per-direction-class value ranges of a population divided by the local
# density, for the canonical D3Q19 order (rest, 6 axis, 12 diagonal).
# These are the value distributions seen in the ligament runs, used to make
# random but physically plausible states; they are inputs, not a formula.
_CLASS = np.array([0] + [1] * 6 + [2] * 12)
_LO = np.array([0.30, 0.045, 0.022])
_HI = np.array([0.36, 0.066, 0.033])


def random_populations(nx: int, ny: int, nz: int, seed: int = BASE_SEED, rho_lo: float = 0.1,
                       rho_hi: float = 2.6, smooth: bool = True) -> np.ndarray:
    """A random state f[19, nz, ny, nx] (float64).

    f_a(x) = d(x) * r_a(x), with d a density-like field in [rho_lo, rho_hi]
    (smooth: a few random Fourier modes on the periodic box; otherwise
    white noise) and r_a uniform in the direction class's range."""
    N = nx * ny * nz
    if smooth:
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        u = uniform(seed, 24)
        d = np.zeros((nz, ny, nx))
        for m in range(4):
            kx, ky, kz = 1 + int(3 * u[6 * m]), int(3 * u[6 * m + 1]), int(3 * u[6 * m + 2])
            ph = 2 * math.pi * u[6 * m + 3]
            amp = 0.5 + u[6 * m + 4]
            d += amp * np.cos(2 * math.pi * (kx * xx / nx + ky * yy / ny + kz * zz / nz) + ph)
        d = (d - d.min()) / max(d.max() - d.min(), 1e-300)
    else:
        d = uniform(seed, N).reshape(nz, ny, nx)
    d = rho_lo + (rho_hi - rho_lo) * d
    r = uniform(seed ^ 0x5DEECE66D, 19 * N).reshape(19, nz, ny, nx)
    lo = _LO[_CLASS][:, None, None, None]
    hi = _HI[_CLASS][:, None, None, None]
    return d[None] * (lo + (hi - lo) * r)


# ----------------------------------------------------------------------------
# Workloads.  Sizes and parameters of the ligament runs; G = -6, psi form 0.
# ----------------------------------------------------------------------------

@dataclass
class Ligament:
    name: str
    nx: int
    ny: int
    nz: int
    R0: float
    lam: float
    eps: float
    tau: float
    phase: float = 0.0
    G: float = -6.0
    width: float = 2.0
    steps: int = 1000
    extra: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz


# Small parity case: 64x32x32, R0 = 8, lambda = 64 (kR0 = 0.785), eps 0.05.
PARITY_64 = Ligament("ligament 64x32x32 R0=8 fp64", 64, 32, 32, 8.0, 64.0, 0.05, 1.0, steps=1000)
# Grid-convergence ligament: 256x128x128, R0 = 32, lambda = 256, eps 0.02.
GRID_256 = Ligament("ligament 256x128x128 R0=32 fp32", 256, 128, 128, 32.0, 256.0, 0.02, 1.0,
                    steps=20000)
# Precision form: 512x256x256, R0 = 48, lambda = 512, eps 0.01, tau 0.8.
PRECISION_512 = Ligament("ligament 512x256x256 R0=48", 512, 256, 256, 48.0, 512.0, 0.01, 0.8,
                         steps=30000)
# Large single ligament: 1024x512x512, R0 = 96, lambda = 1024, eps 0.01, tau 0.7.
LARGE_1024 = Ligament("ligament 1024x512x512 R0=96", 1024, 512, 512, 96.0, 1024.0, 0.01, 0.7,
                      steps=5000)
# The large ligament at tau = 1 instead of 0.7 (tau = 0.7 is unstable for the
# SRT collision at G = -6 from either start): throughput at 268 M nodes.
GRID_1024 = Ligament("ligament 1024x512x512 R0=96 tau=1", 1024, 512, 512, 96.0, 1024.0, 0.01, 1.0,
                     steps=5000)


def batched_sweep(count: int = 48, seed: int = BASE_SEED) -> list[Ligament]:
    """The uneven batch: R0 uniform in {8,12,16,20,24}, lambda = round(r R0)
    with r ~ U[4.5, 12], tau ~ U[0.6, 1.0], phase ~ U[0, 2 pi), eps = 0.05,
    box lambda x 4 R0 x 4 R0."""
    u = uniform(seed ^ 0xBA7C4, 4 * count).reshape(count, 4)
    radii = (8, 12, 16, 20, 24)
    out = []
    for k in range(count):
        R0 = radii[min(int(u[k, 0] * 5), 4)]
        r = 4.5 + 7.5 * u[k, 1]
        lam = int(round(r * R0))
        tau = 0.6 + 0.4 * u[k, 2]
        phase = 2 * math.pi * u[k, 3]
        out.append(Ligament("batch[%d] R0=%d lam=%d" % (k, R0, lam), lam, 4 * R0, 4 * R0,
                            float(R0), float(lam), 0.05, tau, phase=phase))
    return out


def droplet_populations(nx: int, ny: int, nz: int, seed: int = BASE_SEED, p: float = 0.3,
                        rho_l: float = 2.65, rho_v: float = 0.073, mask=None) -> np.ndarray:
    """A state f[19, nz, ny, nx] (float64) whose liquid forms many droplets.

    Liquid nodes (a uniform draw below p, or the given boolean mask) get a
    density in [0.9, 1.1] rho_l, the others one in [0.5, 1.5] rho_v, far from
    the threshold (rho_l + rho_v)/2 in any storage precision.  The density is
    spread over the 19 populations by positive random shares."""
    N = nx * ny * nz
    u = uniform(seed, 2 * N)
    if mask is None:
        mask = (u[:N] < p).reshape(nz, ny, nx)
    mask = np.asarray(mask, dtype=bool)
    v = u[N:].reshape(nz, ny, nx)
    rho = np.where(mask, rho_l * (0.9 + 0.2 * v), rho_v * (0.5 + v))
    share = 0.5 + uniform(seed ^ 0x2545F491, 19 * N).reshape(19, nz, ny, nx)
    share /= share.sum(axis=0, keepdims=True)
    return share * rho[None]
