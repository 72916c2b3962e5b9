"""Second, independent NumPy oracle of the D3Q19 Shan-Chen step (tiny grids).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  It is written
separately from the C oracle, in whole-array NumPy form, and exists only to
cross-check it on small lattices (brute force by an independent route).

The velocity set is generated rather than typed in: every c in {-1,0,1}^3
with |c|^2 <= 2 (D3Q19), weight 1/3, 1/18, 1/36 by |c|^2 = 0, 1, 2 (the
standard weights the paper calls "normalised to unity", reading R6).  Its
direction order is its own (lexicographic); ``perm_to`` maps it onto any
other table.  Arrays: f[a, z, y, x], streaming by ``np.roll`` (periodic).
"""
from __future__ import annotations

import itertools

import numpy as np

VEL = np.array([c for c in itertools.product((-1, 0, 1), repeat=3)
                if sum(v * v for v in c) <= 2], dtype=np.int64)          # (19, 3): cx, cy, cz
WGT = np.array([{0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}[int(v @ v)] for v in VEL])
CS2 = 1.0 / 3.0


def perm_to(c_other: np.ndarray) -> np.ndarray:
    """Index array p with VEL[p[k]] == c_other[k]."""
    return np.array([int(np.flatnonzero((VEL == np.asarray(c)).all(axis=1))[0])
                     for c in c_other])


def shift(a: np.ndarray, c) -> np.ndarray:
    """Array b with b[x + c] = a[x] (periodic) for a[..., z, y, x]."""
    return np.roll(a, shift=(int(c[2]), int(c[1]), int(c[0])), axis=(-3, -2, -1))


def psi_of(rho: np.ndarray, form: int = 0, rho0: float = 1.0) -> np.ndarray:
    return rho.copy() if form == 1 else rho0 * (1.0 - np.exp(-rho / rho0))


def one_step(f: np.ndarray, tau: float, G: float, form: int = 0, rho0: float = 1.0) -> np.ndarray:
    """One step, whole-array form (same equations as the paper, Eqs. 2-6)."""
    rho = f.sum(axis=0)
    j = np.einsum("ak,azyx->kzyx", VEL.astype(float), f)
    psi = psi_of(rho, form, rho0)
    # sum_a w_a psi(x + c_a) c_a : psi(x + c) is psi shifted by -c
    acc = np.zeros((3,) + rho.shape)
    for a in range(19):
        acc += WGT[a] * shift(psi, -VEL[a])[None] * VEL[a][:, None, None, None]
    F = -G * psi[None] * acc
    u = (j + tau * F) / rho[None]
    cu = np.einsum("ak,kzyx->azyx", VEL.astype(float), u)
    uu = (u * u).sum(axis=0)
    feq = WGT[:, None, None, None] * rho[None] * (1.0 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2)
                                                  - uu[None] / (2 * CS2))
    post = f - (f - feq) / tau
    return np.stack([shift(post[a], VEL[a]) for a in range(19)])


def run(f: np.ndarray, tau: float, G: float, nsteps: int, form: int = 0,
        rho0: float = 1.0) -> np.ndarray:
    g = np.array(f, dtype=np.float64)
    for _ in range(nsteps):
        g = one_step(g, tau, G, form, rho0)
    return g
