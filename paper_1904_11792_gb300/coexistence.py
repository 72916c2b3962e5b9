"""Flat-interface coexistence run on the GPU.

The liquid and vapour densities of the pseudo-potential model at a given
(G, tau) are not known in closed form: the equation of state (Eq. 7) fixes
them only together with the forcing scheme.  As the ligament set-up needs
them, they are measured the usual way: a liquid slab across x in a periodic
n x 3 x 3 box is relaxed until the density field stops changing, and the
densities at the slab centre and the vapour centre are read off.  The
converged interface profile rho(d) doubles as the tabulated initial profile
for runs that the sharp tanh initial condition would destabilise.

All stepping runs in liblbm.so (FP64 storage).  Only the slab's starting
populations f_a = w_a rho(x) are filled on the host.
"""
from __future__ import annotations

import math

import numpy as np

from . import lbm as L


def _slab(n: int, rho_l: float, rho_v: float) -> np.ndarray:
    _, w = L.lbm_lattice()
    x = np.arange(n, dtype=np.float64)
    rho = rho_v + 0.5 * (rho_l - rho_v) * (np.tanh(x - 0.25 * n) - np.tanh(x - 0.75 * n))
    f = np.empty((19, 3, 3, n))
    f[:] = (w[:, None] * rho[None, :])[:, None, None, :]
    return f


def coexistence(G: float, tau: float, n: int = 64, tol: float = 1e-10, check: int = 1000,
                max_steps: int = 400000, rho_l0: float | None = None, rho_v0: float | None = None,
                tau_start: float | None = None, psi_form: int = L.LBM_PSI_EXP, rho0: float = 1.0,
                options: dict | None = None):
    """Relax a flat slab at (G, tau); returns dict(rho_l, rho_v, steps, dmax,
    profile, d0, dd) with profile = rho along the outward normal of one
    interface, sampled at d0 + k dd.

    Below tau = 0.8 the slab is first relaxed at tau_start (default 1.0) and
    then continued at tau, since the sharp tanh start can drive the density
    negative at small tau with strong attraction.  options: lattice options
    to set first (e.g. {"collision": 1} for the MRT collision)."""
    if rho_l0 is None:
        rho_l0 = 2.6 if G <= -5.8 else 2.1
    if rho_v0 is None:
        rho_v0 = 0.07 if G <= -5.8 else 0.1
    if tau_start is None:
        tau_start = 1.0 if tau < 0.8 else tau
    lat = L.Lattice(n, 3, 3, tau_start, G, precision="f64", pattern="ab", psi_form=psi_form,
                    rho0=rho0)
    try:
        for k, v in (options or {}).items():
            lat.set_option(k, v)
        lat.set_populations(_slab(n, rho_l0, rho_v0))
        taus = [tau_start] if tau_start == tau else [tau_start, tau]
        steps = 0
        dmax = math.inf
        for t in taus:
            lat.set_option("tau", t)
            prev = lat.rho()[1, 1]
            dmax = math.inf
            while steps < max_steps:
                lat.step(check)
                steps += check
                cur = lat.rho()[1, 1]
                if not np.isfinite(cur).all():
                    raise FloatingPointError("coexistence run diverged at tau=%g" % t)
                dmax = float(np.abs(cur - prev).max())
                prev = cur
                if dmax < tol:
                    break
        rho = prev
    finally:
        lat.close()
    rho_l, rho_v = float(rho[n // 2]), float(rho[0])
    # outward profile of the interface between the slab centre and x = n - 1
    half = 0.5 * (rho_l + rho_v)
    xs = np.arange(n // 2, n)
    seg = rho[n // 2:]
    k = int(np.flatnonzero(seg <= half)[0])
    xc = xs[k - 1] + (seg[k - 1] - half) / (seg[k - 1] - seg[k])
    return dict(rho_l=rho_l, rho_v=rho_v, steps=steps, dmax=dmax, profile=seg.copy(),
                d0=float(xs[0] - xc), dd=1.0)
