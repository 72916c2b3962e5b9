"""Laplace's law for static spherical droplets (P9, the sphere half): a
droplet of radius R in its vapour settles to a pressure jump dp = 2 sigma / R
(pressure of Eq. 7), with the sigma that static periodic cylinders give
(dp = sigma / R, `studies.surface_tension`).  Droplets R = 8, 10, 12, 16 in
periodic boxes of side 4 R (the droplet about 7 % of the volume: in a box
much larger than that a small droplet evaporates into the vapour its
Laplace pressure supersaturates), G = -6, tau = 1, from an equilibrium start
with a tanh profile (width 2) at the flat-interface densities; the radius
from the liquid volume between the settled inside and outside densities."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


@pytest.fixture(scope="module")
def L():
    from paper_1904_11792_gb300 import build, lbm
    build.build()
    lbm.load()
    return lbm


def test_spherical_droplets_follow_laplace(L):
    from paper_1904_11792_gb300 import studies
    from paper_1904_11792_gb300.coexistence import coexistence
    G, tau = -6.0, 1.0
    c = coexistence(G, tau)
    rl, rv = c["rho_l"], c["rho_v"]
    sigma = studies.surface_tension(G, tau, rho_l=rl, rho_v=rv)["sigma"]
    for R in (8.0, 10.0, 12.0, 16.0):
        n = int(4 * R)
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        d = np.sqrt((x - (n - 1) / 2) ** 2 + (y - (n - 1) / 2) ** 2 + (z - (n - 1) / 2) ** 2)
        rho0 = rv + 0.5 * (rl - rv) * (1.0 - np.tanh(2.0 * (d - R) / 2.0))
        f0 = W[:, None, None, None] * rho0[None]
        with L.Lattice(n, n, n, tau, G, precision="f32") as lat:
            lat.set_populations(f0)
            lat.step(6000)
            lat.sync()
            rho = lat.rho()
        psi = 1.0 - np.exp(-rho)
        P = rho / 3.0 + G / 6.0 * psi ** 2
        c0 = n // 2
        r_in, r_out = float(rho[c0, c0, c0]), float(rho[0, 0, 0])
        assert r_in > 0.5 * (rl + rv), (R, r_in)          # the droplet is still there
        dp = float(P[c0, c0, c0] - P[0, 0, 0])
        vol = float(np.clip((rho - r_out) / (r_in - r_out), 0.0, 1.0).sum())
        r_eq = (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
        assert abs(dp * r_eq / (2.0 * sigma) - 1.0) < 0.08, (R, r_eq, dp, sigma)
