"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks a closed
form, an invariant, a special case, a printed value of the paper (Table 1),
an independent implementation (the NumPy micro-oracle) or a brute-force
library routine (networkx connected components).
"""
import math
import os
import warnings
from concurrent.futures import ProcessPoolExecutor
from fractions import Fraction
import multiprocessing as mp

import numpy as np
import pytest

import lbm_inputs
import oracle
from oracle import np_oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# P1: D3Q19 lattice identities (exact rationals)
# --------------------------------------------------------------------------

def test_lattice_isotropy_exact():
    c, w, opp = oracle.lattice()
    wf = [Fraction(x).limit_denominator(100) for x in w]
    for x, q in zip(w, wf):
        assert abs(x - float(q)) <= 1e-16
    assert sorted(set(wf)) == [Fraction(1, 36), Fraction(1, 18), Fraction(1, 3)]
    assert sum(wf) == 1
    for i in range(3):
        assert sum(wf[a] * c[a, i] for a in range(19)) == 0
        for j in range(3):
            assert sum(wf[a] * c[a, i] * c[a, j] for a in range(19)) == Fraction(int(i == j), 3)
            for k in range(3):
                assert sum(wf[a] * c[a, i] * c[a, j] * c[a, k] for a in range(19)) == 0
                for l in range(3):
                    d = lambda p, q: int(p == q)
                    want = Fraction(d(i, j) * d(k, l) + d(i, k) * d(j, l) + d(i, l) * d(j, k), 9)
                    got = sum(wf[a] * c[a, i] * c[a, j] * c[a, k] * c[a, l] for a in range(19))
                    assert got == want
    # weights by speed class, opposite table, canonical order
    for a in range(19):
        assert wf[a] == {0: Fraction(1, 3), 1: Fraction(1, 18), 2: Fraction(1, 36)}[
            int(c[a] @ c[a])]
        assert (c[opp[a]] == -c[a]).all()
    assert (c[0] == 0).all()
    assert [tuple(v) for v in c[1:7]] == [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                          (0, 0, 1), (0, 0, -1)]
    assert len({tuple(v) for v in c}) == 19


# --------------------------------------------------------------------------
# P2: moments of the equilibrium (Eq. 2 with reading R1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (2.7, (0.03, -0.01, 0.02)),
                                   (0.07, (-0.1, 0.05, 0.08))])
def test_equilibrium_moments(rho, u):
    c, w, _ = oracle.lattice()
    fe = oracle.feq(rho, u)
    u = np.array(u)
    assert abs(fe.sum() - rho) <= 1e-15 * rho
    np.testing.assert_allclose(c.T @ fe, rho * u, atol=1e-15 * rho)
    pi = np.einsum("ai,aj,a->ij", c, c, fe)
    np.testing.assert_allclose(pi, rho / 3.0 * np.eye(3) + rho * np.outer(u, u), atol=2e-15 * rho)
    if not u.any():
        np.testing.assert_array_equal(fe, w * rho)


def test_psi_functional():
    # psi = rho0 (1 - exp(-rho / rho0)) (text after Eq. 5); psi = rho form for tests
    assert oracle.psi(0.0) == 0.0
    assert abs(oracle.psi(math.log(2.0)) - 0.5) < 1e-16
    assert abs(oracle.psi(50.0) - 1.0) < 1e-16
    assert abs(oracle.psi(1.0, 0, 2.0) - 2.0 * (1 - math.exp(-0.5))) < 1e-15
    assert oracle.psi(1.7, 1) == 1.7


# --------------------------------------------------------------------------
# P3: uniform states are fixed points (F = 0 for uniform psi)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("u0", [(0.0, 0.0, 0.0), (0.04, -0.02, 0.01)])
def test_uniform_fixed_point(u0):
    rho0 = 0.7
    fe = oracle.feq(rho0, u0)
    f = np.broadcast_to(fe[:, None, None, None], (19, 4, 5, 6)).copy()
    g = oracle.step(f, tau=0.8, G=-6.0, nsteps=50)
    np.testing.assert_allclose(g, f, rtol=2e-15, atol=0)


# --------------------------------------------------------------------------
# P4: single-phase BGK shear wave (G = 0): decay exp(-nu k^2 t),
# nu = (tau - 1/2)/3, and advection by a uniform stream (streaming direction)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("tau,U", [(0.8, 0.0), (1.2, 0.0), (0.9, 0.05)])
def test_shear_wave_decay_and_advection(tau, U):
    nx, ny, nz = 64, 3, 3
    k = 2 * math.pi / nx
    A0 = 1e-3
    x = np.arange(nx)
    f = np.zeros((19, nz, ny, nx))
    for i in range(nx):
        f[:, :, :, i] = oracle.feq(1.0, (U, A0 * math.sin(k * i), 0.0))[:, None, None]

    def amp_phase(g):
        rho, ux, uy, uz = oracle.moments(g, G=0.0, bare=True)
        prof = uy[0, 0]
        z = (prof * np.exp(-1j * k * x)).sum() * 2 / nx
        return abs(z), np.angle(z)

    t1, t2 = 200, 1200
    g1 = oracle.step(f, tau, 0.0, t1)
    g2 = oracle.step(g1, tau, 0.0, t2 - t1)
    a1, p1 = amp_phase(g1)
    a2, p2 = amp_phase(g2)
    nu = (tau - 0.5) / 3.0
    rate = -math.log(a2 / a1) / (t2 - t1)
    assert abs(rate / (nu * k * k) - 1.0) < 0.01
    # a pattern advected by +U: the phase of sin(k(x - U t)) drops by k U t
    err = ((p2 - p1) + k * U * (t2 - t1) + math.pi) % (2 * math.pi) - math.pi
    assert abs(err) < 0.02


# --------------------------------------------------------------------------
# P5: conservation — mass, and total momentum (sum_x F = 0 on a periodic box)
# --------------------------------------------------------------------------

def test_mass_and_momentum_conservation():
    c, _, _ = oracle.lattice()
    f = lbm_inputs.random_populations(12, 10, 8, seed=7)
    M0 = f.sum()
    J0 = np.einsum("ak,azyx->k", c.astype(float), f)
    g = oracle.step(f, tau=0.9, G=-5.5, nsteps=300)
    assert abs(g.sum() - M0) / M0 <= 1e-13
    J1 = np.einsum("ak,azyx->k", c.astype(float), g)
    assert np.abs(J1 - J0).max() <= 1e-12 * M0
    # the force field itself sums to zero
    F = oracle.force(f, G=-5.5)
    assert np.abs(F.sum(axis=(1, 2, 3))).max() <= 1e-13 * np.abs(F).sum()


# The exported velocity of reading R7, u = (j + F/2)/rho.  At a converged
# flat interface (a periodic slab, uniform across y and z) the discrete step
# itself fixes j + F/2 = 0 at every node: steady mass balance makes the
# population flux Phi through every x face the same, and the total momentum
# (zero at the start, conserved because sum F = 0) makes it zero; the
# pre-collision momentum at x is the flux in from both faces' post-collision
# populations and the post-collision momentum (j + F under the velocity
# shift of Eq. 6) the flux out, so j + (j + F) = Phi(x - 1/2) + Phi(x + 1/2)
# = 0.  The bare j/rho = -F/(2 rho) there is of order 1e-2, so a wrong
# half-force factor (0, 1, -1/2) fails.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("tau,G", [(1.0, -6.0), (0.8, -5.3)])
def test_r7_velocity_vanishes_at_a_steady_flat_interface(tau, G):
    r = oracle.coexistence(tau, G, n=48, tol=1e-13, rho_l0=2.4, rho_v0=0.1)
    f = r["f"]
    rho, ux, uy, uz = oracle.moments(f, G)
    _, bx, by, bz = oracle.moments(f, G, bare=True)
    assert np.abs(bx).max() > 5e-3                       # the force does act on the interface
    assert max(np.abs(ux).max(), np.abs(uy).max(), np.abs(uz).max()) < 1e-9
    assert np.abs(by).max() < 1e-14 and np.abs(bz).max() < 1e-14


def test_r7_velocity_total_momentum_is_sum_j():
    # sum_x rho u = sum_x j + sum_x F/2 = sum_x j on a periodic box (sum F = 0)
    c, _, _ = oracle.lattice()
    f = lbm_inputs.random_populations(10, 9, 7, seed=31)
    rho, ux, uy, uz = oracle.moments(f, -5.8)
    J = np.einsum("ak,azyx->k", c.astype(float), f)
    P = np.array([(rho * u).sum() for u in (ux, uy, uz)])
    assert np.abs(P - J).max() <= 1e-12 * rho.sum()
    # and node by node the velocity differs from the bare one by F/(2 rho)
    F = oracle.force(f, -5.8)
    _, bx, by, bz = oracle.moments(f, -5.8, bare=True)
    np.testing.assert_allclose(np.stack([ux, uy, uz]) - np.stack([bx, by, bz]),
                               0.5 * F / rho[None], rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------
# P6: brute force against the independent NumPy oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,tau,G,form", [((8, 8, 8), 0.8, -5.5, 0), ((5, 3, 7), 1.0, -6.0, 0),
                                              ((6, 4, 5), 0.7, -1.0, 1)])
def test_c_oracle_vs_numpy_oracle(shape, tau, G, form):
    nx, ny, nz = shape
    c, _, _ = oracle.lattice()
    p = np_oracle.perm_to(c)            # numpy index of the oracle's direction a
    f = lbm_inputs.random_populations(nx, ny, nz, seed=11, smooth=False, rho_lo=0.3, rho_hi=2.0)
    g_c = oracle.step(f, tau, G, nsteps=20, psi_form=form)
    fn = np.zeros_like(f)
    fn[p] = f
    g_np = np_oracle.run(fn, tau, G, 20, form)[p]
    assert np.abs(g_c - g_np).max() <= 1e-13 * np.abs(g_np).max()


def test_step_nodes_matches_full_step():
    f = lbm_inputs.random_populations(9, 7, 6, seed=3)
    full = oracle.step(f, 0.85, -5.8, 1)
    nodes = np.array([0, 1, 8, 9, 62, 63, 100, 377])
    got = oracle.step_nodes(f, nodes, 0.85, -5.8)
    want = full.reshape(19, -1)[:, nodes].T
    np.testing.assert_allclose(got, want, rtol=1e-15, atol=0)


# --------------------------------------------------------------------------
# P7: Table 1 — flat-interface coexistence densities at G = -5.3
# --------------------------------------------------------------------------

def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def tau_from_oh(R0, rho_l, sigma, Oh=0.1):
    """tau from Oh = nu sqrt(rho_l / (sigma R0)), nu = (tau - 1/2)/3 (reading R10)."""
    nu = Oh * math.sqrt(sigma * R0 / rho_l)
    return 0.5 + 3.0 * nu


def _coex(tau):
    import oracle as o
    r = o.coexistence(tau, -5.3, n=64, tol=1e-10, rho_l0=2.1, rho_v0=0.1)
    return r["rho_l"], r["rho_v"]


def test_table1_coexistence_densities():
    rows = _table1()
    assert len(rows) == 7
    taus = [tau_from_oh(R0, rl, s) for R0, rl, rv, s in rows]
    # the Oh = 0.1 reading gives tau from 0.624 (R0 = 7) to 1.035 (R0 = 84)
    assert abs(taus[0] - 0.624) < 1e-3 and abs(taus[-1] - 1.035) < 1e-3
    with ProcessPoolExecutor(max_workers=min(7, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_coex, taus))
    for (R0, rl, rv, s), (ol, ov) in zip(rows, res):
        assert abs(ol - rl) <= 0.003, (R0, ol, rl)
        assert abs(ov - rv) <= 0.002, (R0, ov, rv)


# --------------------------------------------------------------------------
# Ligament initial condition (set-up section, readings R9, R11-R13)
# --------------------------------------------------------------------------

def test_ligament_init_geometry():
    nx, ny, nz = 32, 25, 25
    R0, lam, eps, ph, rl, rv, W = 6.0, 32.0, 0.1, 0.4, 2.6, 0.07, 2.0
    f = oracle.init_ligament(nx, ny, nz, R0, lam, eps, ph, rl, rv, W)
    c, w, _ = oracle.lattice()
    rho = f.sum(axis=0)
    # zero velocity, populations proportional to the weights
    np.testing.assert_allclose(f / rho[None], np.broadcast_to(w[:, None, None, None], f.shape),
                               rtol=1e-15)
    assert np.abs(np.einsum("ak,azyx->kzyx", c.astype(float), f)).max() < 1e-15
    # axis symmetry about y = z = 12 (the centre node of a 25-wide section)
    np.testing.assert_allclose(rho, rho[:, ::-1, :], rtol=1e-15)
    np.testing.assert_allclose(rho, rho[::-1, :, :], rtol=1e-15)
    np.testing.assert_allclose(rho, np.transpose(rho, (1, 0, 2)), rtol=1e-15)
    # deep inside / far outside, within the tanh tail exp(-2 * 2 * 5.4 / W)
    assert abs(rho[12, 12, 0] - rl) < 1e-5 and abs(rho[0, 0, 0] - rv) < 1e-8
    # half-level radius along +y recovered by inverting the profile at the node
    # nearest the interface: mean R0, amplitude eps*R0, maximum where the
    # phase 2 pi x / lam + ph is 0 (mod 2 pi)
    est = []
    for x in range(nx):
        prof = rho[12, 12:, x]
        r = int(np.argmin(np.abs(prof - 0.5 * (rl + rv))))
        t = 1.0 - 2.0 * (prof[r] - rv) / (rl - rv)
        est.append(r - W / 2.0 * math.atanh(t))
    est = np.array(est)
    assert abs(est.mean() - R0) < 1e-9
    assert abs((est.max() - est.min()) / 2 - eps * R0) < 0.02 * eps * R0
    xs = np.arange(nx)
    z = (est * np.exp(-2j * math.pi * xs / lam)).sum() * 2 / nx
    assert abs(abs(z) - eps * R0) < 1e-9 and abs(np.angle(z) - ph) < 1e-9


# Tabulated-profile initial condition (reading R15): rho = prof(d) with d the
# signed distance to the perturbed interface, linear interpolation between
# the table's nodes and clamped beyond its ends.  Pinned to numpy's own
# piecewise-linear interpolation (np.interp, which clamps the same way) on a
# non-monotone table whose range leaves nodes clamped at both ends, and to
# the pinned tanh initial condition: a finely tabulated tanh profile must
# reproduce orc_init_ligament to the interpolation error.
# --------------------------------------------------------------------------

def _signed_distance(nx, ny, nz, R0, lam, eps, ph):
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    R = R0 * (1.0 + eps * np.cos(2 * math.pi * xx / lam + ph))
    return np.hypot(yy - 0.5 * (ny - 1), zz - 0.5 * (nz - 1)) - R


def test_init_profile_is_clamped_linear_interpolation():
    nx, ny, nz = 20, 22, 22
    R0, lam, eps, ph = 5.0, 20.0, 0.15, 0.9
    prof = 0.05 + 2.6 * lbm_inputs.uniform(77, 23)      # not monotone: every segment differs
    d0, dd = -3.1, 0.45                                  # table covers d in [-3.1, 6.8]
    f = oracle.init_profile(nx, ny, nz, R0, lam, eps, ph, prof, d0, dd)
    _, w, _ = oracle.lattice()
    d = _signed_distance(nx, ny, nz, R0, lam, eps, ph)
    assert (d < d0).any() and (d > d0 + dd * (prof.size - 1)).any()   # both clamps used
    rho = np.interp(d, d0 + dd * np.arange(prof.size), prof)
    np.testing.assert_allclose(f, w[:, None, None, None] * rho[None], rtol=1e-13, atol=0)


def test_init_profile_of_a_fine_tanh_table_is_the_tanh_start():
    nx, ny, nz = 24, 26, 26
    R0, lam, eps, ph, rl, rv, W = 6.0, 24.0, 0.1, 0.4, 2.6, 0.07, 2.0
    d0, dd = -20.0, 0.01
    dk = d0 + dd * np.arange(4001)
    prof = rv + 0.5 * (rl - rv) * (1.0 - np.tanh(2.0 * dk / W))
    f = oracle.init_profile(nx, ny, nz, R0, lam, eps, ph, prof, d0, dd)
    g = oracle.init_ligament(nx, ny, nz, R0, lam, eps, ph, rl, rv, W)
    # linear interpolation error <= dd^2/8 max|rho''|; |rho''| <= 0.77 (rl - rv)(2/W)^2 / 2
    bound = dd * dd / 8 * 0.77 * (rl - rv) * (2.0 / W) ** 2 / 2 / 3   # times w_0 = 1/3
    err = np.abs(f - g).max()
    assert err <= 1.05 * bound, (err, bound)
    assert err > 0.05 * bound         # the table really is interpolated, not evaluated


# --------------------------------------------------------------------------
# Connected components (droplet count) against networkx
# --------------------------------------------------------------------------

def _nx_components(mask):
    import networkx as nx_
    nz, ny, nx = mask.shape
    g = nx_.Graph()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not mask[z, y, x]:
                    continue
                g.add_node((z, y, x))
                for dz, dy, dx in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):
                    q = ((z + dz) % nz, (y + dy) % ny, (x + dx) % nx)
                    if mask[q]:
                        g.add_edge((z, y, x), q)
    return sorted(len(cc) for cc in nx_.connected_components(g))


@pytest.mark.parametrize("seed,shape,p", [(1, (5, 6, 7), 0.3), (2, (4, 4, 4), 0.45),
                                          (3, (3, 8, 5), 0.25), (4, (6, 5, 9), 0.35)])
def test_ccl_vs_networkx(seed, shape, p):
    mask = lbm_inputs.uniform(seed, int(np.prod(shape))).reshape(shape) < p
    n, labels, sizes = oracle.ccl(mask)
    want = _nx_components(mask)
    assert n == len(want)
    assert sorted(sizes.tolist()) == want
    assert ((labels >= 0) == mask).all()


def test_ccl_periodic_wrap():
    mask = np.zeros((5, 5, 8), dtype=bool)
    mask[2, 2, :] = True                 # a line through the x boundary: one component
    mask[0, 0, 0] = mask[4, 0, 0] = True  # joined across z
    n, _, sizes = oracle.ccl(mask)
    assert n == 2 and sorted(sizes.tolist()) == [2, 8]
    mask[2, 2, 3] = False                # cut once: the ring is still one piece
    assert oracle.ccl(mask)[0] == 2
    mask[2, 2, 6] = False                # cut twice: two pieces
    assert oracle.ccl(mask)[0] == 3


# --------------------------------------------------------------------------
# Diagnostics against an independent numpy evaluation
# --------------------------------------------------------------------------

def test_diagnostics_vs_numpy():
    nx, ny, nz = 20, 16, 16
    rl, rv = 2.6, 0.07
    f = oracle.init_ligament(nx, ny, nz, 4.0, 20.0, 0.3, 0.0, rl, rv, 2.0)
    f = oracle.step(f, 1.0, -6.0, 5)
    d, sw, sn = oracle.diagnostics(f, rl, rv, slices=True)
    c, _, _ = oracle.lattice()
    rho = f.sum(axis=0)
    j = np.einsum("ak,azyx->kzyx", c.astype(float), f)
    phi = np.clip((rho - rv) / (rl - rv), 0, 1)
    liq = rho > 0.5 * (rl + rv)
    assert abs(d["mass"] - rho.sum()) <= 1e-12 * rho.sum()
    np.testing.assert_allclose([d["mom_x"], d["mom_y"], d["mom_z"]], j.sum(axis=(1, 2, 3)),
                               atol=1e-12 * rho.sum())
    assert abs(d["liquid_volume_w"] - phi.sum()) <= 1e-12 * phi.sum()
    assert d["liquid_count"] == liq.sum()
    np.testing.assert_allclose(sw, phi.sum(axis=(0, 1)), rtol=1e-12)
    np.testing.assert_array_equal(sn, liq.sum(axis=(0, 1)))
    assert d["min_slice_count"] == liq.sum(axis=(0, 1)).min()
    assert d["min_slice_x"] == int(np.argmin(liq.sum(axis=(0, 1))))
    assert abs(d["max_u"] - (np.sqrt((j ** 2).sum(axis=0)) / rho).max()) < 1e-15
    assert d["numeric_ok"] == 1.0
    assert abs(d["neck_radius"] - math.sqrt(phi.sum(axis=(0, 1)).min() / math.pi)) < 1e-12


# --------------------------------------------------------------------------
# P9: Laplace law on static cylinders, pressure from the EOS (Eq. 7);
# surface tension against Table 1 (R0 = 84 column, tau = 1.035)
# --------------------------------------------------------------------------

def _laplace_cylinder(R):
    import numpy as np
    import oracle as o
    G, tau = -5.3, 1.0351
    r = o.coexistence(tau, G, n=64, tol=1e-10, rho_l0=2.1, rho_v0=0.1)
    n = 49
    f = o.init_ligament(3, n, n, R, 3.0, 0.0, 0.0, r["rho_l"], r["rho_v"], 2.0)
    prev = None
    for _ in range(40):
        f = o.step(f, tau, G, 500)
        rho = f.sum(axis=0)[:, :, 1]
        if prev is not None and np.abs(rho - prev).max() < 1e-9:
            break
        prev = rho
    # Eq. 7: P = rho cs^2 + cs^2 G psi^2 / 2, cs^2 = 1/3
    psi = 1.0 - np.exp(-rho)
    P = rho / 3.0 + G / 6.0 * psi ** 2
    return P[24, 24] - P[0, 0]


def test_laplace_law_and_table1_surface_tension():
    radii = [8.0, 10.0, 12.0, 16.0]
    with ProcessPoolExecutor(max_workers=min(4, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        dps = list(ex.map(_laplace_cylinder, radii))
    # cylinder: dp = sigma / R; dp * R is the same for every radius
    prods = [dp * R for dp, R in zip(dps, radii)]
    assert max(prods) / min(prods) - 1.0 < 0.03, prods
    inv = np.array([1.0 / R for R in radii])
    sigma = float(inv @ np.array(dps) / (inv @ inv))
    sigma_table = _table1()[-1][3]          # R0 = 84 column: tau = 1.035
    assert abs(sigma / sigma_table - 1.0) < 0.05, (sigma, sigma_table)


# --------------------------------------------------------------------------
# P10: Plateau-Rayleigh instability of a periodic ligament: a small cosine
# perturbation grows iff k R0 < 1 (the cut-off of the Rayleigh dispersion)
# --------------------------------------------------------------------------

def _ligament_mode_amplitude(kR):
    import math
    import numpy as np
    import oracle as o
    rl, rv, R0 = 2.648878066946715, 0.0731992478525716, 6.0
    lam = int(round(2 * math.pi * R0 / kR))
    f = o.init_ligament(lam, 24, 24, R0, float(lam), 0.02, 0.0, rl, rv, 2.0)
    out = []
    for t in (200, 800):
        f = o.step(f, 1.0, -6.0, t - (200 if out else 0))
        _, sw, _ = o.diagnostics(f, rl, rv, slices=True)
        r = np.sqrt(sw / math.pi)              # local radius from the liquid area
        x = np.arange(lam)
        out.append(abs((r * np.exp(-2j * math.pi * x / lam)).sum()) * 2 / lam)
    return out


def test_rayleigh_cutoff():
    ks = [0.5, 0.7, 1.2, 1.4]
    with ProcessPoolExecutor(max_workers=min(4, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        amps = list(ex.map(_ligament_mode_amplitude, ks))
    for kR, (a200, a800) in zip(ks, amps):
        if kR < 1.0:
            assert a800 > 3.0 * a200, (kR, a200, a800)   # unstable: grows
        else:
            assert a800 < 0.1 * a200, (kR, a200, a800)   # stable: decays


# --------------------------------------------------------------------------
# P8: flat-interface densities against the mechanical-stability condition of
# the pseudo-potential EOS (Eq. 7): P(rho_l) = P(rho_v) and
# int_{rho_v}^{rho_l} (P(rho_l) - P(rho)) psi'(rho) / psi(rho)^2 drho = 0.
# The velocity-shift forcing (Eq. 6) adds a tau-dependent offset that
# vanishes at tau = 1, where the lattice must meet the condition.
# --------------------------------------------------------------------------

def _mechanical_stability(G):
    from scipy.integrate import quad
    from scipy.optimize import fsolve
    psi = lambda r: 1.0 - math.exp(-r)
    dpsi = lambda r: math.exp(-r)
    P = lambda r: r / 3.0 + G / 6.0 * psi(r) ** 2

    def eqs(v):
        rl, rv = v
        p0 = P(rl)
        with warnings.catch_warnings():
            # trial points of the root finder far from the solution may not
            # integrate to full accuracy; the converged point does
            warnings.simplefilter("ignore")
            integral = quad(lambda r: (p0 - P(r)) * dpsi(r) / psi(r) ** 2, rv, rl, limit=200)[0]
        return [P(rl) - P(rv), integral]
    return fsolve(eqs, [2.3, 0.1], xtol=1e-13)


@pytest.mark.parametrize("G", [-5.3, -6.0])
def test_flat_interface_meets_mechanical_stability_at_tau_one(G):
    rl_th, rv_th = _mechanical_stability(G)
    r = oracle.coexistence(1.0, G, n=64, tol=1e-10, rho_l0=2.4, rho_v0=0.1)
    assert abs(r["rho_l"] / rl_th - 1.0) < 1e-3, (r["rho_l"], rl_th)
    assert abs(r["rho_v"] / rv_th - 1.0) < 1e-2, (r["rho_v"], rv_th)


# --------------------------------------------------------------------------
# Droplet statistics (reading R16/R17) against networkx components and
# closed-form geometry
# --------------------------------------------------------------------------

def _nx_component_nodes(mask):
    import networkx as nx_
    nz, ny, nx = mask.shape
    g = nx_.Graph()
    idx = lambda z, y, x: x + nx * (y + ny * z)
    for z, y, x in zip(*np.nonzero(mask)):
        g.add_node(idx(z, y, x))
        for dz, dy, dx in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):
            q = ((z + dz) % nz, (y + dy) % ny, (x + dx) % nx)
            if mask[q]:
                g.add_edge(idx(z, y, x), idx(*q))
    return [sorted(cc) for cc in nx_.connected_components(g)]


@pytest.mark.parametrize("seed,shape,p", [(11, (6, 7, 9), 0.3), (12, (5, 5, 5), 0.4), (13, (4, 9, 6), 0.25)])
def test_droplets_vs_networkx(seed, shape, p):
    rl, rv = 2.65, 0.073
    nz, ny, nx = shape
    f = lbm_inputs.droplet_populations(nx, ny, nz, seed=seed, p=p, rho_l=rl, rho_v=rv)
    rho = f.sum(axis=0).ravel()
    comps = _nx_component_nodes(rho.reshape(shape) > 0.5 * (rl + rv))
    n, rec = oracle.droplets(f, rl, rv)
    assert n == len(comps) and rec.shape[0] == n
    want = sorted(((len(c), c[0]) for c in comps), key=lambda t: (-t[0], t[1]))
    assert [(int(r[1]), int(r[0])) for r in rec] == want
    by_first = {c[0]: np.array(c) for c in comps}
    for r in rec:
        nodes = by_first[int(r[0])]
        phi = np.clip((rho[nodes] - rv) / (rl - rv), 0.0, 1.0)
        assert r[2] == pytest.approx(phi.sum(), rel=1e-13)
        assert r[3] == pytest.approx(rho[nodes].sum(), rel=1e-13)
        assert int(r[10]) == len(set((nodes % nx).tolist()))


def test_droplet_centroid_on_periodic_box():
    # two balls of radius 2 (33 lattice points each: 1 + 6 + 12 + 8 + 6 at
    # squared distance 0..4), one centred on a corner of the periodic box so
    # that it is cut by the x and y boundaries; each centroid is its centre
    nx, ny, nz = 14, 11, 12
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def ball(c):
        d = [np.minimum(np.abs(a - ca), n - np.abs(a - ca)) for a, ca, n in
             ((xx, c[0], nx), (yy, c[1], ny), (zz, c[2], nz))]
        return d[0] ** 2 + d[1] ** 2 + d[2] ** 2 <= 4
    centres = [(0, ny - 1, 3), (7, 5, 8)]
    mask = ball(centres[0]) | ball(centres[1])
    # a ring along x through y = 5, z = 0: wraps, every x slice, no x centroid
    mask[0, 5, :] = True
    f = lbm_inputs.droplet_populations(nx, ny, nz, seed=5, mask=mask)
    n, rec = oracle.droplets(f, 2.65, 0.073)
    assert n == 3
    ring = rec[2]                        # largest first: the balls (33 nodes) lead
    assert int(ring[1]) == nx and int(ring[10]) == nx and ring[7] < 1e-12
    assert ring[5] == pytest.approx(5.0, abs=1e-12) and ring[6] == pytest.approx(0.0, abs=1e-12)
    assert rec[0][0] < rec[1][0]         # equal sizes: ordered by first node index
    got = sorted((tuple(r[4:7]), int(r[1]), int(r[10])) for r in rec[:2])
    for (c, nodes, xs), want in zip(got, sorted(centres)):
        assert nodes == 33 and xs == 5
        for d, n_ in enumerate((nx, ny, nz)):
            err = abs(c[d] - want[d])
            assert min(err, n_ - err) < 1e-9, (c, want)


def test_droplets_empty_and_full():
    f = lbm_inputs.droplet_populations(6, 5, 4, seed=3, mask=np.zeros((4, 5, 6), bool))
    assert oracle.droplets(f, 2.65, 0.073)[0] == 0
    f = lbm_inputs.droplet_populations(6, 5, 4, seed=3, mask=np.ones((4, 5, 6), bool))
    n, rec = oracle.droplets(f, 2.65, 0.073)
    assert n == 1 and int(rec[0][1]) == 120 and int(rec[0][0]) == 0 and int(rec[0][10]) == 6


# --------------------------------------------------------------------------
# MRT collision with Guo forcing (the operator the conclusions name as the
# next step: moments of d'Humieres et al. 2002, forcing of Guo et al. 2002)
# --------------------------------------------------------------------------

def test_mrt_matrix_orthogonal_with_the_published_norms():
    M = oracle.mrt_matrix()
    c, w, _ = oracle.lattice()
    D = M @ M.T
    assert np.array_equal(D, np.diag(np.diag(D)))
    assert np.diag(D).tolist() == [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24,
                                   4, 4, 4, 8, 8, 8]
    # conserved rows: density and the three momentum components
    assert (M[0] == 1).all()
    assert np.array_equal(M[[3, 5, 7]], c.T)
    # the equilibrium moments of energy and of its square are those of the
    # standard basis: m_eq(e) = rho (-11 + 19 u.u), m_eq(eps) = rho (3 - 11/2 u.u)
    u = np.array([0.03, -0.02, 0.05])
    meq = M @ oracle.feq(1.7, u)
    assert meq[1] == pytest.approx(1.7 * (-11 + 19 * u @ u), abs=1e-13)
    assert meq[2] == pytest.approx(1.7 * (3 - 5.5 * u @ u), abs=1e-13)


def _post_collision(g):
    """f*_a(x) from the state after one streaming step: g_a(x + c_a)."""
    c, _, _ = oracle.lattice()
    return np.stack([np.roll(g[a], shift=(-c[a][2], -c[a][1], -c[a][0]), axis=(0, 1, 2))
                     for a in range(19)])


@pytest.mark.parametrize("rates", ["srt", "mrt", "random"])
def test_guo_forcing_adds_the_force_to_the_momentum(rates):
    # any collision with Guo's forcing keeps rho and moves j to j + F at
    # every node, whatever the rates of the non-conserved moments
    f = lbm_inputs.random_populations(9, 7, 6, seed=81, rho_lo=0.3, rho_hi=2.2)
    G, tau = -5.3, 0.85
    if rates == "srt":
        g = oracle.step_forcing(f, G, 1, rates=None, tau=tau)
    else:
        r = oracle.mrt_rates(tau) if rates == "mrt" else 0.2 + 1.6 * lbm_inputs.uniform(5, 19)
        g = oracle.step_forcing(f, G, 1, rates=r)
    fs = _post_collision(g)
    c, _, _ = oracle.lattice()
    F = oracle.force(f, G)
    assert np.abs(fs.sum(0) - f.sum(0)).max() < 1e-14
    for k in range(3):
        dj = np.tensordot(c[:, k], fs - f, axes=1)
        assert np.abs(dj - F[k]).max() < 1e-14


def test_mrt_with_one_rate_is_srt_guo():
    f = lbm_inputs.random_populations(7, 6, 5, seed=71, rho_lo=0.3, rho_hi=2.2)
    tau = 0.9
    a = oracle.step_forcing(f, -5.3, 3, rates=np.full(19, 1.0 / tau))
    b = oracle.step_forcing(f, -5.3, 3, rates=None, tau=tau)
    assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("tau,others", [(0.8, (1.19, 1.4, 1.2, 1.4, 1.98)), (0.8, (1.6, 1.0, 1.0, 1.0, 1.0)),
                                        (1.3, (1.19, 1.4, 1.2, 1.4, 1.98))])
def test_mrt_shear_wave_decays_at_the_shear_rate(tau, others):
    # nu = (1/s_nu - 1/2)/3 with s_nu = 1/tau, whatever the other rates
    nx, k, A0 = 64, 2 * math.pi / 64, 1e-3
    x = np.arange(nx)
    f = np.zeros((19, 3, 3, nx))
    for i in range(nx):
        f[:, :, :, i] = oracle.feq(1.0, (0.0, A0 * math.sin(k * i), 0.0))[:, None, None]
    rates = oracle.mrt_rates(tau, *others)

    def amp(g):
        uy = oracle.moments(g, G=0.0, bare=True)[2][0, 0]
        return abs((uy * np.exp(-1j * k * x)).sum() * 2 / nx)
    g1 = oracle.step_forcing(f, 0.0, 200, rates=rates)
    g2 = oracle.step_forcing(g1, 0.0, 1000, rates=rates)
    rate = -math.log(amp(g2) / amp(g1)) / 1000
    assert abs(rate / ((tau - 0.5) / 3 * k * k) - 1.0) < 0.01


def test_mrt_flat_interface_is_independent_of_viscosity_and_meets_guo_stability():
    # with Guo forcing the flat interface satisfies the pseudo-potential
    # equal-area condition with weight psi'/psi (the tau = 1 velocity-shift
    # case of P8 has psi'/psi^2), so the densities do not change with the
    # shear rate: the density ratio stays fixed as the viscosity varies
    from scipy.integrate import quad
    from scipy.optimize import fsolve
    G = -5.3
    psi = lambda r: 1.0 - math.exp(-r)
    P = lambda r: r / 3.0 + G / 6.0 * psi(r) ** 2

    def eqs(v):
        rl, rv = v
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            I = quad(lambda r: (P(rl) - P(r)) * math.exp(-r) / psi(r), rv, rl, limit=200)[0]
        return [P(rl) - P(rv), I]
    rl_th, rv_th = fsolve(eqs, [2.1, 0.08], xtol=1e-13)
    got = [oracle.coexistence(1.0, G, n=64, tol=1e-10, rho_l0=2.2, rho_v0=0.15,
                              mrt_rates=oracle.mrt_rates(t), max_steps=200000) for t in (1.0, 1.5)]
    for r in got:
        assert abs(r["rho_l"] / rl_th - 1) < 1e-4 and abs(r["rho_v"] / rv_th - 1) < 1e-3
    assert abs(got[0]["rho_l"] - got[1]["rho_l"]) < 1e-8
    assert abs(got[0]["rho_v"] - got[1]["rho_v"]) < 1e-8
