"""GPU path (liblbm.so, through its C ABI) against the CPU FP64 oracle.

Tolerances (relative, per node, on rho and on the populations):
  FP64 storage: 1e-12 after 100 steps (rounding-order differences only);
  FP32 storage: 1e-5 after 100 steps;
  layout equivalences (AA vs A-B, graph vs eager, checkpoint resume): bitwise.
"""
import math

import numpy as np
import pytest

import lbm_inputs
import oracle

pytestmark = pytest.mark.gpu

G6 = -6.0


@pytest.fixture(scope="module")
def L():
    from paper_1904_11792_gb300 import build, lbm
    build.build()
    lbm.load()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lbm


@pytest.fixture(scope="module")
def coex():
    r = oracle.coexistence(1.0, G6, n=64, tol=1e-10, rho_l0=2.6, rho_v0=0.07)
    return r["rho_l"], r["rho_v"]


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def make(L, shape, tau, G, precision="f64", pattern="ab", **kw):
    nx, ny, nz = shape
    return L.Lattice(nx, ny, nz, tau, G, precision=precision, pattern=pattern, **kw)


# ---------------------------------------------------------------------------
# initial condition
# ---------------------------------------------------------------------------

# tanh and cos of the CUDA math library and of the host libm differ by an ulp or two
@pytest.mark.parametrize("precision,tol", [("f64", 1e-14), ("f32", 1.2e-7)])
def test_init_ligament_matches_oracle(L, coex, precision, tol):
    rl, rv = coex
    shape = (64, 32, 32)
    with make(L, shape, 1.0, G6, precision) as lat:
        lat.init_ligament(8.0, 64.0, 0.05, 0.3, rl, rv, 2.0)
        got = lat.populations()
    want = oracle.init_ligament(*shape, 8.0, 64.0, 0.05, 0.3, rl, rv, 2.0)
    assert rel(got, want) <= tol


def test_init_profile_matches_oracle(L):
    prof = np.linspace(2.6, 0.07, 17)
    shape = (24, 20, 20)
    with make(L, shape, 1.0, G6, "f64") as lat:
        lat.init_profile(5.0, 24.0, 0.1, 1.0, prof, -8.0, 1.0)
        got = lat.populations()
    want = oracle.init_profile(*shape, 5.0, 24.0, 0.1, 1.0, prof, -8.0, 1.0)
    assert rel(got, want) <= 1e-14


# ---------------------------------------------------------------------------
# time-step parity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(37, 11, 9), (3, 3, 3), (5, 3, 7), (130, 6, 5)])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_fp64_random_state_parity(L, shape, pattern):
    f0 = lbm_inputs.random_populations(*shape, seed=21)
    tau, G = 0.9, -5.5
    with make(L, shape, tau, G, "f64", pattern) as lat:
        lat.set_populations(f0)
        lat.step(100)
        got = lat.populations()
        rho = lat.rho()
    want = oracle.step(f0, tau, G, 100)
    assert rel(got, want) <= 1e-12
    assert rel(rho, want.sum(axis=0)) <= 1e-12


def test_fp64_ligament_parity_100_steps(L, coex):
    rl, rv = coex
    shape = (64, 32, 32)
    f0 = oracle.init_ligament(*shape, 8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
    want = oracle.step(f0, 1.0, G6, 100)
    with make(L, shape, 1.0, G6, "f64") as lat:
        lat.init_ligament(8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
        lat.step(100)
        got = lat.populations()
        rho = lat.rho()
    assert rel(rho, want.sum(axis=0)) <= 1e-12
    assert rel(got, want) <= 1e-12


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_fp32_ligament_parity_100_steps(L, coex, pattern):
    rl, rv = coex
    shape = (64, 32, 32)
    f0 = oracle.init_ligament(*shape, 8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
    want = oracle.step(f0, 1.0, G6, 100)
    with make(L, shape, 1.0, G6, "f32", pattern) as lat:
        lat.init_ligament(8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
        lat.step(100)
        rho = lat.rho()
    assert rel(rho, want.sum(axis=0)) <= 1e-5


def test_psi_rho_form_parity(L):
    shape = (12, 9, 7)
    f0 = lbm_inputs.random_populations(*shape, seed=5, rho_lo=0.5, rho_hi=1.5)
    with make(L, shape, 0.7, -0.8, "f64", psi_form=L.LBM_PSI_RHO) as lat:
        lat.set_populations(f0)
        lat.step(30)
        got = lat.populations()
    want = oracle.step(f0, 0.7, -0.8, 30, psi_form=1)
    assert rel(got, want) <= 1e-12


@pytest.mark.parametrize("block", [(32, 1, 1), (64, 2, 2), (128, 2, 1), (32, 4, 2), (256, 1, 1)])
def test_block_shapes_agree_bitwise(L, block):
    shape = (70, 13, 11)
    f0 = lbm_inputs.random_populations(*shape, seed=9)
    res = []
    for b in (None, block):
        with make(L, shape, 0.8, G6, "f32", block=b) as lat:
            lat.set_populations(f0)
            lat.step(7)
            res.append(lat.populations())
    np.testing.assert_array_equal(res[0], res[1])


# ---------------------------------------------------------------------------
# layout equivalences: AA == A-B, graph == eager, checkpoint resume
# ---------------------------------------------------------------------------

# Shapes: nx odd (one node per thread), nx % 4 == 0 with rows that start
# inside a warp (36: nine four-node groups per row; 132: 33, so a warp's
# lanes 0 and 31 sit inside rows), as the four-node gather psi pass before
# the AA odd step handles them.
@pytest.mark.parametrize("precision", ["f64", "f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("nsteps,shape", [(1, (33, 10, 9)), (2, (33, 10, 9)), (7, (33, 10, 9)), (20, (33, 10, 9)),
                                          (2, (36, 10, 9)), (7, (36, 10, 9)), (3, (132, 6, 5)),
                                          (8, (132, 6, 5))])
def test_aa_equals_ab_bitwise(L, precision, nsteps, shape):
    f0 = lbm_inputs.random_populations(*shape, seed=13)
    out = []
    for pattern in ("ab", "aa"):
        with make(L, shape, 0.85, G6, precision, pattern, rho_ref=0.1) as lat:
            lat.set_populations(f0)
            lat.step(nsteps)
            out.append((lat.populations(), lat.rho()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


# Graph replay and eager steps give the same bits, including the
# stochastic-rounding salt of the 2-byte forms (a pair of device words the
# collision kernels advance; the word a step reads follows the A-B array, or
# the step parity for AA) and graph chunks of odd length (diag_interval 3).
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("precision", ["f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("shape,k", [((40, 12, 8), 0), ((64, 8, 10), 0), ((64, 8, 10), 3)])
def test_graph_equals_eager_bitwise(L, pattern, precision, shape, k):
    f0 = lbm_inputs.random_populations(*shape, seed=17)
    out = []
    for graph in (1, 0):
        with make(L, shape, 0.9, G6, precision, pattern, rho_ref=0.1) as lat:
            lat.set_option("graph", graph)
            if k:
                lat.set_option("diag_interval", k)
            lat.set_populations(f0)
            lat.step(3)
            lat.step(10)
            lat.step(7)
            out.append(lat.populations())
    np.testing.assert_array_equal(out[0], out[1])


# A saved state resumes bitwise, the stochastic-rounding salt of the 2-byte
# forms restored from the step count (an odd one here), on the two-kernel
# (48 wide) and the fused (64 wide, A-B) step.
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("precision", ["f32", "f16dev"])
@pytest.mark.parametrize("nx", [48, 64])
def test_checkpoint_resume_bitwise(L, coex, pattern, precision, nx):
    rl, rv = coex
    shape = (nx, 24, 24)
    kw = dict(rho_ref=rv) if precision.endswith("dev") else {}
    with make(L, shape, 1.0, G6, precision, pattern, **kw) as lat:
        lat.init_ligament(6.0, float(nx), 0.05, 0.0, rl, rv, 2.0)
        lat.step(25)
        buf = lat.save_state()
        lat.step(30)
        full = lat.populations()
    with make(L, shape, 1.0, G6, precision, pattern, **kw) as lat:
        lat.load_state(buf)
        assert lat.step_count == 25
        lat.step(30)
        resumed = lat.populations()
    np.testing.assert_array_equal(full, resumed)


# ---------------------------------------------------------------------------
# moments and diagnostics
# ---------------------------------------------------------------------------

def test_moments_match_oracle(L, coex):
    rl, rv = coex
    shape = (32, 20, 20)
    f0 = oracle.init_ligament(*shape, 5.0, 32.0, 0.1, 0.0, rl, rv, 2.0)
    f1 = oracle.step(f0, 1.0, G6, 20)
    want = oracle.moments(f1, G6)
    with make(L, shape, 1.0, G6, "f64") as lat:
        lat.set_populations(f1)
        m = lat.moments()
    assert rel(m["rho"], want[0]) <= 1e-14
    for k, w in zip(("ux", "uy", "uz"), want[1:]):
        assert np.abs(m[k] - w).max() <= 1e-14 * max(1.0, np.abs(w).max())


# The global sums are FP64 from the first add on every storage precision:
# the mass is the FP64 sum of each node's exact density (its FP32 sum plus
# the rounding error of that sum), so it equals the oracle's FP64 sum of the
# same stored state to FP64 rounding plus the 2^-40 relative bound of the
# error term's own FP32 sum; the momentum is per node FP32 (exact zero where
# opposite populations are equal) summed in FP64, 1e-10 of the mass (measured
# 1e-13).  The liquid fraction phi = clamp((rho - rho_v)/(rho_l - rho_v)) is
# an FP32 value per node (exact 0 or 1 outside the interface): at each
# interface node its error is at most about 20 roundings of rho_l, relative
# to rho_l - rho_v, which bounds the FP64 sums of phi.
@pytest.mark.parametrize("precision", ["f64", "f32", "f16dev", "bf16dev"])
def test_diagnostics_and_droplets_match_oracle(L, coex, precision):
    rl, rv = coex
    shape = (40, 24, 24)
    # three blobs and a thin ligament piece: several components, wraps in x
    with make(L, shape, 1.0, G6, precision, rho_ref=rv if precision.endswith("dev") else 0.0) as lat:
        lat.init_ligament(4.5, 20.0, 0.6, 0.0, rl, rv, 2.0)
        lat.step(40)
        d = lat.diagnostics(ccl=True)
        rho = lat.rho()
        f = lat.populations()
    o = oracle.diagnostics(f, rl, rv)
    tol_m = 1e-12 if precision == "f64" else 1e-11
    tol_j = 1e-12 if precision == "f64" else 1e-10
    assert abs(d["mass"] - o["mass"]) <= tol_m * o["mass"], (d["mass"] / o["mass"] - 1)
    for k in range(3):
        dj = d["mom"][k] - (o["mom_x"], o["mom_y"], o["mom_z"])[k]
        assert abs(dj) <= tol_j * o["mass"], (k, dj / o["mass"])
    rho_o = f.sum(axis=0)
    n_if = int(((rho_o > rv) & (rho_o < rl)).sum())
    tol_phi = 1e-12 if precision == "f64" else 20 * 2.0 ** -24 * rho_o.max() / (rl - rv)
    assert abs(d["liquid_volume_w"] - o["liquid_volume_w"]) <= n_if * tol_phi + 1e-12 * o["liquid_volume_w"]
    assert abs(d["min_slice_area_w"] - o["min_slice_area_w"]) <= n_if * tol_phi + 1e-12
    # integer decisions on the GPU's own rho: compare with the oracle on the same field
    liq = rho > 0.5 * (rl + rv)
    assert d["liquid_count"] == int(liq.sum())
    assert d["min_slice_count"] == int(liq.sum(axis=(0, 1)).min())
    assert d["min_slice_x"] == int(np.argmin(liq.sum(axis=(0, 1))))
    n, labels, sizes = oracle.ccl(liq)
    assert d["droplets"] == n
    assert d["droplets_min8"] == int((sizes >= 8).sum())
    assert d["largest_droplet"] == (int(sizes.max()) if n else 0)
    assert d["numeric_ok"] == 1
    assert abs(d["max_u"] - o["max_u"]) <= 1e-6 * max(o["max_u"], 1e-12) + (1e-12 if precision == "f64" else 1e-6)


# The FP64 mass resolves the drift of a few FP32 steps: the fused FP32 step
# conserves mass up to the unbiased rounding of 19 stores per node (the rest
# population closes the balance, reading R22), so over 50 steps of the
# 64x32x32 ligament the relative drift is of order 1e-7 / sqrt(N) per step;
# the diagnostics must report the same drift as the oracle's FP64 sums of
# the two stored states, far below the old FP32-sum floor of ~1e-7.
def test_fp64_mass_resolves_fp32_drift(L, coex):
    rl, rv = coex
    shape = (64, 32, 32)
    with make(L, shape, 1.0, G6, "f32") as lat:
        lat.init_ligament(8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
        d0 = lat.diagnostics()
        f0 = lat.populations()
        lat.step(50)
        d1 = lat.diagnostics()
        f1 = lat.populations()
    m0, m1 = f0.sum(), f1.sum()
    assert abs(d0["mass"] / m0 - 1) <= 1e-12 and abs(d1["mass"] / m1 - 1) <= 1e-12
    drift_gpu = d1["mass"] / d0["mass"] - 1
    drift_orc = m1 / m0 - 1
    assert abs(drift_gpu - drift_orc) <= 2e-12, (drift_gpu, drift_orc)
    assert abs(drift_orc) < 1e-6


def test_droplet_count_random_masks(L):
    # densities built so that the liquid mask is a random pattern with many
    # components, including ones joined across the periodic boundaries
    shape = (17, 9, 11)
    nx, ny, nz = shape
    u = lbm_inputs.uniform(99, nx * ny * nz).reshape(nz, ny, nx)
    rho = np.where(u < 0.35, 2.0, 0.1)
    _, w = L.lbm_lattice()
    f = w[:, None, None, None] * rho[None]
    with make(L, shape, 1.0, G6, "f64") as lat:
        lat.set_populations(f)
        lat.set_option("rho_l", 2.0)
        lat.set_option("rho_v", 0.1)
        d = lat.diagnostics(ccl=True)
    n, _, sizes = oracle.ccl(rho > 1.05)
    assert d["droplets"] == n and d["largest_droplet"] == sizes.max()


# ---------------------------------------------------------------------------
# reduced-precision storage (deviation form): bounded error vs FP64
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision,tol", [("f16dev", 5e-3), ("bf16dev", 4e-2)])
def test_deviation_storage_error(L, coex, precision, tol):
    rl, rv = coex
    shape = (64, 32, 32)
    out = {}
    for p in ("f64", precision):
        with make(L, shape, 1.0, G6, p, rho_ref=rv) as lat:
            lat.init_ligament(8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
            lat.step(100)
            out[p] = (lat.rho(), lat.diagnostics())
    err = np.abs(out[precision][0] - out["f64"][0]) / out["f64"][0]
    assert err.max() <= tol
    drift = abs(out[precision][1]["mass"] - out["f64"][1]["mass"]) / out["f64"][1]["mass"]
    assert drift <= tol


# ---------------------------------------------------------------------------
# full-size grid-convergence box 256x128x128 (FP32, the benchmark's launch
# configuration): one step checked node by node on a sample
# ---------------------------------------------------------------------------

def test_full_size_sampled_one_step(L, coex):
    rl, rv = coex
    w = lbm_inputs.GRID_256
    shape = (w.nx, w.ny, w.nz)
    with make(L, shape, w.tau, w.G, "f32") as lat:
        lat.init_ligament(w.R0, w.lam, w.eps, w.phase, rl, rv, w.width)
        lat.step(50)
        f = lat.populations()
        lat.step(1)
        g = lat.populations()
        d = lat.diagnostics()
    N = w.nx * w.ny * w.nz
    u = lbm_inputs.uniform(4242, 400)
    nodes = np.unique((u * N).astype(np.int64))
    # nodes on the interface and on the periodic faces as well
    nodes = np.concatenate([nodes, [0, N - 1, w.nx - 1, w.nx * w.ny - 1,
                                    (w.ny // 2) * w.nx + (w.nz // 2) * w.nx * w.ny + 24]])
    want = oracle.step_nodes(f, nodes, w.tau, w.G)
    got = g.reshape(19, -1)[:, nodes].T
    assert rel(got, want) <= 1e-5
    # FP64 mass of the stepped state, and one step's drift
    assert abs(d["mass"] - g.sum()) <= 1e-11 * g.sum()
    assert abs(d["mass"] - f.sum()) <= 1e-8 * f.sum()


# The whole 256x128x128 field after 100 steps, node by node: the fused FP32
# step in the launch shape the benchmark gives this lattice (automatic run
# length and block order, in-loop diagnostics every 10 steps, each 10 steps
# one replay of the captured graph) against 100 oracle steps (FP64).
def test_grid256_fp32_full_field_100_steps(L, coex):
    rl, rv = coex
    w = lbm_inputs.GRID_256
    shape = (w.nx, w.ny, w.nz)
    f0 = oracle.init_ligament(*shape, w.R0, w.lam, w.eps, w.phase, rl, rv, w.width)
    want = oracle.step(f0, w.tau, w.G, 100).sum(axis=0)
    del f0
    with make(L, shape, w.tau, w.G, "f32") as lat:
        assert lat.get_option("fused") == 1
        lat.init_ligament(w.R0, w.lam, w.eps, w.phase, rl, rv, w.width)
        lat.set_option("diag_interval", 10)
        for _ in range(10):
            lat.step(10)
        lat.sync()
        assert lat.get_option("fused_fz_used") > 0
        rho = lat.rho()
        hist = lat.diag_history()
    assert len(hist) == 10 and all(h["numeric_ok"] == 1 for h in hist)
    assert rel(rho, want) <= 1e-5


def _patches(t, N, nx, ny, nodes, halo=2):
    """Populations of the (2 halo + 1)^3 periodic neighbourhood of each node,
    gathered on the device from a canonical FP32 array t[19 * N]: shape
    (k, 19, nz', ny', nx') float64 on the host."""
    import torch
    nz = N // (nx * ny)
    i = torch.as_tensor(nodes, dtype=torch.int64, device=t.device)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    d = torch.arange(-halo, halo + 1, device=t.device)
    zz = (z[:, None, None, None] + d[None, :, None, None]) % nz
    yy = (y[:, None, None, None] + d[None, None, :, None]) % ny
    xx = (x[:, None, None, None] + d[None, None, None, :]) % nx
    idx = (xx + nx * (yy + ny * zz)).reshape(len(nodes), -1)
    a = torch.arange(19, device=t.device, dtype=torch.int64)
    g = t[a[None, :, None] * N + idx[:, None, :]]
    w = 2 * halo + 1
    return g.double().cpu().numpy().reshape(len(nodes), 19, w, w, w)


# The 1024x512x512 ligament (268 M nodes), the benchmark's workload, in the
# launch shape the benchmark uses (the fused FP32 step, automatic run length
# and block order): one step checked node by node on sampled nodes.  The
# oracle steps the 5x5x5 periodic neighbourhood of each sampled node, which
# holds everything the node's next populations depend on (the 18 neighbours
# it pulls from and their psi neighbours), gathered on the device from the
# stored state, and its centre must equal the GPU's next populations.
def test_grid1024_sampled_one_step(L, coex):
    import torch
    rl, rv = coex
    w = lbm_inputs.GRID_1024
    N = w.nx * w.ny * w.nz
    with make(L, (w.nx, w.ny, w.nz), w.tau, w.G, "f32") as lat:
        assert lat.get_option("fused") == 1
        lat.init_ligament(w.R0, w.lam, w.eps, w.phase, rl, rv, w.width)
        lat.step(20)                      # even count: the current array is the first
        lat.sync()
        state = lat._buffers[0].view(torch.float32)
        u = lbm_inputs.uniform(4244, 300)
        c = (w.ny // 2) * w.nx + (w.nz // 2) * w.nx * w.ny
        nodes = np.unique(np.concatenate([
            (u * N).astype(np.int64),
            [0, N - 1, w.nx - 1, w.nx * w.ny - 1, c + 17],
            # nodes on the interface (r = R0 along y at several x)
            [x + w.nx * (w.ny // 2 + int(w.R0)) + w.nx * w.ny * (w.nz // 2) for x in (0, 255, 511, 1023)]]))
        before = _patches(state[:19 * N], N, w.nx, w.ny, nodes)
        lat.step(1)
        lat.sync()
        after = state[19 * N:2 * 19 * N]
        got = after[torch.arange(19, device="cuda")[:, None] * N
                    + torch.as_tensor(nodes, device="cuda")[None, :]].double().cpu().numpy().T
    want = np.stack([oracle.step(p, w.tau, w.G, 1)[:, 2, 2, 2] for p in before])
    assert rel(got, want) <= 1e-5


def _patches_gather(t, N, nx, ny, nodes, c, opp, halo=2):
    """As _patches, for a state in the AA gather layout (after an AA even
    step): population a of node p sits in slot opp(a) at p - c_a."""
    import torch
    nz = N // (nx * ny)
    i = torch.as_tensor(nodes, dtype=torch.int64, device=t.device)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    d = torch.arange(-halo, halo + 1, device=t.device)
    w = 2 * halo + 1
    out = []
    for a in range(19):
        zz = (z[:, None, None, None] + d[None, :, None, None] - int(c[a, 2])) % nz
        yy = (y[:, None, None, None] + d[None, None, :, None] - int(c[a, 1])) % ny
        xx = (x[:, None, None, None] + d[None, None, None, :] - int(c[a, 0])) % nx
        out.append(t[int(opp[a]) * N + (xx + nx * (yy + ny * zz)).reshape(len(nodes), -1)])
    return torch.stack(out, dim=1).double().cpu().numpy().reshape(len(nodes), 19, w, w, w)


# The in-place AA pair at the large configuration's size (1024x512x512, the
# FP16-deviation and FP32 AA steps the benchmark reports, default launch
# shapes): the even step (in place, slots swapped) and the odd step (gather
# and scatter, after the four-node gather psi pass for 2-byte storage) each
# checked on sampled nodes against the oracle stepping the node's 5x5x5
# neighbourhood of the decoded state.  After the even step the post-collision
# population a of node x sits in slot opp(a) at x, so the oracle's streamed
# population a of node y is the GPU's slot opp(a) at y - c_a; the odd step's
# input is gathered from that layout and its output is in the natural one.
# Tolerances as the one-step cases: 1e-5 relative for FP32, one storage ulp
# of the stored deviation plus the FP32 arithmetic for FP16.
@pytest.mark.parametrize("precision,eps", [("f32", None), ("f16dev", 2.0 ** -10)])
def test_grid1024_aa_sampled_even_and_odd_steps(L, coex, precision, eps):
    import torch
    rl, rv = coex
    w = lbm_inputs.GRID_1024
    N = w.nx * w.ny * w.nz
    c, wts, opp = oracle.lattice()
    dev = precision.endswith("dev")
    if dev:
        shift = (wts * rv).astype(np.float32).astype(np.float16).astype(np.float64)
        tdt = torch.float16
    else:
        shift = np.zeros(19)
        tdt = torch.float32

    def check(got, want):
        if dev:
            tol = 1.01 * (eps * np.abs(want - shift[None, :]) + 2.0 ** -24) + 4e-7 * np.abs(want)
            err = np.abs(got - want)
            assert (err <= tol).all(), float((err / tol).max())
        else:
            assert rel(got, want) <= 1e-5

    with make(L, (w.nx, w.ny, w.nz), w.tau, w.G, precision, "aa", **(dict(rho_ref=rv) if dev else {})) as lat:
        lat.init_ligament(w.R0, w.lam, w.eps, w.phase, rl, rv, w.width)
        lat.step(20)                      # even count: the natural layout
        lat.sync()
        state = lat._buffers[0].view(tdt)[:19 * N]
        u = lbm_inputs.uniform(4246, 200)
        cz = (w.ny // 2) * w.nx + (w.nz // 2) * w.nx * w.ny
        nodes = np.unique(np.concatenate([
            (u * N).astype(np.int64), [0, N - 1, w.nx - 1, w.nx * w.ny - 1, cz + 17],
            [x + w.nx * (w.ny // 2 + int(w.R0)) + w.nx * w.ny * (w.nz // 2) for x in (0, 3, 511, 1020, 1023)]]))
        ti = torch.as_tensor(nodes, device="cuda")
        xs, ys, zs = ti % w.nx, (ti // w.nx) % w.ny, ti // (w.nx * w.ny)
        # even step
        before = _patches(state, N, w.nx, w.ny, nodes) + shift[None, :, None, None, None]
        lat.step(1)
        lat.sync()
        idx = torch.stack([int(opp[a]) * N + ((xs - int(c[a, 0])) % w.nx + w.nx * (((ys - int(c[a, 1])) % w.ny)
                           + w.ny * ((zs - int(c[a, 2])) % w.nz))) for a in range(19)], dim=1)
        got = state[idx].double().cpu().numpy() + shift[None, :]
        check(got, np.stack([oracle.step(p, w.tau, w.G, 1)[:, 2, 2, 2] for p in before]))
        # odd step
        before = _patches_gather(state, N, w.nx, w.ny, nodes, c, opp) + shift[None, :, None, None, None]
        lat.step(1)
        lat.sync()
        got = state[torch.arange(19, device="cuda")[None, :] * N + ti[:, None]].double().cpu().numpy() + shift[None, :]
        check(got, np.stack([oracle.step(p, w.tau, w.G, 1)[:, 2, 2, 2] for p in before]))


# The benchmark's FP16 / BF16 variants at their full size (1024x512x512,
# fused step, its launch shape): one step on sampled nodes against the
# oracle stepping each node's 5x5x5 neighbourhood of the decoded stored state
# (deviation + the shift w_a rho_ref rounded to the storage format), within
# one storage ulp of the stored deviation plus the FP32 arithmetic, as the
# 256x128x128 case below.
@pytest.mark.parametrize("precision,eps", [("f16dev", 2.0 ** -10), ("bf16dev", 2.0 ** -7)])
def test_grid1024_sampled_one_step_deviation_storage(L, coex, precision, eps):
    import torch
    rl, rv = coex
    w = lbm_inputs.GRID_1024
    N = w.nx * w.ny * w.nz
    wts = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    if precision == "f16dev":
        shift = (wts * rv).astype(np.float32).astype(np.float16).astype(np.float64)
        tdt = torch.float16
    else:   # BF16: the top 16 bits of the FP32 value, rounded to nearest even
        b = (wts * rv).astype(np.float32).view(np.uint32).astype(np.uint64)
        b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
        shift = b.astype(np.uint32).view(np.float32).astype(np.float64)
        tdt = torch.bfloat16
    with make(L, (w.nx, w.ny, w.nz), w.tau, w.G, precision, rho_ref=rv) as lat:
        assert lat.get_option("fused") == 1 and lat.get_option("stochastic_rounding") == 1
        lat.init_ligament(w.R0, w.lam, w.eps, w.phase, rl, rv, w.width)
        lat.step(20)
        lat.sync()
        state = lat._buffers[0].view(tdt)
        u = lbm_inputs.uniform(4245, 300)
        c = (w.ny // 2) * w.nx + (w.nz // 2) * w.nx * w.ny
        nodes = np.unique(np.concatenate([
            (u * N).astype(np.int64), [0, N - 1, w.nx - 1, w.nx * w.ny - 1, c + 17],
            [x + w.nx * (w.ny // 2 + int(w.R0)) + w.nx * w.ny * (w.nz // 2) for x in (0, 255, 511, 1023)]]))
        before = _patches(state[:19 * N], N, w.nx, w.ny, nodes) + shift[None, :, None, None, None]
        lat.step(1)
        lat.sync()
        after = state[19 * N:2 * 19 * N]
        got = after[torch.arange(19, device="cuda")[:, None] * N
                    + torch.as_tensor(nodes, device="cuda")[None, :]].double().cpu().numpy().T + shift[None, :]
    want = np.stack([oracle.step(p, w.tau, w.G, 1)[:, 2, 2, 2] for p in before])
    dev = np.abs(want - shift[None, :])
    tol = 1.01 * (eps * dev + 2.0 ** -24) + 4e-7 * np.abs(want)
    err = np.abs(got - want)
    assert (err <= tol).all(), float((err / tol).max())


# The same full-size sampled step with FP16 / BF16 deviation storage (the
# fused step with stochastic rounding, as the benchmark runs it): the oracle
# steps the decoded stored state; the GPU result, computed in FP32, is stored
# as a deviation from the shift w_a rho_ref rounded to the storage format, so
# it may differ from the oracle by under one storage ulp of that deviation
# (2^-10 or 2^-7 of it, 2^-24 absolute for FP16 subnormals) plus the FP32
# arithmetic (a few 1e-7 of f).
@pytest.mark.parametrize("precision,eps", [("f16dev", 2.0 ** -10), ("bf16dev", 2.0 ** -7)])
def test_full_size_sampled_one_step_deviation_storage(L, coex, precision, eps):
    rl, rv = coex
    w = lbm_inputs.GRID_256
    shape = (w.nx, w.ny, w.nz)
    with make(L, shape, w.tau, w.G, precision, rho_ref=rv) as lat:
        assert lat.get_option("fused") == 1 and lat.get_option("stochastic_rounding") == 1
        lat.init_ligament(w.R0, w.lam, w.eps, w.phase, rl, rv, w.width)
        lat.step(50)
        f = lat.populations()
        lat.step(1)
        g = lat.populations()
    N = w.nx * w.ny * w.nz
    u = lbm_inputs.uniform(4243, 400)
    nodes = np.unique(np.concatenate([(u * N).astype(np.int64),
                                      [0, N - 1, w.nx - 1, (w.ny // 2) * w.nx + (w.nz // 2) * w.nx * w.ny + 24]]))
    want = oracle.step_nodes(f, nodes, w.tau, w.G)
    got = g.reshape(19, -1)[:, nodes].T
    wts = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    cast = np.float16 if precision == "f16dev" else None
    shift = wts * rv
    if cast is not None:
        shift = shift.astype(np.float32).astype(cast).astype(np.float64)
    else:   # BF16: keep the top 16 bits of the FP32 value, rounded to nearest even
        b = shift.astype(np.float32).view(np.uint32).astype(np.uint64)
        b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
        shift = b.astype(np.uint32).view(np.float32).astype(np.float64)
    dev = np.abs(want - shift[None, :])
    tol = 1.01 * (eps * dev + 2.0 ** -24) + 4e-7 * np.abs(want)
    err = np.abs(got - want)
    assert (err <= tol).all(), float((err / tol).max())


# The 1024x512x512 ligament (268 M nodes, 40.8 GB of FP32 populations) in the
# launch shape its benchmark uses: too large to step node by node on the
# host, so checked by what holds at any size: the fused step keeps the mass
# (FP32 storage: to rounding) and the total momentum of the periodic box (the
# pair forces of Eq. 5 cancel), and every density stays finite.
def test_grid1024_fused_conserves_mass_and_momentum(L, coex):
    rl, rv = coex
    w = lbm_inputs.GRID_1024
    with make(L, (w.nx, w.ny, w.nz), w.tau, w.G, "f32") as lat:
        assert lat.get_option("fused") == 1
        lat.init_ligament(w.R0, w.lam, w.eps, w.phase, rl, rv, w.width)
        d0 = lat.diagnostics()
        lat.step(20)
        lat.sync()
        d1 = lat.diagnostics()
    assert d0["numeric_ok"] == 1 and d1["numeric_ok"] == 1
    # FP32 storage: the density sum and the stored values round to nearest,
    # and in the uniform liquid and vapour every node rounds the same way, so
    # the mass moves by a coherent rounding each step (measured 1.1e-7 over
    # these 20 steps, resolved by the FP64 sums); momentum is exactly zero in
    # uniform regions and moves only by interface roundings
    assert abs(d1["mass"] / d0["mass"] - 1) < 1e-6
    for k in range(3):
        assert abs(d1["mom"][k] - d0["mom"][k]) < 1e-7 * d0["mass"]
    assert d1["liquid_count"] > 0 and d1["rho_max"] < 1.2 * rl


# ---------------------------------------------------------------------------
# failure handling without faulting the GPU
# ---------------------------------------------------------------------------

def test_numeric_flag_on_negative_density(L):
    shape = (8, 6, 5)
    f = lbm_inputs.random_populations(*shape, seed=2)
    f[:, 2, 3, 4] = -0.01
    with make(L, shape, 1.0, G6, "f32") as lat:
        lat.set_populations(f)
        assert lat.diagnostics()["numeric_ok"] == 0
        lat.step(1)
        with pytest.raises(L.LbmError) as ei:
            lat.sync()
        assert ei.value.status == L.LBM_ERR_NUMERIC
        lat.sync()  # the flag is cleared once reported


def test_alloc_cap_gives_oom(L, monkeypatch):
    monkeypatch.setenv("LBM_ALLOC_CAP_BYTES", "1024")
    with pytest.raises(L.LbmError) as ei:
        L.lbm_create(64, 64, 64, 1.0, G6)
    assert "LBM_ALLOC_CAP_BYTES" in str(ei.value)
    monkeypatch.delenv("LBM_ALLOC_CAP_BYTES")
    h = L.lbm_create(8, 8, 8, 1.0, G6)
    L.lbm_destroy(h)


def test_step_before_init_is_a_state_error(L):
    h = L.lbm_create(8, 8, 8, 1.0, G6)
    try:
        with pytest.raises(L.LbmError) as ei:
            L.lbm_step(h, 1)
        assert ei.value.status == L.LBM_ERR_STATE
    finally:
        L.lbm_destroy(h)


def test_kernel_timing_counts_launches(L):
    with make(L, (64, 16, 16), 1.0, G6, "f32") as lat:
        lat.set_populations(lbm_inputs.random_populations(64, 16, 16, seed=1))
        lat.set_option("fused", 0)
        lat.set_option("kernel_timing", 1)
        lat.step(6)
        n0, ms0 = L.lbm_kernel_time(lat.h, 0)
        n1, ms1 = L.lbm_kernel_time(lat.h, 1)
        assert n0 == 6 and n1 == 6 and ms0 > 0 and ms1 > 0
        # the single-pass step (the default where it applies) is class 2,
        # its diagnostic steps included
        lat.set_option("fused", 1)
        lat.set_option("diag_interval", 4)
        lat.set_option("kernel_timing", 0)
        lat.set_option("kernel_timing", 1)
        lat.step(6)   # steps 6..11: 8 is a diagnostic step
        n = [L.lbm_kernel_time(lat.h, k)[0] for k in range(3)]
    assert n == [0, 0, 6]


def test_gpu_coexistence_matches_oracle(L):
    from paper_1904_11792_gb300.coexistence import coexistence
    got = coexistence(G6, 1.0, n=64, tol=1e-10)
    want = oracle.coexistence(1.0, G6, n=64, tol=1e-10, rho_l0=2.6, rho_v0=0.07)
    assert abs(got["rho_l"] - want["rho_l"]) <= 1e-8
    assert abs(got["rho_v"] - want["rho_v"]) <= 1e-8


# ---------------------------------------------------------------------------
# diagnostics inside the time loop (option diag_interval)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pattern,k", [("ab", 5), ("aa", 5), ("aa", 3), ("ab", 3)])
def test_diag_history_matches_on_demand(L, coex, pattern, k):
    rl, rv = coex
    shape = (40, 20, 20)
    steps = 4 * k + 2
    with make(L, shape, 1.0, G6, "f32", pattern) as lat:
        lat.init_ligament(5.0, 40.0, 0.1, 0.0, rl, rv, 2.0)
        lat.set_option("diag_interval", k)
        lat.step(1)
        lat.step(steps - 1)
        hist = lat.diag_history()
    want = []
    with make(L, shape, 1.0, G6, "f32", pattern) as lat:
        lat.init_ligament(5.0, 40.0, 0.1, 0.0, rl, rv, 2.0)
        for t in range(steps):
            if t % k == 0:
                want.append(lat.diagnostics())
            lat.step(1)
    assert [h["step"] for h in hist] == list(range(0, steps, k))
    for h, w in zip(hist, want):
        for key in ("mass", "liquid_volume_w", "liquid_count", "min_slice_area_w",
                    "min_slice_count", "min_slice_x", "max_u", "rho_min", "rho_max", "numeric_ok"):
            assert h[key] == w[key], (key, h[key], w[key])
        assert h["mom"] == w["mom"]


# Fused diagnostic steps reduce the same per-node values in another grouping:
# counts and extrema are exact, sums (FP64 from the first add) agree to FP64
# rounding.
@pytest.mark.parametrize("precision", ["f32", "f16dev"])
@pytest.mark.parametrize("shape,k", [((64, 16, 12), 4), ((128, 8, 17), 3)])
def test_fused_diag_history_matches_on_demand(L, coex, precision, shape, k):
    rl, rv = coex
    nx, ny, nz = shape
    steps = 4 * k + 2
    R0 = min(ny, nz) / 4.0

    def make_lat():
        lat = make(L, shape, 1.0, G6, precision, "ab", rho_ref=rv if precision.endswith("dev") else 0.0)
        lat.init_ligament(R0, float(nx), 0.1, 0.0, rl, rv, 2.0)
        return lat

    with make_lat() as lat:
        assert lat.get_option("fused") == 1
        lat.set_option("diag_interval", k)
        lat.step(steps)
        hist = lat.diag_history()
        got_state = lat.populations()
    want = []
    with make_lat() as lat:
        for t in range(steps):
            if t % k == 0:
                want.append(lat.diagnostics())
            lat.step(1)
        want_state = lat.populations()
    np.testing.assert_array_equal(got_state, want_state)
    assert [h["step"] for h in hist] == list(range(0, steps, k))
    for h, w in zip(hist, want):
        for key in ("liquid_count", "min_slice_count", "min_slice_x", "max_u", "rho_min", "rho_max",
                    "numeric_ok"):
            assert h[key] == w[key], (key, h[key], w[key])
        for key in ("mass", "liquid_volume_w", "min_slice_area_w"):
            assert h[key] == pytest.approx(w[key], rel=1e-12), key
        for c in range(3):
            assert abs(h["mom"][c] - w["mom"][c]) <= 1e-12 * w["mass"]


def test_diag_interval_does_not_change_the_state(L):
    shape = (30, 12, 10)
    f0 = lbm_inputs.random_populations(*shape, seed=31)
    out = []
    for k in (0, 4):
        with make(L, shape, 0.9, G6, "f32") as lat:
            lat.set_populations(f0)
            lat.set_option("diag_interval", k)
            lat.step(17)
            out.append(lat.populations())
    np.testing.assert_array_equal(out[0], out[1])


# ---------------------------------------------------------------------------
# two-node (vector) kernels equal the one-node kernels bitwise
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["f64", "f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("shape", [(34, 10, 7), (36, 10, 7)])
def test_vector_kernels_equal_scalar_bitwise(L, precision, pattern, shape):
    # even nx: two-node kernels; nx % 4 == 0: also the four-node psi pass
    f0 = lbm_inputs.random_populations(*shape, seed=41)
    out = []
    for vec in (1, 0):
        with make(L, shape, 0.9, G6, precision, pattern, rho_ref=0.1) as lat:
            lat.set_option("vector", vec)
            assert lat.get_option("vector") == vec
            lat.set_populations(f0)
            lat.step(7)
            out.append((lat.populations(), lat.rho()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("shape", [(36, 11, 9), (4, 3, 5), (64, 32, 32)])
def test_fp64_vector_path_parity(L, shape):
    f0 = lbm_inputs.random_populations(*shape, seed=23)
    with make(L, shape, 0.95, -5.0, "f64", "aa") as lat:
        assert lat.get_option("vector") == 1
        lat.set_populations(f0)
        lat.step(41)
        got = lat.populations()
    want = oracle.step(f0, 0.95, -5.0, 41)
    assert np.isfinite(want).all()
    assert rel(got, want) <= 1e-12


# ---------------------------------------------------------------------------
# fused single-pass step equals the two-kernel step bitwise
# ---------------------------------------------------------------------------

# shapes: several z runs per tile column; a run of one plane (nz = 17); one
# tile row and the shortest periodic z (64 x 4 x 3; 2-byte storage, whose
# tiles have 8 rows: 64 x 8 x 3); three tile rows (4-byte: 192 x 12 x 17,
# 2-byte: 192 x 24 x 17)
@pytest.mark.parametrize("precision", ["f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("shape", [(64, 16, 12), (128, 8, 5), (192, 12, 17), (64, 4, 3)])
def test_fused_equals_two_pass_bitwise(L, precision, shape):
    if precision != "f32" and shape[1] % 8:
        shape = (shape[0], 2 * shape[1], shape[2])
    f0 = lbm_inputs.random_populations(*shape, seed=51)
    out = []
    for fused in (1, 0):
        with make(L, shape, 0.9, -5.5, precision, "ab", rho_ref=0.1) as lat:
            lat.set_option("fused", fused)
            assert lat.get_option("fused") == fused
            lat.set_populations(f0)
            lat.step(1)
            lat.step(6)
            out.append((lat.populations(), lat.rho()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("shape", [(64, 16, 12), (64, 8, 8)])
def test_fused_not_applicable_runs_two_pass(L, shape):
    # FP64 storage, nx not a multiple of 64, and ny not a multiple of the
    # tile rows (4 for 4-byte, 8 for 2-byte storage) take the two-kernel step
    nx, ny, nz = shape
    for precision, sh in (("f64", shape), ("f32", (nx + 32, ny, nz)), ("f32", (nx, ny + 2, nz)),
                          ("f16dev", (nx, ny + 4, nz))):
        with make(L, sh, 0.9, -5.5, precision, "ab") as lat:
            lat.set_option("fused", 1)
            assert lat.get_option("fused") == 0
            lat.set_populations(lbm_inputs.random_populations(*sh, seed=3))
            lat.step(3)
            lat.sync()


def test_fused_with_in_loop_diagnostics_and_oracle(L, coex):
    rl, rv = coex
    shape = (64, 32, 32)
    f0 = oracle.init_ligament(*shape, 8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
    want = oracle.step(f0, 1.0, G6, 100)
    with make(L, shape, 1.0, G6, "f32") as lat:
        lat.set_option("fused", 1)
        lat.set_option("diag_interval", 7)
        lat.init_ligament(8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
        lat.step(100)
        got = lat.populations()
        hist = lat.diag_history()
    assert rel(got, want) <= 1e-5
    assert [h["step"] for h in hist] == list(range(0, 100, 7))


def test_fused_numeric_flag(L):
    shape = (64, 8, 8)
    f = lbm_inputs.random_populations(*shape, seed=2)
    f[:, 3, 4, 5] = -0.01
    with make(L, shape, 1.0, G6, "f32") as lat:
        lat.set_option("fused", 1)
        lat.set_populations(f)
        lat.step(1)
        with pytest.raises(L.LbmError) as ei:
            lat.sync()
        assert ei.value.status == L.LBM_ERR_NUMERIC


# ---------------------------------------------------------------------------
# stochastic rounding of the deviation storage: deterministic, and far less
# mass drift than round-to-nearest through a break-up (the 64x32x32 ligament
# pinches off near step 1400)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["f16dev", "bf16dev"])
def test_stochastic_rounding_mass_drift(L, coex, precision):
    rl, rv = coex
    shape = (64, 32, 32)
    drift = {}
    for sr in (0, 1):
        runs = []
        for _ in range(2 if sr else 1):
            with make(L, shape, 1.0, G6, precision, rho_ref=rv) as lat:
                lat.set_option("stochastic_rounding", sr)
                lat.init_ligament(8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
                m0 = lat.diagnostics()["mass"]
                lat.step(1600)
                m1 = lat.diagnostics()["mass"]
                runs.append((m1, lat.rho()))
        if sr:
            np.testing.assert_array_equal(runs[0][1], runs[1][1])   # deterministic
        drift[sr] = abs(runs[0][0] - m0) / m0
    assert drift[1] < drift[0] / 3.0, drift
    assert drift[1] < (2e-3 if precision == "f16dev" else 1e-2), drift


# A uniform liquid at rest stays put: with the deviation shift on the storage
# grid the shift arithmetic is exact, and stochastic rounding with a per-step
# salt leaves only an unbiased random walk of the mass (a 24-bit shift lost
# 3.4e-4 of the mass in these 2000 FP16 steps).
@pytest.mark.parametrize("precision,tol", [("f16dev", 1e-5), ("bf16dev", 3e-4)])
def test_uniform_liquid_keeps_its_mass(L, coex, precision, tol):
    rl, rv = coex
    shape = (64, 32, 32)
    _, w = L.lbm_lattice()
    f = np.broadcast_to((w * rl)[:, None, None, None], (19,) + shape[::-1]).copy()
    with make(L, shape, 1.0, G6, precision, rho_ref=rv) as lat:
        lat.set_populations(f)
        m0 = lat.diagnostics()["mass"]
        lat.step(2000)
        m1 = lat.diagnostics()["mass"]
    assert abs(m1 / m0 - 1.0) < tol


# Failure detection without a GPU fault: the fused step's waits on its plane
# copies are bounded in time.  The test hook makes every block also wait
# (1 ms) on a barrier nothing completes; the step is reported void through
# LBM_ERR_TIMEOUT, and the context keeps working.
def test_fused_wait_timeout_is_reported_and_recoverable(L):
    shape = (64, 16, 12)
    f0 = lbm_inputs.random_populations(*shape, seed=7)
    with make(L, shape, 0.9, -5.5, "f32") as lat:
        assert lat.get_option("fused") == 1
        lat.set_populations(f0)
        lat.set_option("fused_stall_test", 1.0)
        lat.step(1)
        with pytest.raises(L.LbmError) as ei:
            lat.sync()
        assert ei.value.status == L.LBM_ERR_TIMEOUT
        lat.set_option("fused_stall_test", 0)
        lat.set_populations(f0)
        lat.step(3)
        lat.sync()
        got = lat.populations()
    with make(L, shape, 0.9, -5.5, "f32") as lat:
        lat.set_populations(f0)
        lat.step(3)
        want = lat.populations()
    np.testing.assert_array_equal(got, want)


# The fused step's block order (z runs launched in groups) does not change
# any result: every group size gives the two-kernel step's bits, and the
# diagnostics it reduces in the same pass agree exactly.
@pytest.mark.parametrize("precision", ["f32", "f16dev"])
def test_fused_group_order_is_bitwise_neutral(L, precision):
    # 3 x 3 tiles (64 x 4, or 64 x 8 for 2-byte storage); 5-plane runs: 4 runs
    shape = (192, 12, 20) if precision == "f32" else (192, 24, 20)
    f0 = lbm_inputs.random_populations(*shape, seed=61)
    out = {}
    for fused, grp in ((0, 0), (1, 0), (1, 1), (1, 3), (1, 4), (1, 64)):
        with make(L, shape, 0.9, -5.5, precision, "ab", rho_ref=0.1) as lat:
            lat.set_option("fused", fused)
            assert lat.get_option("fused") == fused
            lat.set_option("fused_fz", 5)
            lat.set_option("fused_group", grp)
            assert lat.get_option("fused_group") == grp
            lat.set_option("diag_interval", 2)
            lat.set_populations(f0)
            lat.step(5)
            hist = lat.diag_history()
            out[(fused, grp)] = (lat.populations(), [h["liquid_count"] for h in hist],
                                 [h["rho_max"] for h in hist], [h["min_slice_count"] for h in hist])
    ref_f = out[(0, 0)][0]
    ref_diag = out[(1, 0)][1:]
    for key, (f, *diag) in out.items():
        np.testing.assert_array_equal(f, ref_f, err_msg=str(key))
        if key[0] == 1:
            assert tuple(diag) == ref_diag, key


def test_fused_launch_shape_is_reported(L):
    # the run length and runs per group the fused step launches with
    with make(L, (128, 8, 40), 0.9, -5.5, "f32") as lat:
        lat.set_option("fused_fz", 8)
        lat.set_option("fused_group", 2)
        assert (lat.get_option("fused_fz_used"), lat.get_option("fused_group_used")) == (8, 2)
        lat.set_option("fused_group", 100)          # at most the 5 runs there are
        assert lat.get_option("fused_group_used") == 5
        lat.set_option("fused_fz", 0)
        lat.set_option("fused_group", 0)
        fz, grp = lat.get_option("fused_fz_used"), lat.get_option("fused_group_used")
        assert 4 <= fz <= 40 and 1 <= grp <= -(-40 // fz)
    with make(L, (64, 8, 8), 0.9, -5.5, "f64") as lat:    # no fused step in FP64
        assert (lat.get_option("fused_fz_used"), lat.get_option("fused_group_used")) == (0, 0)
