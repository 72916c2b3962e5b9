"""Batched form (many uneven ligaments advanced together: by default one
single-pass launch per step for the whole batch, or the two-kernel step with
option fused = 0) against standalone lattices and the oracle: bitwise per
instance."""
import numpy as np
import pytest

import lbm_inputs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1904_11792_gb300 import build, lbm
    build.build()
    lbm.load()
    return lbm


RL, RV = 2.648878066946715, 0.0731992478525716   # G = -6, tau = 1 flat-interface run


def instances(n=5):
    out = []
    for k, inst in enumerate(lbm_inputs.batched_sweep(48)[:n]):
        # shrink to test size: R0 -> R0/4, same aspect (lambda x 4R0 x 4R0)
        R0 = inst.R0 / 4
        lam = max(3, int(round(inst.lam / 4)))
        # tau >= 0.8: the sharp tanh start is unstable below (reading R15)
        tau = 0.8 + 0.5 * (inst.tau - 0.6)
        out.append(dict(nx=lam, ny=int(4 * R0), nz=int(4 * R0), tau=tau, G=-6.0, R0=R0,
                        lam=float(lam), eps=0.05, phase=inst.phase, rho_l=RL, rho_v=RV, width=2.0))
    return out


def standalone(L, d, steps, precision="f32"):
    with L.Lattice(d["nx"], d["ny"], d["nz"], d["tau"], d["G"], precision=precision,
                   rho_ref=d["rho_v"] if precision.endswith("dev") else 0.0) as lat:
        lat.init_ligament(d["R0"], d["lam"], d["eps"], d["phase"], d["rho_l"], d["rho_v"], d["width"])
        lat.step(steps)
        return lat.populations(), lat.diagnostics()


@pytest.mark.parametrize("precision", ["f32", "f16dev"])
def test_batched_equals_standalone_bitwise(L, precision):
    insts = instances(5)
    with L.Batch(insts, precision=precision) as b:
        b.init()
        b.step(1)
        b.step(12)
        got = [b.populations(k) for k in range(len(insts))]
        dg = [b.diagnostics(k) for k in range(len(insts))]
    for k, d in enumerate(insts):
        want, dw = standalone(L, d, 13, precision)
        np.testing.assert_array_equal(got[k], want)
        assert dg[k]["mass"] == dw["mass"] and dg[k]["liquid_count"] == dw["liquid_count"]


def test_sequential_equals_batched_and_block_shapes(L):
    insts = instances(6)
    res = []
    # the batched kernel runs block_x * block_y * block_z threads over
    # consecutive nodes: 256, 128 and a block size that is no power of two
    for mode, block in (("batched", None), ("sequential", None), ("batched", (64, 2, 2)),
                        ("batched", (32, 4, 1)), ("batched", (96, 1, 1))):
        with L.Batch(insts) as b:
            if block:
                b.set_option("fused", 0)          # block shapes of the two-kernel step
                for key, v in zip(("block_x", "block_y", "block_z"), (1, 1, 1)):
                    b.set_option(key, v)
                for key, v in zip(("block_x", "block_y", "block_z"), block):
                    b.set_option(key, v)
            b.init()
            (b.step if mode == "batched" else b.step_sequential)(9)
            res.append([b.populations(k) for k in range(len(insts))])
    for r in res[1:]:
        for a, c in zip(res[0], r):
            np.testing.assert_array_equal(a, c)


def test_batched_instance_matches_oracle(L):
    insts = instances(3)
    with L.Batch(insts, precision="f64") as b:
        b.init()
        b.step(20)
        got = [b.populations(k) for k in range(len(insts))]
    for k, d in enumerate(insts):
        f0 = oracle.init_ligament(d["nx"], d["ny"], d["nz"], d["R0"], d["lam"], d["eps"],
                                  d["phase"], d["rho_l"], d["rho_v"], d["width"])
        want = oracle.step(f0, d["tau"], d["G"], 20)
        assert float(np.max(np.abs(got[k] - want) / want)) <= 1e-12


def test_full_sweep_builds_and_runs(L):
    # the 48-instance sweep at full size: creation, init, a few steps, mass
    # conserved (tau lifted to >= 0.8 for the tanh start, reading R15)
    insts = [dict(nx=i.nx, ny=i.ny, nz=i.nz, tau=max(i.tau, 0.8), G=i.G, R0=i.R0, lam=i.lam, eps=i.eps,
                  phase=i.phase, rho_l=RL, rho_v=RV, width=i.width)
             for i in lbm_inputs.batched_sweep(48)]
    with L.Batch(insts) as b:
        b.init()
        info = b.info()
        assert info["total_nodes"] == sum(d["nx"] * d["ny"] * d["nz"] for d in insts)
        m0 = [b.diagnostics(k)["mass"] for k in (0, 17, 47)]
        b.step(4)
        b.sync()
        m1 = [b.diagnostics(k)["mass"] for k in (0, 17, 47)]
    for a, c in zip(m0, m1):
        assert abs(a - c) <= 1e-6 * a


# The single-pass batched step against the two-kernel batched step, bitwise,
# on instances the tiles of 32 x 8 nodes and z runs cut in every way: odd and
# short x extents, y not a multiple of 8, a z extent shorter than a run,
# several runs with a short last one, the minimum lattice 3 x 3 x 3; every
# storage precision; an odd number of steps (the A-B array parity) and a
# second call that continues the first.
SHAPES = ((37, 12, 9), (3, 3, 3), (70, 20, 37), (33, 8, 16), (5, 11, 3), (64, 16, 40))


@pytest.mark.parametrize("precision", ["f64", "f32", "f16dev", "bf16dev"])
def test_fused_batch_equals_two_kernel_batch(L, precision):
    insts = []
    for k, (nx, ny, nz) in enumerate(SHAPES):
        R0 = max(1.0, min(ny, nz) / 4.0)
        insts.append(dict(nx=nx, ny=ny, nz=nz, tau=0.8 + 0.05 * k, G=-5.5, R0=R0, lam=float(nx), eps=0.1,
                          phase=0.3 * k, rho_l=2.5, rho_v=0.15, width=2.0))
    res = []
    for fused, fz in ((0, 0), (1, 0), (1, 7)):
        with L.Batch(insts, precision=precision) as b:
            b.set_option("fused", fused)
            if fz:
                b.set_option("fused_fz", fz)
            b.init()
            b.step(5)
            b.step(6)
            b.sync()
            res.append([b.populations(k) for k in range(len(insts))])
    for r in res[1:]:
        for k, (a, c) in enumerate(zip(res[0], r)):
            np.testing.assert_array_equal(a, c, err_msg=str(SHAPES[k]))


# The persistent form (option persistent, with either single-pass form: all
# n steps of a call in one cooperative launch, grid barriers between the
# steps, replayed from a graph or launched directly) against one launch per
# step, bitwise: every precision (the stochastic-rounding salt advances
# the same), the instance shapes above, odd step counts and calls that
# continue one another, and fewer persistent blocks than work items (each
# block takes several tiles and z runs per step).
@pytest.mark.parametrize("precision,form,width", [("f64", 1, 0), ("f32", 1, 0), ("f16dev", 1, 0),
                                                  ("bf16dev", 1, 0), ("f32", 2, 0), ("f16dev", 2, 0),
                                                  ("bf16dev", 2, 0), ("f32", 2, 64), ("f16dev", 2, 32)])
def test_persistent_batch_equals_per_step_launches(L, precision, form, width):
    insts = []
    for k, (nx, ny, nz) in enumerate(SHAPES + ((130, 64, 96),)):
        R0 = max(1.0, min(ny, nz) / 4.0)
        insts.append(dict(nx=nx, ny=ny, nz=nz, tau=0.8 + 0.05 * k, G=-5.5, R0=R0, lam=float(nx), eps=0.1,
                          phase=0.3 * k, rho_l=2.5, rho_v=0.15, width=2.0))
    res = []
    for persistent, graph in ((0, 1), (1, 1), (1, 0)):   # the persistent launch from a graph, and direct
        with L.Batch(insts, precision=precision) as b:
            b.set_option("fused", form)
            b.set_option("tile_width", width)
            b.set_option("persistent", persistent)
            b.set_option("graph", graph)
            b.set_option("fused_fz", 4)
            b.init()
            b.step(1)
            b.step(5)
            b.step(6)
            b.sync()
            res.append([b.populations(k) for k in range(len(insts))])
    for r in res[1:]:
        for k in range(len(insts)):
            np.testing.assert_array_equal(r[k], res[0][k])


# The failure path of the persistent form's grid barrier, without a fault: a
# test hook keeps one block from arriving at the first barrier; every other
# block gives up on it after 5 ms, raises the timeout bit and returns.  The
# host reads LBM_ERR_TIMEOUT, and the batch steps correctly afterwards.
@pytest.mark.parametrize("form", [1, 2])
def test_persistent_batch_barrier_timeout(L, form):
    insts = [dict(nx=nx, ny=ny, nz=nz, tau=0.9, G=-5.5, R0=max(1.0, min(ny, nz) / 4.0), lam=float(nx), eps=0.1,
                  phase=0.0, rho_l=2.5, rho_v=0.15, width=2.0) for nx, ny, nz in SHAPES]
    with L.Batch(insts) as b:
        b.set_option("fused", form)
        b.set_option("persistent", 1)
        b.set_option("persistent_stall_test", 5.0)
        b.init()
        b.step(3)
        with pytest.raises(L.LbmError) as ei:
            b.sync()
        assert ei.value.status == L.LBM_ERR_TIMEOUT
        b.set_option("persistent_stall_test", 0)
        b.init()
        b.step(4)
        b.sync()
        got = [b.populations(k) for k in range(len(insts))]
    with L.Batch(insts) as b:
        b.init()
        b.step(4)
        want = [b.populations(k) for k in range(len(insts))]
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)


# The single pass on padded rows (option fused = 2: per-instance tensor maps,
# tiles cut at the instance's edges: tile_width 64, tiles of 64 x 4 (64 x 8
# for 2-byte storage); 32, tiles of 32 x 8 (32 x 16); 0, 64 for FP32 and 32
# for 2-byte storage) against the per-element single pass (fused = 1),
# bitwise: the shapes above plus x extents around the 32- and 64-node tiles
# (31, 33, 63, 64, 65, 96, 130) and y extents that leave a partial tile row
# (9, 13, 17, 33); an odd number of steps over two calls, a run that switches
# form in the middle (the state moves between the pools) and diagnostics
# read in the middle.
TMA_SHAPES = SHAPES + ((63, 9, 7), (64, 8, 5), (65, 13, 6), (130, 20, 37), (31, 17, 5), (96, 33, 4))


@pytest.mark.parametrize("precision,sr,width", [("f32", 1, 0), ("f16dev", 1, 0), ("bf16dev", 1, 0),
                                                ("f16dev", 0, 0), ("bf16dev", 0, 0), ("f32", 1, 32),
                                                ("f16dev", 1, 32), ("f32", 1, 64), ("bf16dev", 0, 64)])
def test_padded_tma_batch_equals_per_element_batch(L, precision, sr, width):
    insts = []
    for k, (nx, ny, nz) in enumerate(TMA_SHAPES):
        R0 = max(1.0, min(ny, nz) / 4.0)
        insts.append(dict(nx=nx, ny=ny, nz=nz, tau=0.8 + 0.04 * k, G=-5.5, R0=R0, lam=float(nx), eps=0.1,
                          phase=0.3 * k, rho_l=2.5, rho_v=0.15, width=2.0))
    res = []
    for forms in ((1, 1), (2, 2), (2, 1), (1, 2)):
        with L.Batch(insts, precision=precision) as b:
            b.set_option("fused_fz", 4)
            b.set_option("tile_width", width)
            b.set_option("stochastic_rounding", sr)
            b.init()
            b.set_option("fused", forms[0])
            b.step(5)
            # a read of two instances in the middle (from the padded form:
            # their states are copied out, the padded pool stays current)
            mid = [b.diagnostics(k)["mass"] for k in (1, len(insts) - 1)]
            b.set_option("fused", forms[1])
            b.step(6)
            b.sync()
            res.append(([b.populations(k) for k in range(len(insts))], mid))
    for r, m in res[1:]:
        assert m == res[0][1]
        for k in range(len(insts)):
            np.testing.assert_array_equal(r[k], res[0][0][k])


# Out-of-memory handling without exhausting the GPU: the allocation cap
# (LBM_ALLOC_CAP_BYTES) applies to the batch's pools at creation and to the
# padded pool of form 2 at its first step; the batch stays usable in form 1.
def test_batch_alloc_cap_gives_oom(L, monkeypatch):
    insts = [dict(nx=3, ny=12, nz=10, tau=0.9, G=-5.5, R0=2.0, lam=3.0, eps=0.1, phase=0.0, rho_l=2.5,
                  rho_v=0.15, width=2.0)]
    monkeypatch.setenv("LBM_ALLOC_CAP_BYTES", "1024")
    with pytest.raises(L.LbmError) as ei:
        L.Batch(insts)
    assert "LBM_ALLOC_CAP_BYTES" in str(ei.value)   # creation returns no handle, only the message
    # FP32, nx = 3: the padded rows (4 elements) make the padded pool 4/3 of
    # the A-B pool, above a cap 1.2 times the pools' size
    n = 3 * 12 * 10
    monkeypatch.setenv("LBM_ALLOC_CAP_BYTES", str(int(1.2 * (2 * 19 * n * 4 + n * 4))))
    with L.Batch(insts) as b:
        b.init()
        with pytest.raises(L.LbmError) as ei:
            b.step(2)
        assert ei.value.status == L.LBM_ERR_OOM
        b.set_option("fused", 1)
        b.step(2)
        b.sync()
        assert b.diagnostics(0)["numeric_ok"] == 1
    monkeypatch.delenv("LBM_ALLOC_CAP_BYTES")
