"""Droplet statistics on the GPU (lbm_droplets and the labelling inside the
time loop) against the oracle's flood-fill droplets on the same state.

Node counts, first node indices and x extents must match exactly; the FP64
sums (volume, mass, centroid sums) are accumulated with atomics in any
order, so they match to rounding: 1e-12 relative for FP64 storage; for
reduced storage the oracle reads the stored populations, and the GPU sums
rho in FP32 (1e-5).
"""
import numpy as np
import pytest

import lbm_inputs
import oracle

pytestmark = pytest.mark.gpu

RL, RV = 2.65, 0.073


@pytest.fixture(scope="module")
def L():
    from paper_1904_11792_gb300 import build, lbm
    build.build()
    lbm.load()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lbm


def lattice(L, shape, precision="f64", pattern="ab"):
    nx, ny, nz = shape
    lat = L.Lattice(nx, ny, nz, 1.0, -6.0, precision=precision, pattern=pattern,
                    rho_ref=RV if precision.endswith("dev") else 0.0)
    lat.set_option("rho_l", RL)
    lat.set_option("rho_v", RV)
    return lat


def compare(got_n, got, want_n, want, shape, tol):
    nx, ny, nz = shape
    assert got_n == want_n
    assert len(got) == want.shape[0]
    for g, w in zip(got, want):
        assert (g["first_node"], g["nodes"], g["x_slices"]) == (int(w[0]), int(w[1]), int(w[10]))
        assert g["volume_w"] == pytest.approx(w[2], rel=tol)
        assert g["mass"] == pytest.approx(w[3], rel=tol)
        for d, n in enumerate((nx, ny, nz)):
            assert g["resultant"][d] == pytest.approx(w[7 + d], abs=max(tol, 1e-12))
            if w[7 + d] > 1e-3:
                e = abs(g["centroid"][d] - w[4 + d])
                assert min(e, n - e) < 1e3 * tol * n, (d, g["centroid"], w[4:7])


@pytest.mark.parametrize("shape,p,seed", [((37, 20, 18), 0.3, 21), ((64, 32, 32), 0.25, 22),
                                           ((33, 9, 40), 0.45, 23)])
def test_droplets_f64_match_oracle(L, shape, p, seed):
    nx, ny, nz = shape
    f = lbm_inputs.droplet_populations(nx, ny, nz, seed=seed, p=p, rho_l=RL, rho_v=RV)
    with lattice(L, shape) as lat:
        lat.set_populations(f)
        n, got = lat.droplets()
    wn, want = oracle.droplets(f, RL, RV)
    compare(n, got, wn, want, shape, 1e-12)


@pytest.mark.parametrize("precision", ["f32", "f16dev", "bf16dev"])
def test_droplets_reduced_storage(L, precision):
    shape = (48, 24, 20)
    f = lbm_inputs.droplet_populations(*shape, seed=31, p=0.3, rho_l=RL, rho_v=RV)
    with lattice(L, shape, precision) as lat:
        lat.set_populations(f)
        stored = lat.populations()
        n, got = lat.droplets()
    wn, want = oracle.droplets(stored, RL, RV)
    compare(n, got, wn, want, shape, 1e-5)


def test_droplets_aa_odd_layout(L):
    # after one AA step the populations sit in the odd-step layout
    shape = (40, 16, 16)
    f = lbm_inputs.droplet_populations(*shape, seed=41, p=0.35, rho_l=RL, rho_v=RV)
    with lattice(L, shape, "f64", "aa") as lat:
        lat.set_populations(f)
        lat.step(1)
        state = lat.populations()
        n, got = lat.droplets()
    wn, want = oracle.droplets(state, RL, RV)
    compare(n, got, wn, want, shape, 1e-12)


def test_droplets_limit_and_edge_cases(L):
    shape = (20, 10, 12)
    with lattice(L, shape) as lat:
        lat.set_populations(lbm_inputs.droplet_populations(*shape, seed=3, mask=np.zeros(shape[::-1], bool)))
        assert lat.droplets()[0] == 0
        lat.set_populations(lbm_inputs.droplet_populations(*shape, seed=3, mask=np.ones(shape[::-1], bool)))
        n, got = lat.droplets()
        assert n == 1 and got[0]["nodes"] == 2400 and got[0]["x_slices"] == 20 and got[0]["first_node"] == 0
        f = lbm_inputs.droplet_populations(*shape, seed=4, p=0.3, rho_l=RL, rho_v=RV)
        lat.set_populations(f)
        n, got = lat.droplets(max_droplets=5)
        wn, want = oracle.droplets(f, RL, RV, max_out=5)
        assert n == wn and len(got) == 5
        compare(n, got, wn, want, shape, 1e-12)
        n0, none = lat.droplets(max_droplets=0)
        assert n0 == wn and none == []


def test_droplet_counts_inside_the_time_loop(L):
    # a ligament past its break-up: records of the in-loop labelling equal
    # the on-demand labelling of the same steps (both deterministic)
    shape = (64, 32, 32)
    c = oracle.coexistence(1.0, -6.0, n=64, tol=1e-10, rho_l0=2.6, rho_v0=0.07)
    rl, rv = c["rho_l"], c["rho_v"]
    nx, ny, nz = shape

    def make():
        lat = L.Lattice(nx, ny, nz, 1.0, -6.0, precision="f32", pattern="ab")
        lat.init_ligament(8.0, 64.0, 0.3, 0.0, rl, rv, 2.0)   # kR0 = 0.79: unstable
        return lat

    with make() as a, make() as b:
        a.set_option("diag_interval", 50)
        a.set_option("diag_ccl", 1)
        a.step(1000)                      # pinches off near step 500
        recs = a.diag_history()
        assert len(recs) == 20
        b.set_option("graph", 0)
        for r in recs[::3]:
            b.step(r["step"] - int(L.lbm_get_option(b.h, "step")))
            d = b.diagnostics(ccl=True)
            assert (r["droplets"], r["droplets_min8"], r["largest_droplet"]) == \
                (d["droplets"], d["droplets_min8"], d["largest_droplet"]), r["step"]
        assert recs[0]["droplets"] == 1 and recs[0]["min_slice_count"] > 0
        assert recs[-1]["min_slice_count"] == 0 and recs[-1]["droplets"] >= 1   # pinched off
        a.set_option("diag_ccl", 0)
        a.step(50)
        assert a.diag_history()[-1]["droplets"] == -1
