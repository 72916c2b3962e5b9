"""The multiple-relaxation-time collision on the GPU (option "collision" = 1)
against the oracle's MRT step with Guo forcing (the operator the paper's
conclusions name as the next step).

Tolerances as for the paper's SRT step: FP64 storage 1e-12 relative after
100 steps, FP32 1e-5; layout equivalences bitwise.
"""
import numpy as np
import pytest

import lbm_inputs
import oracle

pytestmark = pytest.mark.gpu

G53 = -5.3
RATES = dict(mrt_s_e=1.19, mrt_s_eps=1.4, mrt_s_q=1.2, mrt_s_pi=1.4, mrt_s_m=1.98)


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
    r = oracle.coexistence(1.0, G53, n=64, tol=1e-10, rho_l0=2.2, rho_v0=0.15,
                           mrt_rates=oracle.mrt_rates(1.0), max_steps=200000)
    return r["rho_l"], r["rho_v"]


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def mrt_lattice(L, shape, tau, precision="f64", pattern="ab", rates=RATES, **kw):
    nx, ny, nz = shape
    lat = L.Lattice(nx, ny, nz, tau, G53, precision=precision, pattern=pattern, **kw)
    lat.set_option("collision", 1)
    for k, v in rates.items():
        lat.set_option(k, v)
    return lat


def oracle_rates(tau, rates=RATES):
    return oracle.mrt_rates(tau, rates["mrt_s_e"], rates["mrt_s_eps"], rates["mrt_s_q"],
                            rates["mrt_s_pi"], rates["mrt_s_m"])


@pytest.mark.parametrize("shape", [(37, 11, 9), (5, 3, 7), (64, 16, 12)])
def test_mrt_f64_random_state_matches_oracle(L, shape):
    f0 = lbm_inputs.random_populations(*shape, seed=61, rho_lo=0.3, rho_hi=2.2)
    tau = 0.9
    want = oracle.step_forcing(f0, G53, 20, rates=oracle_rates(tau))
    with mrt_lattice(L, shape, tau) as lat:
        lat.set_populations(f0)
        lat.step(20)
        got = lat.populations()
    assert rel(got, want) <= 1e-12


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_mrt_ligament_matches_oracle(L, coex, precision, tol, pattern):
    rl, rv = coex
    shape = (64, 32, 32)
    tau = 0.8
    f0 = oracle.init_ligament(*shape, 8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
    want = oracle.step_forcing(f0, G53, 100, rates=oracle_rates(tau))
    with mrt_lattice(L, shape, tau, precision, pattern) as lat:
        lat.init_ligament(8.0, 64.0, 0.05, 0.0, rl, rv, 2.0)
        lat.step(100)
        got_rho = lat.rho()
        got = lat.populations()
    assert rel(got_rho, want.sum(axis=0)) <= tol
    if precision == "f64":
        assert rel(got, want) <= tol


def test_mrt_with_one_rate_matches_oracle_srt_guo(L):
    shape = (20, 9, 8)
    tau = 0.85
    f0 = lbm_inputs.random_populations(*shape, seed=62, rho_lo=0.3, rho_hi=2.2)
    want = oracle.step_forcing(f0, G53, 10, rates=None, tau=tau)
    one = {k: 1.0 / tau for k in RATES}
    with mrt_lattice(L, shape, tau, rates=one) as lat:
        lat.set_populations(f0)
        lat.step(10)
        got = lat.populations()
    assert rel(got, want) <= 1e-12


@pytest.mark.parametrize("precision", ["f64", "f32", "f16dev"])
def test_mrt_layouts_and_graphs_are_bitwise_equal(L, precision):
    shape = (34, 10, 7)
    f0 = lbm_inputs.random_populations(*shape, seed=63, rho_lo=0.3, rho_hi=2.2)
    out = []
    for pattern, vec, graph in (("ab", 1, 1), ("aa", 1, 1), ("ab", 0, 0), ("aa", 0, 1)):
        with mrt_lattice(L, shape, 0.9, precision, pattern, rho_ref=0.1) as lat:
            lat.set_option("vector", vec)
            lat.set_option("graph", graph)
            assert lat.get_option("fused") == 0      # nx % 64 != 0: two-kernel step
            lat.set_populations(f0)
            lat.step(7)
            out.append(lat.populations())
    for o in out[1:]:
        np.testing.assert_array_equal(o, out[0])


def test_mrt_conserves_mass_and_momentum(L):
    shape = (32, 16, 16)
    f0 = lbm_inputs.random_populations(*shape, seed=64, rho_lo=0.3, rho_hi=2.2)
    with mrt_lattice(L, shape, 0.9) as lat:
        lat.set_populations(f0)
        d0 = lat.diagnostics()
        lat.step(50)
        d1 = lat.diagnostics()
    assert abs(d1["mass"] / d0["mass"] - 1) < 1e-13
    for k in range(3):
        assert abs(d1["mom"][k] - d0["mom"][k]) < 1e-11 * d0["mass"]


def test_mrt_flat_interface_on_gpu_is_viscosity_independent(L, coex):
    from paper_1904_11792_gb300.coexistence import coexistence
    got = [coexistence(G53, tau, n=64, tol=1e-10, rho_l0=2.2, rho_v0=0.15,
                       options=dict(collision=1, **RATES)) for tau in (1.0, 1.5)]
    rl, rv = coex
    for r in got:
        assert abs(r["rho_l"] - rl) < 1e-8 and abs(r["rho_v"] - rv) < 1e-8


def test_mrt_options_are_checked(L):
    with mrt_lattice(L, (8, 8, 8), 1.0) as lat:
        assert lat.get_option("collision") == 1
        assert lat.get_option("mrt_s_q") == pytest.approx(1.2)
        for bad in (0.0, 2.0, -1.0):
            with pytest.raises(L.LbmError) as ei:
                lat.set_option("mrt_s_e", bad)
            assert ei.value.status == L.LBM_ERR_ARG
        with pytest.raises(L.LbmError):
            lat.set_option("collision", 2)


@pytest.mark.parametrize("precision", ["f32", "f16dev"])
def test_mrt_fused_equals_two_kernel_step_bitwise(L, coex, precision):
    rl, rv = coex
    shape = (64, 16, 12)
    out = []
    for fused in (1, 0):
        with mrt_lattice(L, shape, 0.8, precision, rho_ref=rv if precision.endswith("dev") else 0.0) as lat:
            lat.set_option("fused", fused)
            assert lat.get_option("fused") == fused
            lat.init_ligament(4.0, 64.0, 0.1, 0.0, rl, rv, 2.0)
            lat.set_option("diag_interval", 5)
            lat.step(23)
            out.append((lat.populations(), [h["liquid_count"] for h in lat.diag_history()]))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
