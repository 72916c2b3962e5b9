"""Plateau-Rayleigh cut-off on the batched sweep (the 48 uneven ligaments,
lambda x 4 R0 x 4 R0, R0 in {8, ..., 24}, lambda / R0 in [4.5, 12]) through
the batched single-pass step: the cosine perturbation of a ligament grows
iff k R0 < 1, k = 2 pi / lambda (the cut-off of the Rayleigh dispersion
relation; the oracle is pinned to it in test_oracle_pins).  The sweep's
instances with lambda / R0 < 2 pi are Rayleigh-stable and must not break up;
the others must.  tau = 1 for every instance (the drawn tau in [0.6, 1]
leaves some instances unstable for the SRT model at G = -6)."""
import math

import numpy as np
import pytest

import lbm_inputs

pytestmark = pytest.mark.gpu

RL, RV = 2.648878066946715, 0.0731992478525716   # G = -6, tau = 1 flat-interface run


@pytest.fixture(scope="module")
def L():
    from paper_1904_11792_gb300 import build, lbm
    build.build()
    lbm.load()
    return lbm


def _mode_amplitude(f, lam):
    """Amplitude of the fundamental x mode of the local radius sqrt(A(x) / pi),
    A(x) the liquid fraction summed over the slice x (the diagnostics' A_w)."""
    rho = f.sum(axis=0)                                  # [nz, ny, nx]
    phi = np.clip((rho - RV) / (RL - RV), 0.0, 1.0)
    r = np.sqrt(phi.sum(axis=(0, 1)) / math.pi)
    x = np.arange(lam)
    return abs((r * np.exp(-2j * math.pi * x / lam)).sum()) * 2.0 / lam


def test_sweep_rayleigh_cutoff(L):
    sweep = lbm_inputs.batched_sweep(48)
    insts = [dict(nx=i.nx, ny=i.ny, nz=i.nz, tau=1.0, G=-6.0, R0=i.R0, lam=i.lam, eps=i.eps, phase=i.phase,
                  rho_l=RL, rho_v=RV, width=2.0) for i in sweep]
    kR = [2.0 * math.pi * i.R0 / i.lam for i in sweep]
    # the amplitudes are read on the smaller instances (R0 <= 12: up to 0.3 M
    # nodes each), away from the cut-off where the dynamics are slow
    probe = [k for k, i in enumerate(sweep) if i.R0 <= 12 and (kR[k] >= 1.1 or kR[k] <= 0.85)]
    stable = [k for k in range(len(sweep)) if kR[k] >= 1.1]
    assert len(stable) >= 4 and any(kR[k] <= 0.85 for k in probe)
    t1, t2 = 300, 2400
    with L.Batch(insts, precision="f32") as b:
        b.init()
        b.step(t1)
        a1 = {k: _mode_amplitude(b.populations(k), sweep[k].nx) for k in probe}
        b.step(t2 - t1)
        a2 = {k: _mode_amplitude(b.populations(k), sweep[k].nx) for k in probe}
        dg = [b.diagnostics(k) for k in range(len(sweep))]
        b.sync()
    for k in range(len(sweep)):
        assert dg[k]["numeric_ok"] == 1, k
    for k in stable:
        # Rayleigh-stable: never pinched (every x slice keeps liquid nodes)
        assert dg[k]["min_slice_count"] > 0, (k, kR[k], dg[k]["neck_radius"])
    for k in probe:
        if kR[k] >= 1.1:
            assert a2[k] < 0.5 * a1[k], (k, kR[k], a1[k], a2[k])    # decays
        else:
            assert a2[k] > 3.0 * a1[k], (k, kR[k], a1[k], a2[k])    # grows (or has pinched off)
