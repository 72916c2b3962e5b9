"""Ligament break-up studies run through liblbm.so.

``breakup``: one perturbed ligament advanced until the liquid neck pinches
off (the first diagnostic step at which some x-slice holds no liquid node),
then a few more steps, with the droplets counted by connected-component
labelling.  ``precision_study`` runs the same ligament with each storage
precision and reports, against the FP64 run, the break-up time error, the
satellite volume and the mass drift.  ``surface_tension`` measures sigma from
static cylinders (Laplace law with the pressure of Eq. 7), which gives the
capillary time t_cap = sqrt(rho_l R0^3 / sigma) of Eq. 8 for scaling the
break-up time.

CLI:  python -m paper_1904_11792_gb300.studies precision [--size 256 --tau 1.0 ...]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lbm as L
from .coexistence import coexistence


def surface_tension(G: float, tau: float, radii=(8.0, 10.0, 12.0, 16.0), n: int = 49,
                    rho_l: float | None = None, rho_v: float | None = None,
                    tol: float = 1e-9, max_steps: int = 40000) -> dict:
    """sigma from static cylinders along x (Laplace: dp = sigma / R), FP64."""
    if rho_l is None or rho_v is None:
        c = coexistence(G, tau)
        rho_l, rho_v = c["rho_l"], c["rho_v"]
    dps = []
    for R in radii:
        with L.Lattice(4, n, n, tau, G, precision="f64") as lat:
            lat.init_ligament(R, 4.0, 0.0, 0.0, rho_l, rho_v, 2.0)
            prev = None
            steps = 0
            while steps < max_steps:
                lat.step(500)
                steps += 500
                rho = lat.rho()[:, :, 1]
                if prev is not None and np.abs(rho - prev).max() < tol:
                    break
                prev = rho
        psi = 1.0 - np.exp(-rho)
        P = rho / 3.0 + G / 6.0 * psi ** 2            # Eq. 7, cs^2 = 1/3
        c0 = n // 2
        dps.append(float(P[c0, c0] - P[0, 0]))
    inv = np.array([1.0 / R for R in radii])
    sigma = float(inv @ np.array(dps) / (inv @ inv))
    return dict(sigma=sigma, dp=dps, radii=list(radii), rho_l=rho_l, rho_v=rho_v)


def breakup(nx, ny, nz, R0, lam, eps, tau, G=-6.0, precision="f64", pattern="ab",
            rho_l=None, rho_v=None, width=2.0, phase=0.0, diag_interval=10,
            max_steps=60000, after=200, chunk=1000) -> dict:
    """Runs one ligament to break-up; returns the break-up step (None if it
    did not happen within max_steps), the droplets after it, mass drift and
    the neck radius history."""
    if rho_l is None or rho_v is None:
        c = coexistence(G, tau)
        rho_l, rho_v = c["rho_l"], c["rho_v"]
    t0 = time.time()
    with L.Lattice(nx, ny, nz, tau, G, precision=precision, pattern=pattern,
                   rho_ref=rho_v if precision.endswith("dev") else 0.0) as lat:
        lat.init_ligament(R0, lam, eps, phase, rho_l, rho_v, width)
        lat.set_option("diag_interval", diag_interval)
        d0 = lat.diagnostics()
        t_bu = None
        neck = []
        steps = 0
        while steps < max_steps and t_bu is None:
            lat.step(chunk)
            steps += chunk
            for rec in lat.diag_history():
                neck.append((rec["step"], rec["neck_radius"]))
                if not rec["numeric_ok"]:
                    raise FloatingPointError("%s run went non-finite at step %d" % (precision, rec["step"]))
                if t_bu is None and rec["min_slice_count"] == 0:
                    t_bu = rec["step"]
        if t_bu is not None:
            lat.step(after)
        d1 = lat.diagnostics(ccl=True)
        lat.sync()
    sat_nodes = d1["liquid_count"] - d1["largest_droplet"] if d1["droplets"] > 0 else 0
    return dict(precision=precision, breakup_step=t_bu, steps_run=steps + (after if t_bu else 0),
                droplets=d1["droplets"], droplets_min8=d1["droplets_min8"],
                satellite_nodes=int(sat_nodes), liquid_nodes=d1["liquid_count"],
                liquid_volume_w=d1["liquid_volume_w"],
                mass0=d0["mass"], mass1=d1["mass"],
                mass_drift=(d1["mass"] - d0["mass"]) / d0["mass"],
                neck=neck, wall_s=time.time() - t0)


def precision_study(nx, ny, nz, R0, lam, eps, tau, G=-6.0,
                    precisions=("f64", "f32", "f16dev", "bf16dev"), **kw) -> dict:
    c = coexistence(G, tau)
    runs = {p: breakup(nx, ny, nz, R0, lam, eps, tau, G, precision=p, rho_l=c["rho_l"],
                       rho_v=c["rho_v"], **kw) for p in precisions}
    ref = runs["f64"]
    out = {"config": dict(nx=nx, ny=ny, nz=nz, R0=R0, lam=lam, eps=eps, tau=tau, G=G),
           "rho_l": c["rho_l"], "rho_v": c["rho_v"], "runs": {}}
    for p, r in runs.items():
        e = {k: r[k] for k in ("breakup_step", "droplets", "droplets_min8", "satellite_nodes",
                               "liquid_nodes", "mass_drift", "wall_s")}
        if ref["breakup_step"] and r["breakup_step"]:
            e["breakup_error"] = (r["breakup_step"] - ref["breakup_step"]) / ref["breakup_step"]
        if ref["satellite_nodes"]:
            e["satellite_error"] = (r["satellite_nodes"] - ref["satellite_nodes"]) / ref["satellite_nodes"]
        out["runs"][p] = e
    return out


# Table 1 of the paper (section "Results"): R0, rho_l, rho_v, sigma at G0 = 5.3
# (G = -5.3) and Oh = 0.1.
TABLE1 = ((7, 2.112, 0.081, 0.05159), (14, 2.117, 0.084, 0.05345), (28, 2.125, 0.090, 0.05775),
          (42, 2.135, 0.097, 0.06277), (56, 2.145, 0.106, 0.06848), (70, 2.156, 0.116, 0.07491),
          (84, 2.167, 0.126, 0.08206))


def tau_from_oh(R0: float, rho_l: float, sigma: float, Oh: float = 0.1) -> float:
    """tau with Oh = nu sqrt(rho_l / (sigma R0)), nu = (tau - 1/2)/3 (the
    dimensionally consistent reading of Eq. 8)."""
    return 0.5 + 3.0 * Oh * math.sqrt(sigma * R0 / rho_l)


def table1(G: float = -5.3, radii=(8.0, 10.0, 12.0, 16.0)) -> list:
    """Reproduces Table 1 on the GPU: for each column, tau from Oh = 0.1,
    flat-interface rho_l, rho_v and sigma from static cylinders."""
    rows = []
    for R0, rl_p, rv_p, sg_p in TABLE1:
        tau = tau_from_oh(R0, rl_p, sg_p)
        c = coexistence(G, tau, rho_l0=2.1, rho_v0=0.1)
        sg = surface_tension(G, tau, radii=radii, rho_l=c["rho_l"], rho_v=c["rho_v"])
        rows.append(dict(R0=R0, tau=tau, rho_l=c["rho_l"], rho_v=c["rho_v"], sigma=sg["sigma"],
                         paper=dict(rho_l=rl_p, rho_v=rv_p, sigma=sg_p)))
    return rows


def breakup_vs_radius(radii=(7, 14, 28, 42, 56, 70, 84), G: float = -5.3, eps: float = 0.1,
                      kR0: float = 0.7, precision: str = "f32", check: int = 100,
                      max_steps: int = 80000, table=None) -> list:
    """The paper's study (Fig. 2): dimensionless break-up time t_bu / t_cap
    against R0 at G = -5.3, Oh = 0.1, all radii in one batch (box
    lambda x 4 R0 x 4 R0, lambda = 2 pi R0 / kR0, perturbation eps R0)."""
    if table is None:
        table = {r["R0"]: r for r in table1(G)}
    insts = []
    for R0 in radii:
        t = table[R0]
        lam = int(round(2 * math.pi * R0 / kR0))
        insts.append(dict(nx=lam, ny=4 * R0, nz=4 * R0, tau=t["tau"], G=G, R0=float(R0),
                          lam=float(lam), eps=eps, phase=0.0, rho_l=t["rho_l"], rho_v=t["rho_v"],
                          width=2.0))
    t_bu = [None] * len(insts)
    nonfinite = [None] * len(insts)     # step at which an instance lost finiteness
    steps = 0
    with L.Batch(insts, precision=precision) as b:
        b.init()
        while steps < max_steps and any(t is None and n is None for t, n in zip(t_bu, nonfinite)):
            b.step(check)
            steps += check
            for k in range(len(insts)):
                if t_bu[k] is None and nonfinite[k] is None:
                    d = b.diagnostics(k)
                    if not d["numeric_ok"]:
                        nonfinite[k] = steps
                    elif d["min_slice_count"] == 0:
                        t_bu[k] = steps
        try:
            b.sync()
        except L.LbmError as e:
            # an instance past its break-up step (or already reported above)
            # lost finiteness; the instances are independent, so the recorded
            # break-up steps of the others stand
            if e.status != L.LBM_ERR_NUMERIC:
                raise
    out = []
    for k, R0 in enumerate(radii):
        t = table[R0]
        t_cap = math.sqrt(t["rho_l"] * R0 ** 3 / t["sigma"])
        out.append(dict(R0=R0, tau=t["tau"], lam=insts[k]["nx"], nodes=insts[k]["nx"] * 16 * R0 * R0,
                        breakup_step=t_bu[k], nonfinite_step=nonfinite[k], t_cap=t_cap,
                        breakup_over_tcap=(t_bu[k] / t_cap) if t_bu[k] else None))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=("precision", "sigma", "table1", "radius"))
    ap.add_argument("--nx", type=int, default=256)
    ap.add_argument("--ny", type=int, default=128)
    ap.add_argument("--nz", type=int, default=128)
    ap.add_argument("--R0", type=float, default=32.0)
    ap.add_argument("--lam", type=float, default=256.0)
    ap.add_argument("--eps", type=float, default=0.02)
    ap.add_argument("--tau", type=float, default=1.0)
    ap.add_argument("--G", type=float, default=-6.0)
    ap.add_argument("--max-steps", type=int, default=60000)
    ap.add_argument("--precisions", default="f64,f32,f16dev,bf16dev")
    a = ap.parse_args()
    if a.study == "sigma":
        print(json.dumps(surface_tension(a.G, a.tau)))
        return
    if a.study == "table1":
        print(json.dumps(table1()))
        return
    if a.study == "radius":
        t = table1()
        print(json.dumps({"table1": t}), flush=True)
        print(json.dumps({"breakup": breakup_vs_radius(table={r["R0"]: r for r in t},
                                                                     max_steps=a.max_steps)}))
        return
    res = precision_study(a.nx, a.ny, a.nz, a.R0, a.lam, a.eps, a.tau, a.G,
                          precisions=tuple(a.precisions.split(",")), max_steps=a.max_steps)
    sig = surface_tension(a.G, a.tau, rho_l=res["rho_l"], rho_v=res["rho_v"])
    res["sigma"] = sig["sigma"]
    res["t_cap"] = math.sqrt(res["rho_l"] * a.R0 ** 3 / sig["sigma"])
    for r in res["runs"].values():
        if r["breakup_step"]:
            r["breakup_over_tcap"] = r["breakup_step"] / res["t_cap"]
    print(json.dumps(res))


if __name__ == "__main__":
    main()
