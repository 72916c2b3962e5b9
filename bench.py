"""Benchmark of the D3Q19 Shan-Chen time step: GLUPS and fraction of the HBM roofline.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the grid-convergence ligament, periodic 256 x 128 x 128 (4.19 M
nodes), R0 = 32, lambda = 256, eps = 0.02, tau = 1, G = -6, psi =
1 - exp(-rho), FP32 storage and arithmetic, A-B streaming; liquid and
vapour densities from a flat-interface run on the GPU.  One benchmark step
= 10 lattice time steps plus the FP64 diagnostics of the state (mass,
momentum, liquid volume, neck area), the diagnostic interval of this
workload.  Each lattice step runs as the single-pass fused step (whose
diagnostic-step variant also reduces the diagnostics) or as the two kernels
(psi pass, with the diagnostics on the diagnostic step, then
force/collide/stream), whichever the autotuner (run before the timed region)
finds faster on this GPU.  The timed region replays the library's captured
10-step graph once per benchmark step, as a user's lbm_step(10) does; the
per-kernel times for the roofline come from a second pass of the same number
of steps with an event pair around every kernel.  The populations (637 MB
for both arrays) exceed the 129 MB L2, so no cache flush is needed between
steps.  --workload grid1024 runs the same ligament form on 1024 x 512 x 512
(268 M nodes, 40.8 GB of FP32 populations).

--impl reference times the CPU FP64 oracle on this machine's cores on the
same box (one lattice step per benchmark step, a bounded sample).
With N > 1 (torchrun) every rank runs its own replica: the step has no
data-path collective.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbm_inputs  # noqa: E402

WORKLOAD = lbm_inputs.GRID_256
LBM_PER_STEP = 10
METRIC = "D3Q19 Shan-Chen GLUPS (giga lattice-node updates per second)"
UNIT = "GLUPS"
# algorithmic bytes per lattice update of the collide-stream kernel (FP32):
# read 19 f + write 19 f + read psi(x) once
K2_BYTES_PER_LU = {"f64": 19 * 8 * 2 + 8, "f32": 19 * 4 * 2 + 4, "f16dev": 19 * 2 * 2 + 4,
                   "bf16dev": 19 * 2 * 2 + 4}
# two-pass model of the whole step (psi pass reads 19 f and writes psi)
STEP_BYTES_PER_LU = {"f64": 3 * 19 * 8 + 16, "f32": 3 * 19 * 4 + 8, "f16dev": 3 * 19 * 2 + 8,
                     "bf16dev": 3 * 19 * 2 + 8}
# single-pass fused step: read 19 f and write 19 f (psi stays on chip)
FUSED_BYTES_PER_LU = {"f32": 19 * 4 * 2, "f16dev": 19 * 2 * 2, "bf16dev": 19 * 2 * 2}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Max of x over all ranks (the job's time is its slowest replica)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(nodes_per_rank: int, lattice_steps: int, ms: float, world: int) -> float:
    """Whole-job GLUPS: every rank advances its own replica of nodes_per_rank
    nodes by lattice_steps in the (max-over-ranks) time ms."""
    return world * nodes_per_rank * lattice_steps / (ms * 1e-3) / 1e9


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_digest(fused: bool = False) -> str:
    """sha256 over the sources of the time-step kernels (two-kernel step, or
    the single-pass fused step)."""
    h = hashlib.sha256()
    names = ("lbm_node.cuh", "lbm_fused_kernel.cuh", "lbm_device.cuh") if fused else (
        "lbm_node.cuh", "lbm_step.cu", "lbm_device.cuh")
    for name in names:
        with open(os.path.join(ROOT, "paper_1904_11792_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(workload: str, precision: str, pattern: str, fused: bool = False, fused_fz: int = 0,
                fused_group: int = 0):
    """DRAM bytes per launch of the dominant kernel (collide-stream, or the
    fused step) from the committed ncu summary, if it was taken on this
    workload, on the current kernel source and (fused step) with the same
    run length and runs per group as launched now; else None."""
    p = os.path.join(ROOT, "profiles", "collide_stream_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get("workloads", {}).get("%s/%s/%s%s" % (workload, precision, pattern, "/fused" if fused else ""))
    # one record, or a list of records taken with different fused launch shapes
    for r in (e if isinstance(e, list) else [e] if e else []):
        if r.get("kernel_source_sha256") != kernel_digest(fused):
            continue
        if fused and (r.get("fused_fz", 0), r.get("fused_group", 0)) != (fused_fz, fused_group):
            continue
        return float(r["dram_bytes_per_launch_full_size"])
    return None


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5],
                                 hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def coexistence_densities(G, tau):
    from paper_1904_11792_gb300.coexistence import coexistence
    r = coexistence(G, tau, n=64, tol=1e-10)
    return r["rho_l"], r["rho_v"]


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1904_11792_gb300 import build, lbm as L

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    L.load()
    w = lbm_inputs.GRID_1024 if args.workload == "grid1024" else WORKLOAD
    if args.workload == "grid1024":
        # 40.8 GB of FP32 populations: no host-buffer end-to-end leg and no
        # CPU oracle sample at this size
        args.no_extras = True
    N = w.nodes
    if args.rho_l and args.rho_v:
        rho_l, rho_v = args.rho_l, args.rho_v
    else:
        rho_l, rho_v = coexistence_densities(w.G, w.tau)
    # streaming pattern, block shape and register budget from the autotuner
    # (timed on this GPU before the measured region)
    from paper_1904_11792_gb300 import autotune
    patterns = ("ab", "aa") if args.pattern == "auto" else (args.pattern,)
    if args.no_tune:
        choice = dict(pattern=patterns[-1], block=(128, 2, 1), occupancy=0, fused=int(args.fused),
                      fused_fz=args.fused_fz, fused_group=args.fused_group)
    else:
        choice = autotune.tune_lattice(w.nx, w.ny, w.nz, precision=args.precision,
                                       patterns=patterns,
                                       blocks=((128, 2, 1), (64, 4, 1), (32, 8, 1)),
                                       occupancies=(2, 3), tau=w.tau, G=w.G, steps=10,
                                       use_cache=False)
    pattern = choice["pattern"]
    lat = L.Lattice(w.nx, w.ny, w.nz, w.tau, w.G, precision=args.precision, pattern=pattern,
                    rho_ref=rho_v if args.precision.endswith("dev") else 0.0)
    autotune.apply(lat, choice)
    fused = bool(lat.get_option("fused"))
    lat.init_ligament(w.R0, w.lam, w.eps, w.phase, rho_l, rho_v, w.width)
    # diagnostics inside the time loop: the psi pass of every 10th step also
    # reduces mass, momentum, liquid volume and the neck area (FP64)
    lat.set_option("diag_interval", LBM_PER_STEP)
    stream = torch.cuda.current_stream()

    def bench_step():
        lat.step(LBM_PER_STEP)

    for _ in range(args.warmup):
        bench_step()
    lat.sync()
    lat.diag_history()
    # ---- timed region: whole steps as a user runs them (each benchmark step
    # is one replay of the captured 10-step graph), device time by events on
    # the library's stream ----
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            bench_step()
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    lat.sync()
    hist = lat.diag_history()
    # ---- per-kernel device time: the same number of steps again, with an
    # event pair around every kernel (eager launches) ----
    lat.set_option("kernel_timing", 1)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        bench_step()
    torch.cuda.synchronize()
    n_psi, ms_psi = L.lbm_kernel_time(lat.h, 0)
    n_k2, ms_k2 = L.lbm_kernel_time(lat.h, 1)
    n_fu, ms_fu = L.lbm_kernel_time(lat.h, 2)
    lat.set_option("kernel_timing", 0)
    lat.sync()
    lat.diag_history()
    d = hist[-1]
    ms = max_over_ranks(ms, world, device="cuda")
    lbm_steps = args.steps * LBM_PER_STEP
    value = job_value(N, lbm_steps, ms, world)
    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None if args.no_extras else run_e2e(args, lat, L, torch, N)
    peak, peak_kind = peaks()
    k2_avg = ms_k2 / max(n_k2, 1)
    fu_avg = ms_fu / max(n_fu, 1)
    # the dominant kernel: the fused step when it runs, else collide-stream
    if fused:
        kname, bpl, avg, launches = "fused_step", FUSED_BYTES_PER_LU[args.precision], fu_avg, n_fu
        # every step fused; the diagnostic step's variant also writes the
        # partials that two small kernels reduce
        step_model = bpl
        launches_per_step = LBM_PER_STEP + 2
    else:
        kname, bpl, avg, launches = "collide_stream", K2_BYTES_PER_LU[args.precision], k2_avg, n_k2
        step_model = STEP_BYTES_PER_LU[args.precision]
        launches_per_step = 2 * (LBM_PER_STEP - 1) + 4
    achieved = bpl * N / (avg * 1e-3) / 1e9
    fz_used = int(lat.get_option("fused_fz_used")) if fused else 0
    grp_used = int(lat.get_option("fused_group_used")) if fused else 0
    traffic = ncu_traffic(args.workload, args.precision, pattern, fused, fz_used, grp_used)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "f32" else args.precision,
        "data": "synthetic (seeded ligament initial condition, no dataset)",
        "config": {
            "workload": "ligament %dx%dx%d R0=%g lambda=%g eps=%g tau=%g G=%g, %s storage, %s "
                        "streaming" % (w.nx, w.ny, w.nz, w.R0, w.lam, w.eps, w.tau, w.G,
                                       args.precision, pattern.upper()),
            "tuned": {"pattern": pattern, "fused": fused, "fused_fz": choice.get("fused_fz", 0),
                      "fused_group": choice.get("fused_group", 0), "fused_launch": [fz_used, grp_used],
                      "block": choice["block"],
                      "occupancy": choice["occupancy"], "vector": True},
            "nodes": N, "lattice_steps_per_step": LBM_PER_STEP, "diagnostics_every": LBM_PER_STEP,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "no flush: populations %.0f MB > 129 MB L2" % (
                (2 if pattern == "ab" else 1) * 19 * N
                * (4 if args.precision == "f32" else 8 if args.precision == "f64" else 2) / 1e6),
            "rho_l": round(rho_l, 6), "rho_v": round(rho_v, 6),
            "step_model_bytes_per_lu": round(step_model, 1),
            "hbm_frac_step_model": round(value / world * step_model / peak, 4),
        },
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_source": peak_kind,
                     "traffic": traffic, "bytes_per_lu": bpl,
                     "avg_launch_ms": round(avg, 5), "launches": launches,
                     "avg_launch_from": "events around every kernel in a second pass of the same "
                                        "number of steps",
                     "collide_stream_avg_ms": round(k2_avg, 5), "collide_stream_launches": n_k2,
                     "psi_pass_avg_ms": round(ms_psi / max(n_psi, 1), 5)},
        "e2e": e2e,
        "gpu_launches": int(args.steps * launches_per_step),
        "clocks": clocks,
        "diag_last": {"mass": d["mass"], "neck_radius": round(d["neck_radius"], 4),
                      "step": d["step"], "records_in_timed_region": len(hist)},
    }
    if rank == 0 and world == 1 and not args.no_extras:
        line["cpu_baseline"] = cpu_baseline(w, rho_l, rho_v)
    lat.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(args, lat, L, torch, N):
    """Same metric through the C ABI with host buffers: the state is loaded
    from pinned host memory, stepped with a diagnostics read-back every
    benchmark step, and the final density field is read back."""
    lib = L.load()
    nbytes = L.lbm_state_bytes(lat.h)
    host_state = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    rc = lib.lbm_save_state(lat.h, ctypes.c_void_p(host_state.data_ptr()), nbytes)
    L.check(rc)
    host_rho = torch.empty(N, dtype=torch.float64, pin_memory=True)
    diag = (L.lbm_diag * 4)()
    got = ctypes.c_int()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.check(lib.lbm_load_state(lat.h, ctypes.c_void_p(host_state.data_ptr()), nbytes))
    for _ in range(args.steps):
        L.check(lib.lbm_step(lat.h, LBM_PER_STEP))
        # this step's diagnostics record, read back to the host
        L.check(lib.lbm_diag_history(lat.h, diag, 4, ctypes.byref(got)))
    L.check(lib.lbm_moments(lat.h, ctypes.c_void_p(host_rho.data_ptr()), None, None, None))
    t1 = time.perf_counter()
    steps = args.steps * LBM_PER_STEP
    return {"value": round(N * steps / (t1 - t0) / 1e9, 4), "unit": UNIT,
            "h2d_bytes_per_step": int(nbytes // args.steps),
            "d2h_bytes_per_step": int(ctypes.sizeof(L.lbm_diag) + 8 * N // args.steps),
            "note": "host wall clock around the C ABI calls: state upload, graph-replayed steps "
                    "with a diagnostics read-back each benchmark step, density download"}


def cpu_baseline(w, rho_l, rho_v, budget_s: float = 12.0):
    """The oracle, as it stands, on this machine's cores: FP64 A-B steps of the
    same 256x128x128 ligament, as many as fit in about budget_s seconds."""
    import oracle
    f = oracle.init_ligament(w.nx, w.ny, w.nz, w.R0, w.lam, w.eps, w.phase, rho_l, rho_v, w.width)
    f = oracle.step(f, w.tau, w.G, 1)          # first touch of the buffers, untimed
    n, el = 0, 0.0
    t = time.perf_counter()
    while el < budget_s and n < 5000:           # blocks of 8 steps until the budget is spent
        f = oracle.step(f, w.tau, w.G, 8)
        n += 8
        el = time.perf_counter() - t
    return {"value": round(w.nodes * n / el / 1e9, 6), "unit": UNIT,
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d FP64 A-B steps of the %dx%dx%d ligament (%.1f s)" % (
                n, w.nx, w.ny, w.nz, el)}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    w = WORKLOAD
    rc = oracle.coexistence(w.tau, w.G, n=64, tol=1e-10, rho_l0=2.6, rho_v0=0.07)
    f = oracle.init_ligament(w.nx, w.ny, w.nz, w.R0, w.lam, w.eps, w.phase, rc["rho_l"],
                             rc["rho_v"], w.width)
    # a benchmark step is up to LBM_PER_STEP lattice steps, as in the GPU
    # arm, fewer when that keeps the whole run within about two minutes of
    # host time (about 0.07 s per lattice step on 16 cores)
    per = max(1, min(LBM_PER_STEP, 1700 // max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        f = oracle.step(f, w.tau, w.G, per)
    t = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.step(f, w.tau, w.G, per)
    el = time.perf_counter() - t
    value = w.nodes * args.steps * per / el / 1e9
    sample = "%d FP64 A-B lattice steps of the %dx%dx%d ligament, %d per benchmark step" % (
        args.steps * per, w.nx, w.ny, w.nz, per)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded ligament initial condition, no dataset)",
        "config": {"workload": "ligament %dx%dx%d R0=%g lambda=%g eps=%g tau=%g G=%g, CPU FP64 "
                               "oracle" % (w.nx, w.ny, w.nz, w.R0, w.lam, w.eps, w.tau, w.G),
                   "nodes": w.nodes},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args):
    """The batched sweep: 48 periodic ligaments of uneven size (R0 in
    {8..24}, box lambda x 4R0 x 4R0, tau in [0.6, 1]), FP32, stepped as one
    graph-replayed pair of launches per step for the whole batch (block size
    and register budget from the autotuner), against the same steps as
    48 x 2 launches per step, each instance launched as a standalone lattice
    of its size runs by default."""
    import torch
    from paper_1904_11792_gb300 import autotune, build, lbm as L
    torch.cuda.set_device(dist_env()[2])
    build.build()
    L.load()
    rho_l, rho_v = (args.rho_l, args.rho_v) if (args.rho_l and args.rho_v) else \
        coexistence_densities(-6.0, 1.0)
    sweep = lbm_inputs.batched_sweep(48)
    insts = [dict(nx=i.nx, ny=i.ny, nz=i.nz, tau=i.tau, G=i.G, R0=i.R0, lam=i.lam, eps=i.eps,
                  phase=i.phase, rho_l=rho_l, rho_v=rho_v, width=i.width) for i in sweep]
    total = sum(d["nx"] * d["ny"] * d["nz"] for d in insts)
    stream = torch.cuda.current_stream()
    with L.Batch(insts, precision=args.precision) as b:
        b.init()
        tuned = autotune.tune_batch(b, blocks=((256, 1, 1), (128, 1, 1)), occupancies=(2, 3, 4), steps=10)
        b.init()

        def timed(fn, nsteps):
            for _ in range(args.warmup):
                fn(LBM_PER_STEP)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(nsteps):
                fn(LBM_PER_STEP)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        with Clocks(dist_env()[2]) as clk:
            ms_b = timed(b.step, args.steps)
        ms_s = timed(b.step_sequential, args.steps)
        unstable = [k for k in range(len(insts)) if b.diagnostics(k)["numeric_ok"] != 1]
        try:
            b.sync()
        except L.LbmError:
            pass
    steps = args.steps * LBM_PER_STEP
    value = total * steps / (ms_b * 1e-3) / 1e9
    seq = total * steps / (ms_s * 1e-3) / 1e9
    peak, _ = peaks()
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_b / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
        "data": "synthetic (seeded ligament sweep, no dataset)",
        "config": {"workload": "batched sweep: 48 periodic ligaments, R0 in {8,12,16,20,24}, "
                               "lambda/R0 in [4.5,12], tau in [0.6,1.0], G=-6, eps=0.05, box "
                               "lambda x 4R0 x 4R0, %s A-B" % args.precision,
                   "total_nodes": total, "lattice_steps_per_step": LBM_PER_STEP,
                   "mode": "one psi + one collide launch per step for all instances, graph",
                   "tuned": tuned,
                   "sequential_glups": round(seq, 4),
                   "speedup_vs_sequential": round(value / seq, 3),
                   "hbm_frac_step_model": round(value * STEP_BYTES_PER_LU[args.precision] / peak, 4),
                   "unstable_instances": unstable,
                   "note": "instances with tau < ~0.75 go non-finite from the tanh start "
                           "(G=-6 SRT stability limit); their launches still run in full"},
        "clocks": clk.summary(),
        "gpu_launches": int(args.steps * LBM_PER_STEP * 2),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("grid256", "grid1024", "batch48"), default="grid256",
                    help="grid256: the headline ligament; grid1024: the 1024x512x512 ligament "
                         "(268 M nodes; device legs only); batch48: the batched sweep")
    ap.add_argument("--precision", choices=("f32", "f64", "f16dev", "bf16dev"), default="f32")
    ap.add_argument("--pattern", choices=("auto", "ab", "aa"), default="auto",
                    help="streaming pattern; auto = the autotuner's choice")
    ap.add_argument("--rho-l", type=float, default=None,
                    help="liquid density (with --rho-v: skip the flat-interface run)")
    ap.add_argument("--rho-v", type=float, default=None)
    ap.add_argument("--fused", action="store_true",
                    help="with --no-tune: the single-pass fused step on non-diagnostic A-B steps "
                         "(the autotuner otherwise chooses)")
    ap.add_argument("--fused-fz", type=int, default=0,
                    help="with --no-tune --fused: z planes per block (0 = automatic)")
    ap.add_argument("--fused-group", type=int, default=0,
                    help="with --no-tune --fused: z runs per group of the block order (0 = automatic)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (default launch configuration; profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the end-to-end and CPU-baseline legs (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch48":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
