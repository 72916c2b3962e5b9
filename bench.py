"""Benchmark of the D3Q19 Shan-Chen time step: GLUPS and fraction of the HBM roofline.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload grid1024|grid256|batch48]

Workload (default, grid1024): the large periodic ligament, 1024 x 512 x 512
(268 M nodes), R0 = 96, lambda = 1024, eps = 0.01, G = -6, psi =
1 - exp(-rho), tanh start of width 2 at the flat-interface densities of a GPU
run; tau = 1 (tau = 0.7 goes non-finite for this collision at G = -6 from
either start, so the lattice runs at the grid-convergence ligament's tau).
Headline: FP32 storage and arithmetic, the step form the autotuner (run
before the timed region) finds fastest on this GPU: the single-pass fused
A-B step, or the two-kernel A-B / AA step with its block shape.  One
benchmark step = 10 lattice time steps with the FP64 diagnostics of the
first (mass, momentum, liquid volume, neck area) reduced inside the loop;
the timed region replays the library's captured 10-step graph once per
benchmark step, as a user's lbm_step(10) does.  The populations (40.8 GB
A-B) exceed the 129 MB L2 many times over: no cache flush is needed.

The same JSON line carries the metric's comparisons ("variants"): FP16 and
BF16 deviation storage (FP32 arithmetic) in the fused A-B step, FP32 and
FP16-dev with AA in-place streaming (the two-kernel step), and the batched
sweep of 48 uneven ligaments as one graph-captured pair of launches per step
against 48 x 2 launches per step.  The dominant kernel's launch time comes
from graph replay of plain (diagnostic-free) steps, one fused launch each.

--workload grid256 runs the headline on the 256 x 128 x 128 grid-convergence
ligament; --workload batch48 prints the batched sweep as its own line.
--impl reference times the CPU FP64 oracle on this machine's cores on a
bounded sample of the same workload (a 1024 x 512 x 8 slab: the full FP64
A-B state would need 82 GB of host memory; the oracle's work per node does
not depend on the box).  With N > 1 (torchrun) every rank runs its own
replica: the step has no data-path collective.
"""
from __future__ import annotations

import argparse
import ctypes
import dataclasses
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbm_inputs  # noqa: E402

WORKLOADS = {"grid1024": lbm_inputs.GRID_1024, "grid256": lbm_inputs.GRID_256}
LBM_PER_STEP = 10
METRIC = "D3Q19 Shan-Chen GLUPS (giga lattice-node updates per second)"
UNIT = "GLUPS"
ELEM = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}
# algorithmic bytes per lattice update (s = bytes per stored population):
# collide-stream kernel: read 19 f + psi(x), write 19 f
K2_BYTES_PER_LU = {p: 19 * s * 2 + (8 if p == "f64" else 4) for p, s in ELEM.items()}
# two-kernel step: the psi pass reads 19 f and writes psi, then collide-stream
STEP_BYTES_PER_LU = {p: 3 * 19 * s + (16 if p == "f64" else 8) for p, s in ELEM.items()}
# single-pass fused step: read 19 f and write 19 f (psi stays on chip)
FUSED_BYTES_PER_LU = {p: 19 * s * 2 for p, s in ELEM.items() if p != "f64"}
# variants carried in the headline line: (name, precision, pattern)
VARIANTS = (("f16dev_ab", "f16dev", "ab"), ("bf16dev_ab", "bf16dev", "ab"), ("f32_aa", "f32", "aa"),
            ("f16dev_aa", "f16dev", "aa"))
SLAB_NZ = 8     # z planes of the oracle's sample of the 1024 x 512 x 512 workload


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


def source_code_bytes(text: str) -> bytes:
    """A source file without its comments and blank lines: what the compiler
    sees of it (so that the digest below changes with the code, not with the
    text around it)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln.strip()).encode()


def kernel_digest(fused: bool = False, read=None) -> str:
    """sha256 over the code (comments stripped) of the time-step kernels'
    sources (two-kernel step, or the single-pass fused step); `read` maps a
    file name to its text (default: the files of this tree)."""
    h = hashlib.sha256()
    names = ("lbm_node.cuh", "lbm_fused_kernel.cuh", "lbm_device.cuh") if fused else (
        "lbm_node.cuh", "lbm_step.cu", "lbm_device.cuh")
    for name in names:
        if read is None:
            with open(os.path.join(ROOT, "paper_1904_11792_gb300", "csrc", name)) as fh:
                text = fh.read()
        else:
            text = read(name)
        h.update(source_code_bytes(text))
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

    def __init__(self, index: int, period_ms: int = 50):
        self.index = index
        self.period_ms = period_ms
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
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
                "samples": len(rows), "period_ms": self.period_ms}


def coexistence_densities(G, tau):
    from paper_1904_11792_gb300.coexistence import coexistence
    r = coexistence(G, tau, n=64, tol=1e-10)
    return r["rho_l"], r["rho_v"]


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure_lattice(torch, L, autotune, w, precision, patterns, args, rho_l, rho_v, world=1, clocks=None,
                    full_tune=True):
    """Times one lattice configuration: tuner choice, the timed benchmark
    steps (graph replay of lbm_step(10) with in-loop diagnostics every 10
    steps), and the per-step time of plain steps (graph replay, no
    diagnostics), from which the fused step's launch time follows."""
    import torch.distributed as dist
    dev = precision.endswith("dev")
    if args.no_tune:
        choice = dict(pattern=patterns[-1], block=(128, 2, 1), occupancy=0, fused=int(args.fused),
                      fused_fz=args.fused_fz, fused_group=args.fused_group)
    elif full_tune:
        choice = autotune.tune_lattice(w.nx, w.ny, w.nz, precision=precision, patterns=patterns,
                                       blocks=((128, 2, 1), (64, 4, 1), (32, 8, 1)), occupancies=(2, 3),
                                       tau=w.tau, G=w.G, steps=10, use_cache=False)
    else:
        # variants: the fused step's launch shapes where it applies (A-B),
        # two block shapes of the two-kernel step otherwise
        choice = autotune.tune_lattice(w.nx, w.ny, w.nz, precision=precision, patterns=patterns,
                                       blocks=((128, 2, 1), (64, 4, 1)) if patterns == ("aa",) else
                                       ((128, 2, 1),),
                                       occupancies=(2, 3), tau=w.tau, G=w.G, steps=10, use_cache=False,
                                       fused_runs=(8, 12, 16, 32), fused_groups=(1, 4), reps=2)
    pattern = choice["pattern"]
    lat = L.Lattice(w.nx, w.ny, w.nz, w.tau, w.G, precision=precision, pattern=pattern,
                    rho_ref=rho_v if dev else 0.0)
    try:
        autotune.apply(lat, choice)
        fused = bool(lat.get_option("fused"))
        lat.init_ligament(w.R0, w.lam, w.eps, w.phase, rho_l, rho_v, w.width)
        lat.set_option("diag_interval", LBM_PER_STEP)
        stream = torch.cuda.current_stream()
        for _ in range(args.warmup):
            lat.step(LBM_PER_STEP)
        lat.sync()
        lat.diag_history()
        t0, t1 = _events(torch)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.__enter__()
        t0.record(stream)
        for _ in range(args.steps):
            lat.step(LBM_PER_STEP)
        t1.record(stream)
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.__exit__(None, None, None)
        if world > 1:
            dist.barrier()
        ms = t0.elapsed_time(t1)
        lat.sync()
        hist = lat.diag_history()
        # plain steps (no in-loop diagnostics): every lattice step is one
        # launch of the fused kernel, or psi pass + collide-stream
        lat.set_option("diag_interval", 0)
        lat.step(LBM_PER_STEP)
        torch.cuda.synchronize()
        p0, p1 = _events(torch)
        p0.record(stream)
        for _ in range(args.steps):
            lat.step(LBM_PER_STEP)
        p1.record(stream)
        torch.cuda.synchronize()
        ms_plain = p0.elapsed_time(p1)
        lat.sync()
        fz_used = int(lat.get_option("fused_fz_used")) if fused else 0
        grp_used = int(lat.get_option("fused_group_used")) if fused else 0
        out = dict(lat=None, choice=choice, pattern=pattern, fused=fused, ms=ms, ms_plain=ms_plain,
                   hist=hist, fz_used=fz_used, grp_used=grp_used)
        if args.keep_lattice:
            out["lat"] = lat
            lat = None
        return out
    finally:
        if lat is not None:
            lat.close()


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1904_11792_gb300 import autotune, build, lbm as L

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    L.load()
    w = WORKLOADS[args.workload]
    if args.nz > 0:
        w = dataclasses.replace(w, nz=args.nz)
    N = w.nodes
    if args.rho_l and args.rho_v:
        rho_l, rho_v = args.rho_l, args.rho_v
    else:
        rho_l, rho_v = coexistence_densities(w.G, w.tau)
    patterns = ("ab", "aa") if args.pattern == "auto" else (args.pattern,)
    peak, peak_kind = peaks()
    clk = Clocks(local)
    args.keep_lattice = not args.no_extras
    m = measure_lattice(torch, L, autotune, w, args.precision, patterns, args, rho_l, rho_v, world, clk)
    lat = m["lat"]
    ms = max_over_ranks(m["ms"], world, device="cuda")
    lbm_steps = args.steps * LBM_PER_STEP
    value = job_value(N, lbm_steps, ms, world)
    ms_step = ms / args.steps
    plain_step_ms = m["ms_plain"] / lbm_steps
    fused = m["fused"]
    # the dominant kernel: the fused step when it runs (one launch per plain
    # step), else collide-stream (its share of the plain step from the
    # eager per-kernel timing below)
    if fused:
        kname, bpl, avg = "fused_step", FUSED_BYTES_PER_LU[args.precision], plain_step_ms
        avg_from = ("graph replay of %d plain steps (no in-loop diagnostics), one fused launch per step, "
                    "CUDA events on the library stream" % lbm_steps)
        step_model = bpl
        launches_per_step = LBM_PER_STEP + 2
    else:
        kname, bpl = "collide_stream", K2_BYTES_PER_LU[args.precision]
        n_k2, ms_k2 = 0, 0.0
        if lat is not None:
            lat.set_option("kernel_timing", 1)
            lat.step(LBM_PER_STEP * 4)
            n_k2, ms_k2 = L.lbm_kernel_time(lat.h, 1)
            lat.set_option("kernel_timing", 0)
            lat.sync()
        avg = ms_k2 / n_k2 if n_k2 else plain_step_ms
        avg_from = "events around each collide-stream launch (eager steps)"
        step_model = STEP_BYTES_PER_LU[args.precision]
        launches_per_step = 2 * (LBM_PER_STEP - 1) + 4
    achieved = bpl * N / (avg * 1e-3) / 1e9
    traffic = None if args.nz > 0 else ncu_traffic(args.workload, args.precision, m["pattern"], fused,
                                                   m["fz_used"], m["grp_used"])
    d = m["hist"][-1] if m["hist"] else {}
    e2e = None
    if lat is not None:
        e2e = run_e2e(args, lat, L, torch, N)
        lat.close()
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision in ("f32", "f16dev", "bf16dev") else args.precision,
        "data": "synthetic (seeded ligament initial condition, no dataset)",
        "config": {
            "workload": "ligament %dx%dx%d R0=%g lambda=%g eps=%g tau=%g G=%g, %s storage, %s "
                        "streaming" % (w.nx, w.ny, w.nz, w.R0, w.lam, w.eps, w.tau, w.G,
                                       args.precision, m["pattern"].upper()),
            "tuned": {"pattern": m["pattern"], "fused": fused, "fused_fz": m["choice"].get("fused_fz", 0),
                      "fused_group": m["choice"].get("fused_group", 0),
                      "fused_launch": [m["fz_used"], m["grp_used"]], "block": m["choice"]["block"],
                      "occupancy": m["choice"]["occupancy"], "vector": True},
            "nodes": N, "lattice_steps_per_step": LBM_PER_STEP, "diagnostics_every": LBM_PER_STEP,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "no flush: populations %.1f GB > 129 MB L2" % (
                (2 if m["pattern"] == "ab" else 1) * 19 * N * ELEM[args.precision] / 1e9),
            "rho_l": round(rho_l, 6), "rho_v": round(rho_v, 6),
            "step_model_bytes_per_lu": step_model,
            "hbm_frac_step_model": round(value / world * step_model / peak, 4),
        },
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs, STREAM-style copy)",
                     "traffic": traffic, "bytes_per_lu": bpl, "avg_launch_ms": round(avg, 5),
                     "avg_launch_from": avg_from,
                     "kernel_time_check": {"ten_launches_ms": round(10 * avg, 4),
                                           "ms_per_step": round(ms_step, 4),
                                           "ok": bool(10 * avg <= ms_step * 1.001)}},
        "e2e": e2e,
        "gpu_launches": int(args.steps * launches_per_step),
        "clocks": clk.summary(),
        "diag_last": {"mass": d.get("mass"), "neck_radius": round(d.get("neck_radius", 0.0), 4),
                      "step": d.get("step"), "records_in_timed_region": len(m["hist"])},
    }
    if not args.no_variants and args.precision == "f32":
        line["variants"] = run_variants(args, torch, L, autotune, w, rho_l, rho_v, value / world, peak, world)
    if rank == 0 and world == 1 and not args.no_extras:
        line["cpu_baseline"] = cpu_baseline(w, rho_l, rho_v)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_variants(args, torch, L, autotune, w, rho_l, rho_v, fp32_glups, peak, world):
    """FP16/BF16 deviation storage and AA in-place streaming on the same
    workload, and the batched sweep, each timed like the headline."""
    out = {}
    keep = args.keep_lattice
    args.keep_lattice = False
    N = w.nodes
    for name, prec, pattern in VARIANTS:
        try:
            m = measure_lattice(torch, L, autotune, w, prec, (pattern,), args, rho_l, rho_v, world,
                                full_tune=False)
        except Exception as ex:       # a variant that fails is reported, not fatal to the line
            out[name] = {"precision": prec, "pattern": pattern, "error": str(ex)[:300]}
            continue
        ms = max_over_ranks(m["ms"], world, device="cuda")
        v = N * args.steps * LBM_PER_STEP / (ms * 1e-3) / 1e9
        bpl = FUSED_BYTES_PER_LU[prec] if m["fused"] else STEP_BYTES_PER_LU[prec]
        plain = m["ms_plain"] / (args.steps * LBM_PER_STEP)
        e = {"precision": prec, "pattern": pattern, "step_form": "fused" if m["fused"] else "two-kernel",
             "value": round(v, 4), "ms_per_step": round(ms / args.steps, 4), "vs_fp32": round(v / fp32_glups, 4),
             "bytes_per_lu": bpl, "hbm_frac_step_model": round(v * bpl / peak, 4),
             "plain_step_ms": round(plain, 5),
             "plain_step_hbm_frac": round(bpl * N / (plain * 1e-3) / 1e9 / peak, 4),
             "fused_launch": [m["fz_used"], m["grp_used"]] if m["fused"] else None,
             "numeric_ok": all(h["numeric_ok"] == 1 for h in m["hist"])}
        if m["fused"]:
            e["traffic"] = None if args.nz > 0 else ncu_traffic(args.workload, prec, pattern, True,
                                                                m["fz_used"], m["grp_used"])
        out[name] = e
    try:
        out["batched_sweep48"] = batch_sweep(args, torch, L, autotune, rho_l, rho_v)
    except Exception as ex:
        out["batched_sweep48"] = {"error": str(ex)[:300]}
    args.keep_lattice = keep
    return out


def host_memory_available() -> int:
    """Bytes of host memory this process may still take: MemAvailable,
    bounded by the cgroup's limit less its current use where one is set."""
    avail = None
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    try:
        with open("/sys/fs/cgroup/memory.max") as fh:
            lim = fh.read().strip()
        with open("/sys/fs/cgroup/memory.current") as fh:
            cur = int(fh.read().strip())
        if lim != "max":
            room = int(lim) - cur
            avail = room if avail is None else min(avail, room)
    except (OSError, ValueError):
        pass
    return avail if avail is not None else 0


def run_e2e(args, lat, L, torch, N):
    """Same metric through the C ABI with host buffers: the state is loaded
    from pinned host memory, stepped with a diagnostics read-back every
    benchmark step, and the final density field is read back."""
    lib = L.load()
    nbytes = L.lbm_state_bytes(lat.h)
    need = nbytes + 8 * N
    if 2 * need > host_memory_available():
        return {"value": None, "unit": UNIT, "h2d_bytes_per_step": int(nbytes // args.steps),
                "d2h_bytes_per_step": int(8 * N // args.steps),
                "note": "not run: the pinned host buffers (%.1f GB) need more than half of the host memory "
                        "available (%.1f GB)" % (need / 1e9, host_memory_available() / 1e9)}
    host_state = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    L.check(lib.lbm_save_state(lat.h, ctypes.c_void_p(host_state.data_ptr()), nbytes))
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
            "note": "host wall clock around the C ABI calls: state upload from pinned memory (%.1f GB), "
                    "graph-replayed steps with a diagnostics read-back each benchmark step, density "
                    "download (%.1f GB); transfers amortised per benchmark step" % (nbytes / 1e9, 8 * N / 1e9)}


def oracle_sample(w, rho_l, rho_v):
    """The oracle's state for a bounded sample of workload w: the lattice
    itself when its FP64 A-B state is small, else a slab of SLAB_NZ z planes
    of the same x-y cross-section (the same per-node work)."""
    import oracle
    nz = w.nz if w.nodes <= (1 << 23) else SLAB_NZ
    f = oracle.init_ligament(w.nx, w.ny, nz, w.R0, w.lam, w.eps, w.phase, rho_l, rho_v, w.width)
    what = ("the %dx%dx%d ligament" % (w.nx, w.ny, w.nz) if nz == w.nz else
            "a %dx%dx%d periodic slab of the %dx%dx%d ligament's cross-section (the full FP64 A-B state "
            "needs %.0f GB of host memory)" % (w.nx, w.ny, nz, w.nx, w.ny, w.nz, 2 * 19 * 8 * w.nodes / 1e9))
    return f, w.nx * w.ny * nz, what


def cpu_baseline(w, rho_l, rho_v, budget_s: float = 12.0):
    """The oracle, as it stands, on this machine's cores: FP64 A-B steps of a
    bounded sample of the workload, as many as fit in about budget_s seconds."""
    import oracle
    f, n_nodes, what = oracle_sample(w, rho_l, rho_v)
    f = oracle.step(f, w.tau, w.G, 1)          # first touch of the buffers, untimed
    n, el = 0, 0.0
    t = time.perf_counter()
    while el < budget_s and n < 5000:           # blocks of 4 steps until the budget is spent
        f = oracle.step(f, w.tau, w.G, 4)
        n += 4
        el = time.perf_counter() - t
    return {"value": round(n_nodes * n / el / 1e9, 6), "unit": UNIT,
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d FP64 A-B steps of %s (%.1f s)" % (n, what, el)}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    w = WORKLOADS.get(args.workload, lbm_inputs.GRID_1024)
    rc = oracle.coexistence(w.tau, w.G, n=64, tol=1e-10, rho_l0=2.6, rho_v0=0.07)
    f, n_nodes, what = oracle_sample(w, rc["rho_l"], rc["rho_v"])
    # a benchmark step is up to LBM_PER_STEP lattice steps of the sample, as
    # in the GPU arm, fewer when that keeps the whole run within about two
    # minutes of host time (about 0.07 s per lattice step of 4 M nodes on 16
    # cores)
    budget = 1700 * (1 << 22) // n_nodes
    per = max(1, min(LBM_PER_STEP, budget // max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        f = oracle.step(f, w.tau, w.G, per)
    t = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.step(f, w.tau, w.G, per)
    el = time.perf_counter() - t
    value = n_nodes * args.steps * per / el / 1e9
    sample = "%d FP64 A-B lattice steps of %s, %d per benchmark step" % (args.steps * per, what, per)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded ligament initial condition, no dataset)",
        "config": {"workload": "ligament %dx%dx%d R0=%g lambda=%g eps=%g tau=%g G=%g, CPU FP64 "
                               "oracle" % (w.nx, w.ny, w.nz, w.R0, w.lam, w.eps, w.tau, w.G),
                   "nodes": w.nodes, "sample_nodes": n_nodes},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_sweep(args, torch, L, autotune, rho_l, rho_v, precision="f32"):
    """The batched sweep: 48 periodic ligaments of uneven size (R0 in
    {8..24}, box lambda x 4R0 x 4R0), stepped as one graph-replayed pair of
    launches per step for the whole batch (block size and register budget
    from the autotuner), against the same steps as 48 x 2 launches per step,
    each instance launched as a standalone lattice of its size.  At the drawn
    tau in [0.6, 1] some instances go non-finite (the SRT stability limit at
    G = -6, reading R15); they are listed from an untimed run, and the two
    arms are timed, each from the same initial state, on the sweep with tau
    raised to the smallest floor (0.8, 0.9 or 1) at which every instance
    stays finite through all the steps the timing takes."""
    sweep = lbm_inputs.batched_sweep(48)[:args.batch_size]
    n_steps = (args.warmup + args.steps) * LBM_PER_STEP + 40

    def insts(floor):
        return [dict(nx=i.nx, ny=i.ny, nz=i.nz, tau=max(i.tau, floor), G=i.G, R0=i.R0,
                     lam=i.lam, eps=i.eps, phase=i.phase, rho_l=rho_l, rho_v=rho_v, width=i.width)
                for i in sweep]

    def unstable_after(floor):
        with L.Batch(insts(floor), precision=precision) as b:
            b.init()
            b.step(n_steps)
            bad = [k for k in range(len(sweep)) if b.diagnostics(k)["numeric_ok"] != 1]
            try:
                b.sync()
            except L.LbmError:
                pass
        return bad

    if args.no_tune:
        # profiling runs: the floor measured on GB300, no stability scan
        unstable_drawn, floor = None, 0.9
    else:
        unstable_drawn = unstable_after(0.0)
        floor = None
        for fl in (0.8, 0.9, 1.0):
            if not unstable_after(fl):
                floor = fl
                break
    if floor is None:
        return {"error": "no tau floor up to 1 keeps all 48 instances finite for %d steps" % n_steps,
                "unstable_at_drawn_tau": unstable_drawn}
    stable = insts(floor)
    total = sum(d["nx"] * d["ny"] * d["nz"] for d in stable)
    stream = torch.cuda.current_stream()
    with L.Batch(stable, precision=precision) as b:
        b.init()
        if args.no_tune:
            tuned = dict(fused=args.batch_fused, fused_fz=16, fused_group=0, block=[0, 0, 0], occupancy=0)
            per_elem = dict(fused=1, fused_fz=16, block=[0, 0, 0], occupancy=0)
            other = dict(fused=0, fused_fz=0, block=[128, 1, 1], occupancy=3)
        else:
            tuned = autotune.tune_batch(b, blocks=((256, 1, 1), (128, 1, 1)), occupancies=(2, 3, 4), steps=10)
            # the other step forms, for the record: the per-element single
            # pass (form 1, which the persistent launch uses) and the best
            # two-kernel shape
            per_elem = autotune.tune_batch(b, blocks=(), occupancies=(), steps=10, fused_forms=(1,))
            other = autotune.tune_batch(b, blocks=((256, 1, 1), (128, 1, 1)), occupancies=(2, 3, 4), steps=10,
                                        fused_runs=())
        autotune.apply_batch(b, tuned)

        def timed(fn):
            b.init()                       # each arm from the same initial state
            for _ in range(args.warmup):
                fn(LBM_PER_STEP)
            torch.cuda.synchronize()
            e0, e1 = _events(torch)
            e0.record(stream)
            for _ in range(args.steps):
                fn(LBM_PER_STEP)
            e1.record(stream)
            torch.cuda.synchronize()
            ok = all(b.diagnostics(k)["numeric_ok"] == 1 for k in range(len(stable)))
            try:
                b.sync()
            except L.LbmError:
                ok = False
            return e0.elapsed_time(e1), ok

        ms_b, ok_b = timed(b.step)
        ms_s, ok_s = timed(b.step_sequential)
        # the same form as one persistent cooperative launch per benchmark
        # step (10 lattice steps, grid barriers between them; the two-kernel
        # form has none: the per-element single pass stands in)
        if not tuned.get("fused"):
            autotune.apply_batch(b, per_elem)
        b.set_option("persistent", 1)
        ms_p, ok_p = timed(b.step)
        b.set_option("persistent", 0)
        # the per-element single pass, one launch per step
        autotune.apply_batch(b, per_elem)
        ms_e, ok_e = timed(b.step)
        autotune.apply_batch(b, other)
        ms_o, ok_o = timed(b.step)
    steps = args.steps * LBM_PER_STEP
    glups = lambda ms: total * steps / (ms * 1e-3) / 1e9
    value, seq, oth, elem, pers = glups(ms_b), glups(ms_s), glups(ms_o), glups(ms_e), glups(ms_p)
    peak, _ = peaks()
    bpl = FUSED_BYTES_PER_LU[precision] if tuned.get("fused") else STEP_BYTES_PER_LU[precision]
    forms = {0: "two-kernel", 1: "single-pass, per-element copies (one launch per step)",
             2: "single-pass, TMA on padded rows (one launch per step)"}
    return {"value": round(value, 4), "unit": UNIT, "ms_per_step": round(ms_b / args.steps, 4),
            "step_form": forms[int(tuned.get("fused", 0))],
            "sequential_value": round(seq, 4), "speedup_vs_sequential": round(value / seq, 3),
            "other_form_value": round(oth, 4), "other_form": other,
            "per_element_value": round(elem, 4), "per_element_form": per_elem,
            "persistent_value": round(pers, 4),
            "persistent_form": "the timed single-pass form, %d steps per cooperative launch of persistent "
                               "blocks with grid barriers between the steps" % LBM_PER_STEP,
            "total_nodes": total, "precision": precision, "tuned": tuned,
            "bytes_per_lu": bpl, "hbm_frac_step_model": round(value * bpl / peak, 4),
            "hbm_frac_floor_160": round(value * 160 / peak, 4),
            "numeric_ok_batched": ok_b and ok_o and ok_p and ok_e, "numeric_ok_sequential": ok_s,
            "sweep": "%d periodic ligaments, R0 in {8,12,16,20,24}, lambda/R0 in [4.5,12], eps=0.05, G=-6, "
                     "box lambda x 4R0 x 4R0, tau drawn in [0.6,1.0]" % len(sweep),
            "timed_tau_floor": floor,
            "unstable_at_drawn_tau": unstable_drawn,
            "mode": "one launch per step (single-pass) or one psi + one collide launch per step (two-kernel) for "
                    "all instances, graph replay, against 48 x 2 launches per step"}


def run_batch(args):
    import torch
    from paper_1904_11792_gb300 import autotune, build, lbm as L
    torch.cuda.set_device(dist_env()[2])
    build.build()
    L.load()
    rho_l, rho_v = (args.rho_l, args.rho_v) if (args.rho_l and args.rho_v) else \
        coexistence_densities(-6.0, 1.0)
    with Clocks(dist_env()[2]) as clk:
        r = batch_sweep(args, torch, L, autotune, rho_l, rho_v, args.precision)
    line = {
        "metric": METRIC, "value": r.get("value"), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r.get("ms_per_step"),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ligament sweep, no dataset)",
        "config": dict({"workload": "batched sweep: " + r.get("sweep", "")}, **{k: v for k, v in r.items()
                                                                        if k not in ("value", "unit")}),
        "clocks": clk.summary(),
        "gpu_launches": int(args.steps * LBM_PER_STEP * 2),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("grid1024", "grid256", "batch48"), default="grid1024",
                    help="grid1024: the 1024x512x512 ligament (268 M nodes), the headline; grid256: the "
                         "256x128x128 grid-convergence ligament; batch48: the batched sweep alone")
    ap.add_argument("--precision", choices=("f32", "f64", "f16dev", "bf16dev"), default="f32")
    ap.add_argument("--pattern", choices=("auto", "ab", "aa"), default="auto",
                    help="streaming pattern; auto = the autotuner's choice")
    ap.add_argument("--rho-l", type=float, default=None,
                    help="liquid density (with --rho-v: skip the flat-interface run)")
    ap.add_argument("--rho-v", type=float, default=None)
    ap.add_argument("--fused", action="store_true",
                    help="with --no-tune: the single-pass fused step (the autotuner otherwise chooses)")
    ap.add_argument("--fused-fz", type=int, default=0,
                    help="with --no-tune --fused: z planes per block (0 = automatic)")
    ap.add_argument("--fused-group", type=int, default=0,
                    help="with --no-tune --fused: z runs per group of the block order (0 = automatic)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (default launch configuration; profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the end-to-end and CPU-baseline legs (profiling runs)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP16/BF16/AA/batched comparisons (profiling runs)")
    ap.add_argument("--batch-fused", type=int, choices=(0, 1, 2), default=2,
                    help="with --no-tune: the batched step form timed first (2: TMA single pass on padded rows, "
                         "1: per-element single pass, 0: two kernels)")
    ap.add_argument("--batch-size", type=int, default=48,
                    help="batch48: the first K instances of the sweep (profiling runs on a smaller batch)")
    ap.add_argument("--nz", type=int, default=0,
                    help="grid workloads: the same lattice with this many z planes (counter captures on a few "
                         "GB whose traffic scales to the full lattice by the plane count); no traffic record "
                         "is reported for it")
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
