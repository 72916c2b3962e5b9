"""Autotuner of the time-step launch configuration.

For a lattice size and storage precision it times, on the GPU, the streaming
pattern (A-B or AA), the collide-stream block shape and the register budget
variant (blocks per SM) of the two-kernel step, and the single-pass fused step
where it applies, picks the fastest whole step, and caches the choice in a
JSON file keyed by device, size and precision.  For a batch it tunes the
batched kernel's block shape.  All timing is CUDA events around real steps of
the library (kernel_timing for per-kernel times).
"""
from __future__ import annotations

import json
import os
import time

from . import lbm as L

DEFAULT_BLOCKS = ((256, 1, 1), (128, 2, 1), (64, 4, 1), (32, 8, 1), (64, 2, 2), (32, 4, 2),
                  (128, 1, 2), (32, 2, 4))
DEFAULT_OCC = (2, 3, 4)


def cache_path() -> str:
    p = os.environ.get("LBM_TUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "lbm_gb300_tune.json")


def _load_cache() -> dict:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save_cache(c: dict) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(c, fh, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def _device_key() -> str:
    import torch
    return torch.cuda.get_device_name()


def _key(kind, dims, precision, extra="") -> str:
    return "%s|%s|%s|%s|%s" % (_device_key(), kind, "x".join(map(str, dims)), precision, extra)


def _fits(block, nx):
    return block[0] <= max(32, nx) * 2


def tune_lattice(nx, ny, nz, precision="f32", patterns=("ab", "aa"), blocks=DEFAULT_BLOCKS,
                 occupancies=DEFAULT_OCC, tau=1.0, G=-6.0, steps=20, use_cache=True,
                 verbose=False, fused_runs=(8, 12, 16, 24, 32), fused_groups=(1, 2, 4),
                 reps=3) -> dict:
    """Best (pattern, fused, block, occupancy) for one lattice; returns a dict
    with the choice and the measured per-step time (best of `reps` timings of
    `steps` steps) and GLUPS."""
    import torch
    key = _key("lattice", (nx, ny, nz), precision, ",".join(patterns))
    cache = _load_cache() if use_cache else {}
    if use_cache and key in cache:
        return cache[key]
    rl, rv = 2.6489, 0.0732
    N = nx * ny * nz
    best = None
    trials = []
    for pattern in patterns:
        with L.Lattice(nx, ny, nz, tau, G, precision=precision, pattern=pattern,
                       rho_ref=rv if precision.endswith("dev") else 0.0) as lat:
            lat.init_ligament(min(ny, nz) / 4.0, float(nx), 0.02, 0.0, rl, rv, 2.0)
            lat.set_option("fused", 1)
            # the GPU leaves its idle clocks during the first few milliseconds
            # of work: warm up before the first trial, and keep the best of
            # `reps` timings of each candidate
            lat.step(max(40, steps))
            torch.cuda.synchronize()
            if lat.get_option("fused"):
                for fz, grp in [(z, gr) for z in (0,) + tuple(z for z in fused_runs if z < nz)
                                for gr in (0,) + tuple(fused_groups)]:
                    lat.set_option("fused_fz", fz)
                    lat.set_option("fused_group", grp)
                    lat.step(4)
                    torch.cuda.synchronize()
                    step_ms = float("inf")
                    for _ in range(reps):
                        lat.set_option("kernel_timing", 1)
                        lat.step(steps)
                        n2, ms2 = L.lbm_kernel_time(lat.h, 2)
                        lat.set_option("kernel_timing", 0)
                        step_ms = min(step_ms, ms2 / max(n2, 1))
                    t = dict(pattern=pattern, fused=1, fused_fz=fz, fused_group=grp, block=[0, 0, 0], occupancy=0,
                             step_ms=step_ms, glups=N / (step_ms * 1e-3) / 1e9)
                    trials.append(t)
                    if verbose:
                        print(json.dumps(t))
                    if best is None or step_ms < best["step_ms"]:
                        best = t
                lat.set_option("fused_fz", 0)
                lat.set_option("fused_group", 0)
            lat.set_option("fused", 0)
            for occ in occupancies:
                for b in blocks:
                    if not _fits(b, nx):
                        continue
                    for k, v in zip(("block_x", "block_y", "block_z"), (1, 1, 1)):
                        lat.set_option(k, v)
                    for k, v in zip(("block_x", "block_y", "block_z"), b):
                        lat.set_option(k, v)
                    lat.set_option("occupancy", occ)
                    lat.step(4)
                    torch.cuda.synchronize()
                    step_ms = float("inf")
                    for _ in range(reps):
                        lat.set_option("kernel_timing", 1)
                        lat.step(steps)
                        n0, ms0 = L.lbm_kernel_time(lat.h, 0)
                        n1, ms1 = L.lbm_kernel_time(lat.h, 1)
                        lat.set_option("kernel_timing", 0)
                        step_ms = min(step_ms, ms0 / max(n0, 1) + ms1 / max(n1, 1))
                    t = dict(pattern=pattern, fused=0, block=list(b), occupancy=occ, step_ms=step_ms,
                             glups=N / (step_ms * 1e-3) / 1e9)
                    trials.append(t)
                    if verbose:
                        print(json.dumps(t))
                    if best is None or step_ms < best["step_ms"]:
                        best = t
    best = dict(best, trials=len(trials), tuned_at=time.strftime("%Y-%m-%dT%H:%M:%S"))
    if use_cache:
        cache = _load_cache()
        cache[key] = best
        _save_cache(cache)
    return best


def apply(lat: "L.Lattice", choice: dict) -> None:
    """Applies a tuned choice to a lattice: the fused step, or the two-kernel
    step with its block shape and occupancy (the pattern is fixed at
    creation: create the lattice with choice['pattern'])."""
    lat.set_option("fused", int(choice.get("fused", 0)))
    if choice.get("fused"):
        lat.set_option("fused_fz", int(choice.get("fused_fz", 0)))
        lat.set_option("fused_group", int(choice.get("fused_group", 0)))
        return
    for k, v in zip(("block_x", "block_y", "block_z"), (1, 1, 1)):
        lat.set_option(k, v)
    for k, v in zip(("block_x", "block_y", "block_z"), choice["block"]):
        lat.set_option(k, v)
    lat.set_option("occupancy", choice["occupancy"])


def tune_batch(batch: "L.Batch", blocks=((256, 1, 1), (128, 1, 1), (64, 1, 1)), occupancies=(2, 3, 4),
               steps=20, verbose=False, fused_runs=(8, 16, 32), fused_forms=(2, 1), tile_widths=(64, 32)) -> dict:
    """Times the batched step - the single-pass forms (2: TMA on padded
    rows, on tiles of each width in tile_widths, with z runs in groups of
    one or all of a tile's runs; 1: per-element copies) for each z run
    length, and the two-kernel form for each block size / occupancy - and
    leaves the batch configured with the fastest; returns the choice."""
    import torch
    best = None

    def timed():
        batch.step(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.step(steps)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    cands = [dict(fused=form, fused_fz=fz, fused_group=grp, tile_width=tw, block=[0, 0, 0], occupancy=0)
             for form in fused_forms for fz in fused_runs for grp in ((0, 1) if form == 2 else (0,))
             for tw in (tile_widths if form == 2 else (0,))]
    cands += [dict(fused=0, fused_fz=0, block=list(b), occupancy=occ) for occ in occupancies for b in blocks]
    for c in cands:
        apply_batch(batch, c)
        t = dict(c, step_ms=timed())
        if verbose:
            print(json.dumps(t))
        if best is None or t["step_ms"] < best["step_ms"]:
            best = t
    apply_batch(batch, best)
    return best


def apply_batch(batch: "L.Batch", choice: dict) -> None:
    """Applies a tuned batch choice (single-pass with its run length, or the
    two-kernel step with its block shape and occupancy)."""
    batch.set_option("fused", int(choice.get("fused", 0)))   # 0, 1 or 2
    if choice.get("fused"):
        batch.set_option("fused_fz", int(choice["fused_fz"]))
        batch.set_option("fused_group", int(choice.get("fused_group", 0)))
        batch.set_option("tile_width", int(choice.get("tile_width", 0)))
        return
    for k, v in zip(("block_x", "block_y", "block_z"), (1, 1, 1)):
        batch.set_option(k, v)
    for k, v in zip(("block_x", "block_y", "block_z"), choice["block"]):
        batch.set_option(k, v)
    batch.set_option("occupancy", choice["occupancy"])
