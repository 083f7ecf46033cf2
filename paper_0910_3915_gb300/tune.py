"""Schedule autotuner for the fused step kernel.

The step kernel's work split is a kernel variant (planes staged into shared
memory by TMA, or loaded from global memory by the compute threads), the
number of TMA stages, a tile height (4, 8 or 16 rows of 32 nodes per CTA)
and a number of z segments per tile column. None of them changes a single
value of the result (the kernel is bitwise schedule-independent); they only
change occupancy, halo overhead and wave balance. ``tune`` times candidate
schedules on the lattice itself with CUDA events, restores the lattice state
afterwards (checkpoint round-trip), applies the fastest schedule and returns
the table of timings.
"""
from __future__ import annotations

import json
import os

SEGMENTS = (1, 2, 4, 8, 16)
TMA_PAIRS = ((4, 2), (4, 3), (8, 2), (8, 3), (16, 2))  # (tile height, stages)
LDG_TILES = (4, 8)


def candidates(nz_fluid: int, precision: str, segments=SEGMENTS):
    out = []
    for ty, ns in TMA_PAIRS:
        if ty == 16 and precision == "f32":
            continue  # two FP32 stages of 18 rows exceed shared memory
        out += [("tma", ns, ty, s) for s in segments if nz_fluid // s >= 4]
    for ty in LDG_TILES:
        out += [("ldg", 0, ty, s) for s in segments if nz_fluid // s >= 4]
    return out


def apply(lat, cand):
    variant, stages, ty, seg = cand
    lat.set_step_variant(variant, stages).set_schedule(ty, seg)


def tune(lat, steps: int = 64, segments=SEGMENTS, cache: str | None = None):
    """Pick the fastest (variant, stages, tile_y, z_segments) for ``lat``; returns (best, table)."""
    import torch

    key = f"{lat.precision}:{lat.nx}x{lat.ny}x{lat.nz}:{torch.cuda.get_device_name()}"
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            best = tuple(table[key]["best"])
            apply(lat, best)
            return best, table[key]["ms"]
    state = lat.save()
    stream = torch.cuda.current_stream()
    timings = {}
    for cand in candidates(lat.nz - 2, lat.precision, segments):
        apply(lat, cand)
        lat.step(steps)  # warm-up, graph capture
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        lat.sync()
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        e1.synchronize()
        timings["%s:%d:%d:%d" % cand] = e0.elapsed_time(e1) / steps
    lat.load(state)
    best_key = min(timings, key=timings.get)
    v, ns, ty, seg = best_key.split(":")
    best = (v, int(ns), int(ty), int(seg))
    apply(lat, best)
    if cache:
        table = {}
        if os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        table[key] = {"best": list(best), "ms": timings}
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return best, timings
