"""Schedule autotuner for the fused step kernel.

The step kernel's work split is a tile height (4, 8 or 16 rows of 32 nodes
per CTA) and a number of z segments per tile column. Neither changes a
single value of the result (the kernel is bitwise schedule-independent);
they only change occupancy, halo overhead and wave balance. ``tune`` times
candidate schedules on the lattice itself with CUDA events, restores the
lattice state afterwards (checkpoint round-trip), applies the fastest
schedule and returns the table of timings.
"""
from __future__ import annotations

import json
import os

DEFAULT_TILES = (4, 8, 16)
DEFAULT_SEGMENTS = (1, 2, 3, 4, 6, 8, 12, 16)


def candidates(nz_fluid: int, tiles=DEFAULT_TILES, segments=DEFAULT_SEGMENTS):
    return [(t, s) for t in tiles for s in segments if nz_fluid // s >= 4]


def tune(lat, steps: int = 64, tiles=DEFAULT_TILES, segments=DEFAULT_SEGMENTS, cache: str | None = None):
    """Pick the fastest (tile_y, z_segments) for ``lat``; returns (best, table)."""
    import torch

    key = f"{lat.precision}:{lat.nx}x{lat.ny}x{lat.nz}:{torch.cuda.get_device_name()}"
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            best = tuple(table[key]["best"])
            lat.set_schedule(*best)
            return best, table[key]["ms"]
    state = lat.save()
    stream = torch.cuda.current_stream()
    timings = {}
    for ty, seg in candidates(lat.nz - 2, tiles, segments):
        lat.set_schedule(ty, seg)
        lat.step(steps)  # warm-up, graph capture
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        lat.sync()
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        e1.synchronize()
        timings[f"{ty}x{seg}"] = e0.elapsed_time(e1) / steps
    lat.load(state)
    best_key = min(timings, key=timings.get)
    best = tuple(int(v) for v in best_key.split("x"))
    lat.set_schedule(*best)
    if cache:
        table = {}
        if os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        table[key] = {"best": list(best), "ms": timings}
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return best, timings
