#!/usr/bin/env python
"""Throughput of the two-component Shan-Chen D3Q19 step on one GB300 (or N, as replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload single|precision-f16|precision-bf16|small]

One bench "step" is one lattice time step of the whole hot path: moments,
psi, Shan-Chen and wall force, force-shifted cubic BGK and streaming with
mid-grid bounce-back (one fused kernel launch). The timed region also holds
the FP64 conservation reductions every 1000 steps and one contact-angle
measurement at the end. Default workload: the 128^3 droplet (R = 30, FP32,
g_br = 0.08, W36 weights with force scale 1.25, wall parameter 0.05).

Prints ONE JSON line (rank 0). MLUPS counts fluid-node updates per second.
Under torchrun each rank runs its own lattice (independent replicas, weak
scaling, no data-path collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline (FP32 / BF16-stored vs FP64 oracle, contact-angle err in deg)"
CONTACT = dict(g_br=0.08, force_weights=1, force_scale=1.25)
WORKLOADS = {
    "single": dict(dims=(128, 128, 128), radius=30.0, precision="f32", w=0.05),
    "precision-f16": dict(dims=(256, 256, 128), radius=60.0, precision="f16", w=0.05),
    "precision-bf16": dict(dims=(256, 256, 128), radius=60.0, precision="bf16", w=0.05),
    "small": dict(dims=(32, 32, 32), radius=8.0, precision="f32", w=0.05),
    # 64 cubic boxes, edges from {48, 64, 80, 96}, R = 0.3 edge, per-box g_br and wall value
    "sweep": dict(boxes=64, seed=3, precision="f32"),
    # 11 wall values in [-0.1, 0.1] on the 128^3 droplet, 20000 steps, as one batch
    "angles": dict(dims=(128, 128, 128), radius=30.0, precision="f32", steps=20000,
                   w=[round(-0.1 + 0.02 * i, 3) for i in range(11)]),
    # size convergence: cubic lattices of edge 32 .. 256 with the droplet scaled with the box (R = 0.234 L,
    # the 128^3 droplet's ratio), three wall values, the same fixed step count for every size
    # z-slab decomposition with a halo exchange every step. One process: the 128^3 droplet as 2 slabs on one
    # GPU (the exchange's cost against the single lattice). Under torchrun: one slab of 126 fluid planes per
    # rank, a 128 x 128 x (126 N + 2) lattice with the droplet on its bottom wall (NCCL messages, weak scaling)
    "slabs": dict(dims=(128, 128, 128), radius=30.0, precision="f32", w=0.05, nslab=2, schedule=(4, 38, 4)),
    "sizes": dict(edges=(32, 64, 128, 256), radius_frac=30.0 / 128.0, precision="f32", steps=20000,
                  w=(0.03, 0.06, 0.09)),
    # the paper's own parameter set (Sec. 4): g = 0.16, W36 weights at force scale 1, a one-sided wall
    # (eta_wall_r, eta_wall_b) = (0, eta) with eta = 0.1 / 0.2 / 0.3, drops of initial volume 70^3 in 128^3
    # and 141^3 in 256^3 (hemispheres of that volume on the wall), the same step count for both sizes
    "sizes-paper": dict(edges=(128, 256), drop_edge={128: 70, 256: 141}, precision="f32", steps=20000,
                        w=(0.1, 0.2, 0.3), prm=dict(g_br=0.16, force_weights=1, force_scale=1.0),
                        wall="one-sided"),
    # adjoint calibration: 64^3, R = 16, 2000 steps, checkpoints every 100
    "adjoint": dict(dims=(64, 64, 64), radius=16.0, precision="f32", steps=2000, ckpt=100),
    # surface tensions (Sec. 4.1-4.2): 8x8x128 periodic lamellae (gamma_LG), 8x8x(64+2) slabs of each
    # phase between the walls (gamma_SL, gamma_SG), a free droplet (radial gamma_LG) and sessile
    # droplets (geometric, Huang and radial-Young angles), 11 wall values in [-0.1, 0.1]
    "young": dict(lamella=(8, 8, 128), slab=(8, 8, 66), free=(64, 64, 64), free_radius=16.0,
                  sessile=(96, 96, 96), sessile_radius=24.0, steps=10000, sessile_steps=8000,
                  w=[round(-0.1 + 0.02 * i, 3) for i in range(11)]),
}
BYTES_PER_LU = {"f32": 304, "f16": 152, "bf16": 152}
CONS_EVERY = 1000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="single")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-samples", action="store_true",
                    help="default workload: skip the 16-bit storage and batched-sweep throughput samples")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="precision workloads: skip the accuracy runs against FP32 and the oracle")
    ap.add_argument("--schedule", default=None,
                    help="fixed step schedule variant:stages:tile_y:z_segments[:y_tiles] (e.g. ldg:0:8:4:19); "
                         "for --workload sweep variant:tile_y:planes_per_item (e.g. tma:4:16); skips tuning")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


STEP_SOURCES = ("step.cu", "step_common.cuh", "lb_internal.cuh", "step_tma.cuh", "api.cu")  # api.cu: the layout


def step_source_sha256() -> str:
    """sha256 over the step kernel's sources (the files its code comes from)."""
    h = hashlib.sha256()
    for name in STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_0910_3915_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def step_kernel_traffic(workload: str, schedule: str | None):
    """(per-launch DRAM bytes of the step kernel, the schedule they were taken
    under) from the committed ncu summary: `schedule` itself, else a recorded
    schedule of the same variant, stages and tile height (the z segments and
    y-tiles move the bytes by the few halo planes only); (None, None) when the
    kernel's sources changed since it was taken or nothing close was captured."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("step_sources_sha256") != step_source_sha256() or not schedule:
            return None, None
        table = rec.get("bytes_per_launch", {})
        if f"{workload} {schedule}" in table:
            return table[f"{workload} {schedule}"], schedule
        family = ":".join(schedule.split(":")[:3])
        for key, val in sorted(table.items()):
            wl, sched = key.split(" ", 1)
            if wl == workload and ":".join(sched.split(":")[:3]) == family:
                return val, sched
        return None, None
    except Exception:
        return None, None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", device_id, f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_mlups(dims, radius, w, seconds: float):
    """The FP64 oracle on the same workload, a bounded number of steps."""
    import oracle
    from paper_0910_3915_gb300 import workloads as W
    nx, ny, nz = dims
    rr, rb = W.droplet_fields(nx, ny, nz, radius, seed=0)
    er, eb = W.wall_split(w)
    st = oracle.State(rr, rb, W.wall_mask(nx, ny, nz), oracle.Params(**CONTACT, eta_wall_r=er, eta_wall_b=eb))
    t = time.perf_counter()
    st.step(1)
    one = time.perf_counter() - t
    n = max(1, min(1000, int(seconds / max(one, 1e-6))))
    t = time.perf_counter()
    st.step(n)
    el = time.perf_counter() - t
    nf = nx * ny * (nz - 2)
    return nf * n / el / 1e6, n, el


def oracle_mlups_one_core(dims, radius, w, seconds: float):
    """oracle_mlups with one OpenMP thread (a child process: the thread count is
    fixed when the oracle library starts)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_mlups(%r, %r, %r, %r)))" % (ROOT, tuple(dims), radius, w, seconds))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def run_reference(args):
    from paper_0910_3915_gb300 import replicas

    ws, rank, _ = replicas.world()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    nx, ny, nz = wl["dims"]
    # A full-lattice oracle step takes a sizeable fraction of a second, so the K requested steps
    # are represented by a bounded sample: as many full-lattice oracle steps as fit in about a
    # minute (after one untimed step), timed as a whole; throughput is per lattice update either way.
    mlups, n, el = oracle_mlups(wl["dims"], wl["radius"], wl["w"], seconds=60.0)
    cores = omp_threads()
    sample = (f"{nx}x{ny}x{nz} droplet: {n} full-lattice oracle steps timed ({el:.1f} s, after 1 untimed step) "
              f"stand in for the {args.steps} requested steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / n * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"droplet {nx}x{ny}x{nz} R={wl['radius']:g} (FP64 CPU oracle)"},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_0910_3915_gb300 import lbsc, tune
    from paper_0910_3915_gb300 import workloads as W

    from paper_0910_3915_gb300 import replicas

    ws, rank, local = replicas.world()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.workload]
    nx, ny, nz = wl["dims"]
    prec = wl["precision"]
    nf = nx * ny * (nz - 2)
    er, eb = W.wall_split(wl["w"])
    prm = dict(CONTACT, eta_wall_r=er, eta_wall_b=eb)
    rr, rb = W.droplet_fields(nx, ny, nz, wl["radius"], seed=rank)
    stream = torch.cuda.current_stream()
    K, Wm = args.steps, max(3, args.warmup)

    lat = lbsc.Lattice(rr, rb, prec).set_params(**prm)
    cons_load = lat.conservation()
    schedule = None
    if args.schedule:
        schedule = tune.parse(args.schedule)
        tune.apply(lat, schedule)
    elif not args.no_tune:
        schedule, _ = tune.tune(lat)
    lat.step(Wm)
    lat.measure(5.0)  # warm-up of the measurement kernels too (their first launch loads them)
    lat.sync()

    try:
        dev_id = str(torch.cuda.get_device_properties(local).uuid)
        dev_id = dev_id if dev_id.startswith("GPU-") else "GPU-" + dev_id
    except Exception:
        dev_id = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
    sampler = ClockSampler(dev_id)
    time.sleep(0.3)
    replicas.barrier()
    torch.cuda.synchronize()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    t0, t1 = ev(), ev()
    chunks = []
    launches = 0
    t0.record(stream)
    done = 0
    while done < K:
        m = min(CONS_EVERY, K - done)
        a, b = ev(), ev()
        a.record(stream)
        lat.step(m)
        b.record(stream)
        chunks.append((a, b))
        launches += m
        done += m
        if done < K:
            lat.conservation()  # one kernel
            launches += 1
    # the last conservation sums and the contact angle in one pass over the populations
    cons_end, angle = lat.measure(5.0)  # conservation (with phi), angle and finish kernels
    launches += 3
    t1.record(stream)
    torch.cuda.synchronize()
    replicas.barrier()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    step_ms = sum(a.elapsed_time(b) for a, b in chunks) / K
    units, secs = replicas.whole_job(nf * K, ms * 1e-3, device="cuda")  # all ranks' updates, slowest rank
    ms = secs * 1e3
    value = units / secs / 1e6
    cons = lat.conservation()
    lat.close()

    # End to end through the C ABI with host buffers. The context is allocated before the timed region
    # (the allocation is not a copy); timed are: the initial densities from pinned host memory into it
    # (lb_reset: host-to-device copy, initialisation kernel and its input check), the same steps and
    # reductions as above, and the results back on the host (the conservation sums and the contact angle).
    rr_p = torch.from_numpy(rr).pin_memory().numpy()
    rb_p = torch.from_numpy(rb).pin_memory().numpy()
    lat2 = lbsc.Lattice(rr, rb, prec).set_params(**prm)
    if schedule:
        tune.apply(lat2, schedule)
    lat2.step(Wm)
    lat2.measure(5.0)
    torch.cuda.synchronize()
    replicas.barrier()
    te = time.perf_counter()
    lat2.reset(rr_p, rb_p)
    done, n_cons = 0, 0
    while done < K:
        m = min(CONS_EVERY, K - done)
        lat2.step(m)
        done += m
        n_cons += 1
        if done < K:
            lat2.conservation()
    lat2.measure(5.0)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - te
    lat2.close()
    h2d = 2 * rr.size * 8
    d2h = n_cons * 8 * 8 + 19 * 8
    e_units, e_secs = replicas.whole_job(nf * K, e2e_s, device="cuda")
    e2e = e_units / e_secs / 1e6

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, peak_kind = peaks()
    bpl = BYTES_PER_LU[prec]
    achieved = nf * bpl / (step_ms * 1e-3) / 1e9
    traffic, traffic_sched = step_kernel_traffic(args.workload, tune.name(schedule) if schedule else None)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": traffic,
            "traffic_schedule": traffic_sched,
            "peak_source": peak_kind,
            "kernel": "step_tma_kernel" if schedule and schedule[0] == "tma" else "step_kernel",
            "algorithmic_bytes_per_launch": nf * bpl}
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        c_mlups, c_n, c_el = oracle_mlups(wl["dims"], wl["radius"], wl["w"], seconds=15.0)
        cpu = {"value": round(c_mlups, 3), "unit": "MLUPS", "cores": omp_threads(), "kind": "oracle",
               "sample": f"{nx}x{ny}x{nz} droplet, {c_n} oracle steps ({c_el:.1f} s)"}
        one = oracle_mlups_one_core(wl["dims"], wl["radius"], wl["w"], seconds=8.0)
        if one:
            cpu["one_core"] = {"value": round(one[0], 3), "unit": "MLUPS", "cores": 1,
                               "sample": f"{one[1]} oracle steps ({one[2]:.1f} s)"}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws, "steps": K, "warmup": Wm,
        "ms_per_step": round(ms / K, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": prec, "data": "synthetic",
        "config": {"workload": f"droplet {nx}x{ny}x{nz} R={wl['radius']:g} {prec.upper()}",
                   "lattice": [nx, ny, nz], "fluid_nodes": nf, "params": prm,
                   "schedule": ({"variant": schedule[0], "stages": schedule[1], "tile": f"32x{schedule[2]}",
                                 "z_segments": schedule[3],
                                 "y_tiles": schedule[4] or -(-ny // schedule[2])} if schedule else "default"),
                   "l2": "inputs larger than L2 (state %.0f MB, L2 129 MB)" % (nx * ny * nz * bpl / 1e6),
                   "timed": f"{K} steps + FP64 conservation every {CONS_EVERY} + 1 contact angle "
                            "(the last sums and the angle in one pass)"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e, 1), "unit": "MLUPS", "h2d_bytes_per_step": round(h2d / K, 1),
                "d2h_bytes_per_step": round(d2h / K, 1)},
        "gpu_launches": launches,
        "clocks": clocks,
        "step_kernel_ms": round(step_ms, 5),
        "theta_deg": round(angle["theta_deg"], 3) if angle["ok"] else None,
        "mass_rel_drift": None,
    }
    # drift over every step taken (tuning, warm-up, timed), against the stored state after loading;
    # the rounding of the FP64 input densities into the storage format is reported separately
    m0 = float(rr[1:-1].sum()), float(rb[1:-1].sum())
    line["mass_rel_drift"] = [float(cons[k] / cons_load[k] - 1) for k in (0, 1)]
    line["load_mass_rel_err"] = [float(cons_load[k] / m0[k] - 1) for k in (0, 1)]
    if args.workload.startswith("precision") and ws == 1 and not args.no_accuracy:
        line["accuracy"] = precision_accuracy(prec, 10000)
    if args.workload == "single" and not args.no_samples:
        line["samples"] = throughput_samples(K, Wm, peak)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_sweep(args):
    """Batched parameter sweep: all boxes in one persistent launch per step
    (graph-captured), against the same boxes stepped one after another."""
    import torch

    from paper_0910_3915_gb300 import lbsc
    from paper_0910_3915_gb300 import workloads as W

    from paper_0910_3915_gb300 import replicas

    ws, rank, local = replicas.world()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = WORKLOADS["sweep"]
    all_boxes = W.sweep_boxes(wl["boxes"], seed=wl["seed"])
    # under torchrun each rank advances its round-robin share of the boxes (no data-path exchange)
    idx = replicas.shard(range(len(all_boxes)), rank, ws)
    boxes = [all_boxes[i] for i in idx]
    fields, params = [], []
    for bx in boxes:
        fields.append(W.droplet_fields(bx.edge, bx.edge, bx.edge, bx.radius, seed=bx.seed))
        er, eb = W.wall_split(bx.w)
        params.append(lbsc.Params(g_br=bx.g_br, eta_wall_r=er, eta_wall_b=eb, force_weights=1, force_scale=1.25))
    nf = sum(bx.edge * bx.edge * (bx.edge - 2) for bx in boxes)
    K, Wm = args.steps, max(3, args.warmup)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    from paper_0910_3915_gb300 import tune

    batch = lbsc.Batch(fields, params, wl["precision"])
    if args.schedule:  # 'variant:tile_y:planes_per_item', e.g. tma:4:16
        v, ty, planes = args.schedule.split(":")
        best = (v, int(ty), int(planes))
        batch.set_step_variant(v).set_schedule(best[1], best[2])
    else:
        best, _ = tune.tune_batch(batch)
    batch.step(Wm)
    torch.cuda.synchronize()
    replicas.barrier()
    t0, t1 = ev(), ev()
    t0.record(stream)
    batch.step(K)
    t1.record(stream)
    torch.cuda.synchronize()
    replicas.barrier()
    units, secs = replicas.whole_job(nf * K, t0.elapsed_time(t1) * 1e-3, device="cuda")
    ms_batch = secs * 1e3
    angles = batch.contact_angles(5.0)
    batch.close()

    lats = [lbsc.Lattice(rr, rb, wl["precision"]).set_params(p) for (rr, rb), p in zip(fields, params)]
    for lat in lats:
        lat.step(Wm)
    torch.cuda.synchronize()
    replicas.barrier()
    t0.record(stream)
    for lat in lats:
        lat.step(K)
    t1.record(stream)
    torch.cuda.synchronize()
    replicas.barrier()
    _, seq_secs = replicas.whole_job(nf * K, t0.elapsed_time(t1) * 1e-3, device="cuda")
    ms_seq = seq_secs * 1e3
    for lat in lats:
        lat.close()
    if dist:
        got = [None] * ws
        dist.all_gather_object(got, (idx, angles))
        order = {}
        for ix, an in got:
            order.update(zip(ix, an))
        angles = [order[i] for i in range(len(all_boxes))]
        dist.destroy_process_group()
    boxes = all_boxes
    nf = sum(bx.edge * bx.edge * (bx.edge - 2) for bx in boxes)
    if rank != 0:
        return
    value = units / secs / 1e6
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws, "steps": K, "warmup": Wm,
        "ms_per_step": round(ms_batch / K, 5), "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": wl["precision"], "data": "synthetic",
        "config": {"workload": f"batched sweep: {len(boxes)} cubic boxes, edges from 48/64/80/96, R = 0.3 edge"
                               + (f", round-robin over {ws} ranks" if ws > 1 else ""),
                   "fluid_nodes": nf,
                   "schedule": {"variant": best[0], "tile": f"32x{best[1]}", "planes_per_item": best[2]},
                   "l2": "inputs larger than L2"},
        "sequential_mlups": round(nf * K / (ms_seq * 1e-3) / 1e6, 1),
        "speedup_vs_sequential": round(ms_seq / ms_batch, 3),
        "roofline": {"bound": "hbm", "achieved": round(nf * 304 / (ms_batch / K * 1e-3) / 1e9 / ws, 1),
                     "peak": peaks()[0], "unit": "GB/s",
                     "frac": round(nf * 304 / (ms_batch / K * 1e-3) / 1e9 / ws / peaks()[0], 4),
                     "note": "per GPU" if ws > 1 else None,
                     "kernel": "batch_tma_kernel" if best[0] == "tma" else "batch_step_kernel"},
        "theta_deg": [round(a["theta_deg"], 2) if a["ok"] else None for a in angles],
        "droplets": droplet_validity(boxes, angles),
    }
    print(json.dumps(line), flush=True)


# a measured droplet whose phase contrast max(rho_r - rho_b) fell below this (from 0.66 initially) is a
# diffuse, partly dissolved drop: its angle is reported but flagged
CONTRAST_MIN = 0.3


def droplet_validity(boxes, angles):
    """Per-box validity of the sweep's angles: the library's status (why an angle
    is missing) and a contrast check, with each invalid box's parameters."""
    from paper_0910_3915_gb300 import lbsc
    bad = []
    for i, (bx, a) in enumerate(zip(boxes, angles)):
        reason = None
        if a["status"] != lbsc.LB_DROP_OK:
            reason = lbsc.DROP_STATUS.get(a["status"], "status %d" % a["status"])
        elif a["phi_max"] < CONTRAST_MIN:
            reason = "diffuse: max(rho_r - rho_b) = %.3f < %.2f" % (a["phi_max"], CONTRAST_MIN)
        if reason:
            bad.append({"box": i, "edge": bx.edge, "g_br": round(bx.g_br, 4), "w": round(bx.w, 4), "reason": reason,
                        "phi_max": round(a["phi_max"], 4),
                        "theta_deg": round(a["theta_deg"], 2) if a["ok"] else None})
    return {"valid": len(boxes) - len(bad), "total": len(boxes), "contrast_min": CONTRAST_MIN, "invalid": bad}


def run_slabs(args):
    """The lattice split into z slabs, one exchange of face messages per step."""
    import torch

    from paper_0910_3915_gb300 import lbsc, replicas, slabs
    from paper_0910_3915_gb300 import workloads as W

    ws, rank, local = replicas.world()
    torch.cuda.set_device(local)
    dist = None
    wl = WORKLOADS["slabs"]
    nx, ny, nz = wl["dims"]
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        nz = (nz - 2) * ws + 2
    prec = wl["precision"]
    nf = nx * ny * (nz - 2)
    er, eb = W.wall_split(wl["w"])
    prm = dict(CONTACT, eta_wall_r=er, eta_wall_b=eb)
    rr, rb = W.droplet_fields(nx, ny, nz, wl["radius"], seed=0)
    K, Wm = args.steps, max(3, args.warmup)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ty, nty, seg = wl["schedule"]
    if ws == 1:
        dec = slabs.Slabs(rr, rb, wl["nslab"], prec).set_params(**prm).set_tiling(ty, nty, seg)
    else:
        dec = slabs.DistributedSlab(rr, rb, prec).set_params(**prm)
        dec.lat.set_tiling(ty, nty, seg)
    dec.step(Wm)
    torch.cuda.synchronize()
    replicas.barrier()
    t0, t1 = ev(), ev()
    t0.record(stream)
    dec.step(K)
    t1.record(stream)
    torch.cuda.synchronize()
    replicas.barrier()
    units, secs = replicas.whole_job(nx * ny * (dec.bounds[rank][1] - dec.bounds[rank][0]) * K if ws > 1 else nf * K,
                                     t0.elapsed_time(t1) * 1e-3, device="cuda")
    cons = dec.conservation()
    single = None
    if ws == 1:
        dec.close()
        lat = lbsc.Lattice(rr, rb, prec).set_params(**prm).set_tiling(ty, nty, seg)
        lat.step(Wm)
        torch.cuda.synchronize()
        t0.record(stream)
        lat.step(K)
        t1.record(stream)
        torch.cuda.synchronize()
        single = nf * K / (t0.elapsed_time(t1) * 1e-3) / 1e6
        lat.close()
    else:
        dec.close()
        dist.destroy_process_group()
    if rank != 0:
        return
    value = units / secs / 1e6
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws, "steps": K, "warmup": Wm,
        "ms_per_step": round(secs * 1e3 / K, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": prec, "data": "synthetic",
        "config": {"workload": f"droplet {nx}x{ny}x{nz} R={wl['radius']:g} {prec.upper()} in "
                               f"{wl['nslab'] if ws == 1 else ws} z slabs" + (" on one GPU" if ws == 1 else ", one per GPU"),
                   "lattice": [nx, ny, nz], "fluid_nodes": nf,
                   "schedule": {"tile": f"32x{ty}", "y_tiles": nty, "z_segments": seg},
                   "exchange": "lattice to lattice (lb_halo_exchange)" if ws == 1 else "NCCL send/recv of face messages"},
        "mass": [float(cons[0]), float(cons[1])],
    }
    if single is not None:
        line["single_lattice_mlups"] = round(single, 1)
        line["vs_single_lattice"] = round(value / single, 4)
    print(json.dumps(line), flush=True)


def cap_centroid_height(volume: float, theta_deg: float) -> float:
    """Height above its base of the centroid of a spherical cap of the given
    volume and contact angle: V = pi R^3 (1 - c)^2 (2 + c) / 3, h = R (1 - c),
    centroid 3 (2R - h)^2 / (4 (3R - h)) from the sphere centre, c = cos theta."""
    c = math.cos(math.radians(theta_deg))
    R = (3.0 * volume / (math.pi * (1 - c) ** 2 * (2 + c))) ** (1.0 / 3.0)
    h = R * (1 - c)
    return 3.0 * (2 * R - h) ** 2 / (4.0 * (3 * R - h)) - (R - h)


def run_adjoint(args):
    """Adjoint throughput, a check against finite differences of the same
    observable, and calibration of the wall parameter to target contact angles."""
    import numpy as np
    import torch

    from paper_0910_3915_gb300 import lbsc
    from paper_0910_3915_gb300 import workloads as W

    torch.cuda.set_device(0)
    wl = WORKLOADS["adjoint"]
    nx, ny, nz = wl["dims"]
    T, ck = wl["steps"], wl["ckpt"]
    nf = nx * ny * (nz - 2)
    rr, rb = W.droplet_fields(nx, ny, nz, wl["radius"], seed=0)
    lat = lbsc.Lattice(rr, rb, wl["precision"]).set_params(**CONTACT)
    s0 = lat.save()
    lat.step_backward(10, ck)  # warm-up
    lat.load(s0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    J0, g0 = lat.step_backward(T, ck)
    adj_s = time.perf_counter() - t
    lat.load(s0)
    t = time.perf_counter()
    lat.step(T)
    lat.sync()
    fwd_s = time.perf_counter() - t

    # central differences of the same observable on the GPU (FP32, h = 1e-2), 200 steps; the
    # check against FP64 oracle differences is a test (tests/test_gpu_adjoint.py)
    Tc, h = 200, 1e-2
    lat.load(s0)
    Jc, gc = lat.step_backward(Tc, ck)

    def gJ(prm):
        lat.load(s0)
        lat.set_params(**prm)
        lat.step(Tc)
        return lat.observable("com_soft")

    fd = []
    for comp in ("eta_wall_r", "eta_wall_b"):
        jp = gJ(dict(CONTACT, **{comp: h}))
        jm = gJ(dict(CONTACT, **{comp: -h}))
        fd.append((jp - jm) / (2 * h))
    lat.set_params(**CONTACT)
    fd_err = float(np.max(np.abs(np.array(gc) - fd)) / np.max(np.abs(fd)))

    # calibration: Newton steps on J(w) = J*(theta*) with dJ/dw from the adjoint
    lat.load(s0)
    lat.step(T)
    r, b, _, _ = lat.moments()
    vol = float((1.0 / (1.0 + np.exp(-(r - b) / 0.05)))[1:-1].sum())
    calib = []
    for target in (60.0, 90.0, 120.0):
        Jt = cap_centroid_height(vol, target)
        w, hist = 0.0, []
        for _ in range(6):
            lat.load(s0)
            lat.set_params(**CONTACT, eta_wall_r=-w, eta_wall_b=w)
            J, g = lat.step_backward(T, ck)
            dJdw = g[1] - g[0]
            hist.append((round(w, 5), round(J, 4)))
            if abs(J - Jt) < 1e-3 or dJdw == 0:
                break
            w = float(np.clip(w - (J - Jt) / dJdw, -0.15, 0.15))
        lat.load(s0)
        lat.set_params(**CONTACT, eta_wall_r=-w, eta_wall_b=w)
        lat.step(T)
        ca = lat.contact_angle(5.0)
        calib.append({"theta_target": target, "J_target": round(Jt, 4), "w": round(w, 5),
                      "theta_measured": round(ca["theta_deg"], 2) if ca["ok"] else None,
                      "theta_fit": round(ca["theta_fit_deg"], 2), "iterations": hist})
    lat.close()
    line = {
        "metric": METRIC, "value": round(nf * T / adj_s / 1e6, 1), "unit": "MLUPS",
        "n_gpus": 1, "steps": T, "warmup": 1, "ms_per_step": round(adj_s / T * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl["precision"], "data": "synthetic",
        "config": {"workload": f"adjoint calibration: droplet {nx}^3 R={wl['radius']:g}, {T} steps, checkpoint every {ck}",
                   "observable": "soft droplet centre height, sigma(phi/0.05) weights"},
        "adjoint_seconds": round(adj_s, 3), "forward_seconds": round(fwd_s, 3),
        "adjoint_over_forward": round(adj_s / fwd_s, 2),
        "gradient": [float(g0[0]), float(g0[1])], "J": J0,
        "fd_check": {"steps": Tc, "h": h, "adjoint": [float(gc[0]), float(gc[1])], "gpu_fd": fd,
                     "max_rel_err": fd_err},
        "calibration": calib,
    }
    print(json.dumps(line), flush=True)


def bulk_densities(rr, rb):
    """Bulk r density inside the drop and outside (medians over the cores of each phase)."""
    import numpy as np
    phi = (rr - rb)[1:-1]
    r = rr[1:-1]
    inside = r[phi > 0.8 * phi.max()]
    outside = r[phi < 0.8 * phi.min()]
    return float(np.median(inside)), float(np.median(outside))


def run_angles(args):
    """Contact angle against the wall parameter on the 128^3 droplet (Sec. 4, Fig. 4 right):
    geometric theta, sphere-fit theta, the half-max |phi| interfaces as error bars, and
    Huang's closed-form estimate (Eq. huangSigmaLG) for comparison."""
    import torch

    from paper_0910_3915_gb300 import lbsc
    from paper_0910_3915_gb300 import workloads as W

    torch.cuda.set_device(0)
    wl = WORKLOADS["angles"]
    nx, ny, nz = wl["dims"]
    T = args.steps if args.steps != 20000 else wl["steps"]
    ws = wl["w"]
    fields = [W.droplet_fields(nx, ny, nz, wl["radius"], seed=0) for _ in ws]
    params = [lbsc.Params(**CONTACT, eta_wall_r=W.wall_split(w)[0], eta_wall_b=W.wall_split(w)[1]) for w in ws]
    batch = lbsc.Batch(fields, params, wl["precision"])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch.step(64)
    torch.cuda.synchronize()
    e0.record(stream)
    batch.step(T - 64)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nf = nx * ny * (nz - 2) * len(ws)
    rows = []
    for i, w in enumerate(ws):
        box = batch.box(i)
        rr, rb, _, cons = box.moments()
        phi = rr - rb
        a0 = box.contact_angle(5.0)
        hi = box.contact_angle(5.0, level=0.5 * float(phi[1:-1].max()))
        lo = box.contact_angle(5.0, level=0.5 * float(phi[1:-1].min()))
        r_in, r_out = bulk_densities(rr, rb)
        # Huang's closed form (Eq. huangSigmaLG) with the measured bulk densities
        th_h = lbsc.huang_theta(W.wall_split(w)[0], W.wall_split(w)[1], r_in, r_out)
        rows.append({"w": w, "theta": round(a0["theta_deg"], 2) if a0["ok"] else None,
                     "theta_fit": round(a0["theta_fit_deg"], 2),
                     "theta_halfmax": [round(hi["theta_deg"], 2) if hi["ok"] else None,
                                       round(lo["theta_deg"], 2) if lo["ok"] else None],
                     "huang": round(th_h, 2), "rho_in": round(r_in, 4), "rho_out": round(r_out, 4),
                     "h": round(a0["h"], 2), "b": round(a0["b"], 2)})
    batch.close()
    line = {
        "metric": METRIC, "value": round(nf * (T - 64) / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "n_gpus": 1,
        "steps": T, "warmup": 64, "ms_per_step": round(ms / (T - 64), 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl["precision"], "data": "synthetic",
        "config": {"workload": f"theta vs wall parameter: {len(ws)} droplets {nx}^3 R={wl['radius']:g}, {T} steps, one batch"},
        "angles": rows,
    }
    print(json.dumps(line), flush=True)


def run_sizes(args):
    """Contact angle against the lattice size (Sec. 4, Fig. 4 left): cubic lattices of edge
    32, 64, 128 and 256 with the droplet radius scaled with the edge, for three wall values.
    The lattices up to 128^3 run as one batch, the 256^3 ones one at a time. Every lattice
    takes the same number of steps; the angle is also taken 10% of the steps before the
    end, and the change over that last tenth is reported as the convergence indicator."""
    import torch

    from paper_0910_3915_gb300 import lbsc
    from paper_0910_3915_gb300 import workloads as W

    torch.cuda.set_device(0)
    wl = WORKLOADS[args.workload]
    T = args.steps if args.steps != 20000 else wl["steps"]
    T1 = T - T // 10
    ws, edges = wl["w"], wl["edges"]
    base = wl.get("prm", CONTACT)

    def radius(L):
        if "drop_edge" in wl:  # a hemisphere of the paper's initial drop volume e^3
            return (3.0 * wl["drop_edge"][L] ** 3 / (2.0 * math.pi)) ** (1.0 / 3.0)
        return wl["radius_frac"] * L

    def wall(w):
        return (0.0, w) if wl.get("wall") == "one-sided" else W.wall_split(w)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    res = {}
    total_ms, total_lu = 0.0, 0

    def angle_of(obj, L):
        # reference plane 5 l.u. above the wall; 3 l.u. for the 32^3 droplet (R = 7.5)
        a = obj.contact_angle(3.0 if L < 64 else 5.0)
        return a["theta_deg"] if a["ok"] else None

    small = [L for L in edges if L < 256]
    cases = [(L, w) for L in small for w in ws]
    fields = [W.droplet_fields(L, L, L, radius(L), seed=0) for L, _ in cases]
    params = [lbsc.Params(**base, eta_wall_r=wall(w)[0], eta_wall_b=wall(w)[1]) for _, w in cases]
    batch = lbsc.Batch(fields, params, wl["precision"])
    e0, e1 = ev(), ev()
    e0.record(stream)
    batch.step(T1)
    e1.record(stream)
    torch.cuda.synchronize()
    mid = [angle_of(batch.box(i), L) for i, (L, _) in enumerate(cases)]
    e2, e3 = ev(), ev()
    e2.record(stream)
    batch.step(T - T1)
    e3.record(stream)
    torch.cuda.synchronize()
    total_ms += e0.elapsed_time(e1) + e2.elapsed_time(e3)
    total_lu += sum(L * L * (L - 2) for L, _ in cases) * T
    for i, (L, w) in enumerate(cases):
        res[(L, w)] = (angle_of(batch.box(i), L), mid[i])
    batch.close()
    for L in [L for L in edges if L >= 256]:
        for w in ws:
            rr, rb = W.droplet_fields(L, L, L, radius(L), seed=0)
            er, eb = wall(w)
            lat = lbsc.Lattice(rr, rb, wl["precision"]).set_params(**base, eta_wall_r=er, eta_wall_b=eb)
            e0, e1 = ev(), ev()
            e0.record(stream)
            lat.step(T1)
            e1.record(stream)
            torch.cuda.synchronize()
            th_mid = angle_of(lat, L)
            e2, e3 = ev(), ev()
            e2.record(stream)
            lat.step(T - T1)
            e3.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1) + e2.elapsed_time(e3)
            total_lu += L * L * (L - 2) * T
            res[(L, w)] = (angle_of(lat, L), th_mid)
            lat.close()
    rows = []
    for w in ws:
        row = {"w": w, "theta": {}, "dtheta_last_tenth": {}}
        for L in edges:
            th, th_mid = res[(L, w)]
            row["theta"][str(L)] = round(th, 3) if th is not None else None
            row["dtheta_last_tenth"][str(L)] = (round(abs(th - th_mid), 3)
                                                if th is not None and th_mid is not None else None)
        th128, th256 = res.get((128, w), (None,))[0], res.get((256, w), (None,))[0]
        if th128 is not None and th256 is not None:
            row["rel_change_128_to_256"] = round(abs(th256 - th128) / th128, 5)
        rows.append(row)
    line = {
        "metric": METRIC, "value": round(total_lu / (total_ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "n_gpus": 1,
        "steps": T, "warmup": 0, "ms_per_step": round(total_ms / T, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl["precision"], "data": "synthetic",
        "config": {"workload": "theta vs lattice size: cubic %s, R = %s, %s = %s, %d steps each"
                               % ("/".join(str(L) for L in edges),
                                  "/".join("%.1f" % radius(L) for L in edges), "eta (one-sided)"
                                  if wl.get("wall") == "one-sided" else "w", list(ws), T),
                   "params": base},
        "sizes": rows,
    }
    print(json.dumps(line), flush=True)


def run_young(args):
    """Contact angles from surface tensions (Sec. 4.1-4.2): Young's equation with
    planar tensions (Eq. gammaMechDef on lamellae and wall slabs), the radial
    tension of a free droplet (Eq. mechRadGamma), and for sessile droplets
    the geometric angle, Huang's closed form and Young's equation with the
    drop's own radial gamma_LG."""
    import numpy as np
    import torch

    from paper_0910_3915_gb300 import lbsc
    from paper_0910_3915_gb300 import workloads as W

    torch.cuda.set_device(0)
    wl = WORKLOADS["young"]
    T = args.steps if args.steps != 20000 else wl["steps"]
    Ts = args.steps if args.steps != 20000 else wl["sessile_steps"]
    ws = wl["w"]
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    # gamma_LG: two periodic lamellae, two interfaces
    lx, ly, lz = wl["lamella"]
    rr, rb = W.lamella_fields(lx, ly, lz)
    lam = lbsc.Lattice(rr, rb).set_geometry(W.periodic_mask(lx, ly, lz)).set_params(**CONTACT)
    lam.step(T)
    prof, gsum = lam.pressure_profile()
    g_lg = 0.5 * gsum
    lam.close()
    # gamma_SL, gamma_SG: slabs of liquid (r-rich) and gas (b-rich) between the walls, one batch
    sx, sy, sz = wl["slab"]
    fields, params = [], []
    for w in ws:
        er, eb = W.wall_split(w)
        for phase in ("liquid", "gas"):
            fields.append(W.slab_fields(sx, sy, sz, phase))
            params.append(lbsc.Params(**CONTACT, eta_wall_r=er, eta_wall_b=eb))
    batch = lbsc.Batch(fields, params, "f32")
    batch.step(64)
    torch.cuda.synchronize()
    t0.record(stream)
    batch.step(T - 64)
    t1.record(stream)
    torch.cuda.synchronize()
    slab_ms = t0.elapsed_time(t1)
    tens = []
    for i in range(len(ws)):
        sl = 0.5 * batch.box(2 * i).pressure_profile()[1]
        sg = 0.5 * batch.box(2 * i + 1).pressure_profile()[1]
        tens.append((sl, sg))
    batch.close()
    # radial gamma_LG of a free droplet in a periodic box
    n = wl["free"][0]
    c = (n / 2, n / 2, n / 2)
    rr, rb = W.droplet_fields(n, n, n, wl["free_radius"], seed=0, centre=c)
    fr = lbsc.Lattice(rr, rb).set_geometry(W.periodic_mask(n, n, n)).set_params(**CONTACT)
    fr.step(T)
    _, g_rad_free, rs_free = fr.pressure_radial(c, 1.0, n // 2, 0.0, n / 2 - 5)
    fr.close()
    # sessile droplets: geometric angle, Huang, radial gamma_LG about the fitted centre
    m = wl["sessile"][0]
    fields = [W.droplet_fields(m, m, m, wl["sessile_radius"], seed=0) for _ in ws]
    params = [lbsc.Params(**CONTACT, eta_wall_r=W.wall_split(w)[0], eta_wall_b=W.wall_split(w)[1]) for w in ws]
    sb = lbsc.Batch(fields, params, "f32")
    sb.step(Ts)
    rows = []
    for i, w in enumerate(ws):
        box = sb.box(i)
        a = box.contact_angle(5.0)
        rr_, rb_, _, _ = box.moments()
        r_in, r_out = bulk_densities(rr_, rb_)
        g_rad = rs = None
        if a["ok"] and a["n_points"] >= 4:
            cen = (a["xc"], a["yc"], a["zc"])
            _, g_rad, rs = box.pressure_radial(cen, 1.0, 2 * m, 5.5, m / 2 - 5)
        sl, sg = tens[i]
        row = {"w": w, "gamma_sl": sl, "gamma_sg": sg,
               "theta_young_planar": round(lbsc.young_theta(sg, sl, g_lg), 2),
               "theta_geometric": round(a["theta_deg"], 2) if a["ok"] else None,
               "theta_huang": round(lbsc.huang_theta(W.wall_split(w)[0], W.wall_split(w)[1], r_in, r_out), 2),
               "gamma_lg_radial": g_rad, "R_s": rs,
               "theta_young_radial": (round(lbsc.young_theta(sg, sl, g_rad), 2)
                                      if g_rad is not None and g_rad > 0 else None)}
        rows.append(row)
    sb.close()
    nf = len(ws) * 2 * sx * sy * (sz - 2)
    line = {
        "metric": METRIC, "value": round(nf * (T - 64) / (slab_ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "n_gpus": 1,
        "steps": T, "warmup": 64, "ms_per_step": round(slab_ms / (T - 64), 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"planar and radial surface tensions: {2 * len(ws)} wall slabs {sx}x{sy}x{sz} as one "
                               f"batch (timed), lamellae {lx}x{ly}x{lz}, free drop {n}^3, "
                               f"{len(ws)} sessile drops {m}^3 R={wl['sessile_radius']:g} ({Ts} steps)"},
        "gamma_lg_planar": g_lg, "gamma_lg_radial_free": g_rad_free, "R_s_free": rs_free,
        "angles": rows,
    }
    print(json.dumps(line), flush=True)


def throughput_samples(K: int, Wm: int, peak: float):
    """Throughput of the 16-bit storage workload (256x256x128, R = 60, BF16 and
    FP16) and of the batched sweep (64 boxes), the same K steps after Wm
    warm-up steps, each tuned on itself and timed with CUDA events on its
    stream. The roofline's achieved bandwidth counts the algorithmic bytes per
    fluid-node update over the whole step (every kernel the step launches)."""
    import torch

    from paper_0910_3915_gb300 import lbsc, tune
    from paper_0910_3915_gb300 import workloads as W

    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {}
    for prec in ("bf16", "f16"):
        wl = WORKLOADS["precision-" + prec]
        nx, ny, nz = wl["dims"]
        nf = nx * ny * (nz - 2)
        er, eb = W.wall_split(wl["w"])
        rr, rb = W.droplet_fields(nx, ny, nz, wl["radius"], seed=0)
        lat = lbsc.Lattice(rr, rb, prec).set_params(**dict(CONTACT, eta_wall_r=er, eta_wall_b=eb))
        sched, _ = tune.tune(lat, steps=32)
        lat.step(Wm)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        lat.step(K)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / K
        lat.close()
        ach = nf * BYTES_PER_LU[prec] / (ms * 1e-3) / 1e9
        out["precision_" + prec] = {
            "workload": f"droplet {nx}x{ny}x{nz} R={wl['radius']:g} {prec.upper()} storage, FP32 arithmetic",
            "value": round(nf / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "steps": K, "ms_per_step": round(ms, 5),
            "schedule": tune.name(sched),
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(ach / peak, 4), "bytes_per_lu": BYTES_PER_LU[prec],
                         "kernel": "step_tma_kernel" if sched[0] == "tma" else "step_kernel"}}
    wl = WORKLOADS["sweep"]
    boxes = W.sweep_boxes(wl["boxes"], seed=wl["seed"])
    fields, params = [], []
    for bx in boxes:
        fields.append(W.droplet_fields(bx.edge, bx.edge, bx.edge, bx.radius, seed=bx.seed))
        er, eb = W.wall_split(bx.w)
        params.append(lbsc.Params(g_br=bx.g_br, eta_wall_r=er, eta_wall_b=eb, force_weights=1, force_scale=1.25))
    nf = sum(bx.edge * bx.edge * (bx.edge - 2) for bx in boxes)
    batch = lbsc.Batch(fields, params, wl["precision"])
    (b_var, b_ty, b_planes), _ = tune.tune_batch(batch, steps=32)
    batch.step(Wm)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(stream)
    batch.step(K)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / K
    batch.close()
    ach = nf * 304 / (ms * 1e-3) / 1e9
    out["sweep"] = {
        "workload": f"batched sweep: {len(boxes)} cubic boxes, edges from 48/64/80/96, R = 0.3 edge, one launch a step",
        "value": round(nf / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "steps": K, "ms_per_step": round(ms, 5),
        "schedule": {"variant": b_var, "tile": f"32x{b_ty}", "planes_per_item": b_planes},
        "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(ach / peak, 4), "bytes_per_lu": 304,
                     "kernel": "batch_tma_kernel" if b_var == "tma" else "batch_step_kernel"}}
    return out


def precision_accuracy(prec: str, steps: int):
    """16-bit storage against FP32 on the full lattice (the comparison with the
    FP64 oracle on the 64x64x32 copy is a test: tests/test_gpu_parity.py)."""
    import numpy as np

    from paper_0910_3915_gb300 import lbsc
    from paper_0910_3915_gb300 import workloads as W

    out = {}
    er, eb = W.wall_split(0.05)
    prm = dict(CONTACT, eta_wall_r=er, eta_wall_b=eb)
    # full size: 16-bit vs FP32
    nx, ny, nz = 256, 256, 128
    rr, rb = W.droplet_fields(nx, ny, nz, 60.0, seed=0)
    res = {}
    for p in ("f32", prec):
        lat = lbsc.Lattice(rr, rb, p).set_params(**prm)
        m0 = lat.conservation()[:2]
        lat.step(steps)
        r, b, _, cons = lat.moments()
        res[p] = (r, b, lat.contact_angle(5.0), cons[:2] / m0 - 1.0)
        lat.close()
    fl = np.s_[1:-1]
    rel = max(float(np.max(np.abs(res[prec][k][fl] - res["f32"][k][fl]) / np.abs(res["f32"][k][fl]))) for k in (0, 1))
    rms = max(float(np.sqrt(np.mean(((res[prec][k][fl] - res["f32"][k][fl]) / res["f32"][k][fl]) ** 2))) for k in (0, 1))
    out["vs_fp32_256x256x128"] = {"steps": steps, "max_rel_density_err": rel, "rms_rel_density_err": rms,
                                  "theta_fp32": res["f32"][2]["theta_deg"], "theta": res[prec][2]["theta_deg"],
                                  "theta_err_deg": abs(res[prec][2]["theta_deg"] - res["f32"][2]["theta_deg"]),
                                  "mass_drift": [float(v) for v in res[prec][3]],
                                  "mass_drift_fp32": [float(v) for v in res["f32"][3]]}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "slabs":
        run_slabs(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "angles":
        run_angles(args)
    elif args.workload == "young":
        run_young(args)
    elif args.workload in ("sizes", "sizes-paper"):
        run_sizes(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
