"""Host logic of bench.py that needs no GPU: the committed DRAM-traffic record
matches the step kernels' sources, and the roofline's traffic lookup takes the
tuned schedule's record, else that of a recorded schedule of the same kernel
family (variant, stages, tile height), and names which."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_is_well_formed():
    rec = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")))
    assert len(rec["step_sources_sha256"]) == 64
    assert rec["bytes_per_launch"]
    for key, val in rec["bytes_per_launch"].items():
        workload, sched = key.split(" ", 1)
        assert workload in bench.WORKLOADS and len(sched.split(":")) == 5
        assert 4e8 < val < 2e9  # 128^3 FP32 about 0.6 GB, 256x256x128 16-bit about 1.3 GB


def test_traffic_lookup_exact_then_family():
    full = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")))
    rec = full["bytes_per_launch"]
    if full["step_sources_sha256"] != bench.step_source_sha256():
        # the step kernels changed since the record was taken: every lookup says "unknown"
        assert bench.step_kernel_traffic(*sorted(rec)[0].split(" ", 1)) == (None, None)
        return
    key = sorted(rec)[0]
    workload, sched = key.split(" ", 1)
    assert bench.step_kernel_traffic(workload, sched) == (rec[key], sched)
    v, ns, ty = sched.split(":")[:3]
    other = f"{v}:{ns}:{ty}:13:0"  # an unrecorded schedule of the same family
    val, used = bench.step_kernel_traffic(workload, other)
    assert val is not None and used.split(":")[:3] == [v, ns, ty]
    assert bench.step_kernel_traffic(workload, "ldg:0:16:3:0") == (None, None)  # no recorded 16-row kernel
    assert bench.step_kernel_traffic(workload, None) == (None, None)
