"""Host logic of bench.py that needs no GPU: the committed DRAM-traffic record
matches the step kernels' sources, and the roofline's traffic lookup takes the
tuned schedule's record, else that of a recorded schedule of the same kernel
family (variant, stages, tile height), and names which; the reference arm (the
oracle timed on the host cores) prints the contract's line, and only on rank 0."""
import argparse
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


def _reference_args():
    return argparse.Namespace(gpus=1, steps=7, warmup=3, workload="small", impl="reference")


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    real = bench.oracle_mlups
    monkeypatch.setattr(bench, "oracle_mlups", lambda dims, radius, w, seconds: real(dims, radius, w, 0.2))
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.run_reference(_reference_args())
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "MLUPS"
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 7, 3)
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["dtype"] == "f64"
    assert "32x32x32" in line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and "oracle steps" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_off_rank_zero(monkeypatch, capsys):
    def never(*a, **k):
        raise AssertionError("the oracle must not run on a rank other than 0")

    monkeypatch.setattr(bench, "oracle_mlups", never)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.run_reference(_reference_args())
    assert capsys.readouterr().out == ""
