"""Bounds-checked build (a stand-in for a memory checker, which is closed on
this pool): the library compiled with LBSC_DEBUG_BOUNDS checks every
population index of the step kernels against its buffer and reports a
violation through the status word instead of touching memory. Every kernel
variant and awkward shape runs clean under it, and its results equal the
release build's bit for bit (the checks change no value)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_0910_3915_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CONTACT = dict(g_br=0.08, force_weights=1, force_scale=1.25, eta_wall_r=-0.04, eta_wall_b=0.04)

# (precision, (nx, ny, nz), variant, stages, tile rows, y-tiles, z segments, general geometry)
CASES = [
    ("f32", (37, 23, 21), "ldg", 0, 8, 0, 3, False),
    ("f32", (37, 23, 21), "ldg", 0, 4, 7, 2, False),
    ("f32", (33, 17, 9), "ldg", 0, 16, 0, 1, False),
    ("f32", (37, 23, 21), "tma", 2, 8, 5, 2, False),
    ("f32", (40, 24, 16), "tma", 3, 4, 0, 4, False),
    ("f16", (37, 23, 21), "tma", 2, 16, 2, 3, False),
    ("bf16", (37, 23, 21), "ldg", 0, 8, 23, 1, False),
    ("f32", (36, 20, 16), "ldg", 0, 8, 3, 2, True),
    ("bf16", (36, 20, 16), "ldg", 0, 4, 0, 1, True),
]

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
from paper_0910_3915_gb300 import lbsc, workloads as W
from test_gpu_bounds import CASES, CONTACT, run_case
assert lbsc.build_flags() & lbsc.LB_BUILD_BOUNDS_CHECKED
out = {f"c{i}": run_case(lbsc, *c) for i, c in enumerate(CASES)}
np.savez(sys.argv[2], **out)
"""


def geometry(nx, ny, nz):
    solid = W.wall_mask(nx, ny, nz)
    solid[1:5, 6:10, 4:8] = 1
    solid[1:3, :, nx - 6:] = 1
    return solid


def run_case(lbsc, prec, dims, variant, stages, ty, nty, seg, general):
    nx, ny, nz = dims
    rr, rb = W.droplet_fields(nx, ny, nz, 6.0, seed=4)
    lat = lbsc.Lattice(rr, rb, prec)
    if general:
        lat.set_geometry(geometry(nx, ny, nz))
    lat.set_params(**CONTACT).set_step_variant(variant, stages).set_tiling(ty, nty, seg)
    lat.step(40)  # one graph replay (32 steps) and single launches
    lat.sync()    # raises LBError (LB_ERR_STATE) if an index left its buffer
    n = lat.populations()
    lat.close()
    return n


def test_bounds_checked_build_runs_clean_and_matches_release(tmp_path):
    from paper_0910_3915_gb300 import build as B
    from paper_0910_3915_gb300 import lbsc
    path = B.build(debug_bounds=True)
    out = tmp_path / "debug.npz"
    env = dict(os.environ, LBSC_LIBRARY=path)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(out)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    dbg = np.load(out)
    lbsc.load()
    assert not lbsc.build_flags() & lbsc.LB_BUILD_BOUNDS_CHECKED
    for i, c in enumerate(CASES):
        assert np.array_equal(dbg[f"c{i}"], run_case(lbsc, *c), equal_nan=True), c
