"""lb_conservation_static: the conservation sums for callers that cannot allocate.

Some callers must not allocate device memory where they need these sums (for
example while their stream is being captured into a CUDA graph, or inside a
section whose allocator policy forbids it). lb_conservation_static keeps its
scratch in a fixed device array of the library instead of memory a context
allocates. This test calls it through the C ABI on populations taken from a
lattice and checks its sums against lb_conservation of the same lattice, on
two calls in a row. The file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_0910_3915_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sums(lbsc, torch, lat, solid_dev):
    n = torch.from_numpy(np.ascontiguousarray(lat.populations())).cuda()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    nz, ny, nx = lat.shape
    lbsc.conservation_static(n.data_ptr(), solid_dev.data_ptr(), nx, ny, nz, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_static_scratch_sums_match_context_sums():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_3915_gb300 import lbsc
    nx, ny, nz = 40, 28, 18
    rr, rb = W.droplet_fields(nx, ny, nz, 7.0, seed=21)
    lat = lbsc.Lattice(rr, rb).set_params(g_br=0.08, force_weights=1, force_scale=1.25,
                                          eta_wall_r=-0.04, eta_wall_b=0.04)
    solid = torch.from_numpy(W.wall_mask(nx, ny, nz)).cuda()
    for steps in (40, 25):  # two calls in a row, on different states
        lat.step(steps)
        ref = lat.conservation()
        got = _sums(lbsc, torch, lat, solid)
        mass = ref[0] + ref[1]
        assert np.allclose(got[:2], ref[:2], rtol=1e-6, atol=0)
        assert np.allclose(got[2:5], ref[2:5], rtol=0, atol=1e-6 * mass)
        assert got[5] == 0 and got[6] == ref[6] == nx * ny * (nz - 2)
        again = _sums(lbsc, torch, lat, solid)
        assert np.array_equal(again, got)
    lat.close()


def test_static_scratch_rejects_oversize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_3915_gb300 import lbsc
    lib = lbsc.load()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.lb_conservation_static(ctypes.c_void_p(out.data_ptr()), None, 1024, 1024, 65,
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert rc == lbsc.LB_ERR_ARG
    assert b"maximum" in lib.lb_last_error(None)
