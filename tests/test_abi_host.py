"""Host-side checks of the C ABI that need no GPU: the library loads, it
exports every entry point include/lbsc.h declares, the binding's constants
match the header, and argument validation fails before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbsc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_0910_3915_gb300 import build, lbsc
    build.build()
    return lbsc.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(lb_\w+)\s*\(", text, flags=re.M)))


def test_batch_argument_errors_before_cuda(lib):
    from paper_0910_3915_gb300 import lbsc
    b = ctypes.c_void_p()
    dims = (ctypes.c_int * 3)(8, 8, 2)  # nz < 3: no room for the walls
    rr = np.ones(128)
    dp = rr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    prm = (lbsc.lb_params * 1)(lbsc.Params().c())
    assert lib.lb_batch_create(ctypes.byref(b), 1, dims, dp, dp, prm, lbsc.LB_F32, None) == lbsc.LB_ERR_ARG
    assert lib.lb_batch_create(ctypes.byref(b), 0, dims, dp, dp, prm, lbsc.LB_F32, None) == lbsc.LB_ERR_ARG
    assert b.value is None
    assert b"dimensions" in lib.lb_batch_last_error(None) or b"argument" in lib.lb_batch_last_error(None)
    assert lib.lb_batch_step(None, 1) == lbsc.LB_ERR_ARG
    assert lib.lb_batch_set_step_variant(None, lbsc.LB_STEP_TMA) == lbsc.LB_ERR_ARG
    lib.lb_batch_free(None)


def test_measure_and_round_selftest_argument_errors_before_cuda(lib):
    """lb_measure and lb_selftest_round refuse bad arguments before any CUDA call."""
    from paper_0910_3915_gb300 import lbsc
    cons = np.zeros(8)
    d = lbsc.lb_droplet()
    dp = cons.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.lb_measure(None, dp, 5.0, ctypes.byref(d)) == lbsc.LB_ERR_ARG
    v = np.zeros(4, np.float32)
    m = np.zeros(2, np.uint32)
    out = np.zeros(6, np.uint32)
    fp = v.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    up = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint))
    op = out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint))
    assert lib.lb_selftest_round(lbsc.LB_F32, fp, up, 2, op) == lbsc.LB_ERR_ARG  # 16-bit formats only
    assert lib.lb_selftest_round(lbsc.LB_BF16, fp, up, 0, op) == lbsc.LB_ERR_ARG
    assert lib.lb_selftest_round(lbsc.LB_BF16, None, up, 2, op) == lbsc.LB_ERR_ARG


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lb_init", "lb_set_geometry", "lb_set_params", "lb_step", "lb_moments",
                     "lb_contact_angle", "lb_last_error", "lb_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_0910_3915_gb300 import lbsc
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(n for n, _, _ in lbsc.SIGNATURES) == names


def test_constants_match_header():
    from paper_0910_3915_gb300 import lbsc
    text = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+(LB_\w+)\s+\(?(-?\d+)\)?", text))
    for name in ("LB_OK", "LB_ERR_ARG", "LB_ERR_CUDA", "LB_ERR_NAN", "LB_ERR_BARRIER_TIMEOUT",
                 "LB_ERR_STATE", "LB_ERR_UNSUPPORTED", "LB_F32", "LB_F16", "LB_BF16",
                 "LB_WEIGHTS_UNIT", "LB_WEIGHTS_W36", "LB_STEP_AUTO", "LB_STEP_LDG", "LB_STEP_TMA", "LB_OBS_COM",
                 "LB_OBS_COM_SOFT", "LB_OBS_WETTED", "LB_BUILD_BOUNDS_CHECKED"):
        assert int(defs[name]) == getattr(lbsc, name), name


def test_struct_layouts_match_header(lib):
    from paper_0910_3915_gb300 import lbsc
    assert ctypes.sizeof(lbsc.lb_params) == 7 * 8
    # 10 doubles, ok and n_points, phi_max and phi_min, status, tail padding to 8 bytes
    assert ctypes.sizeof(lbsc.lb_droplet) == 10 * 8 + 2 * 4 + 2 * 8 + 4 + 4
    assert lbsc.lb_droplet.phi_max.offset == 88 and lbsc.lb_droplet.status.offset == 104


def test_argument_errors_before_cuda(lib):
    from paper_0910_3915_gb300 import lbsc
    ctx = ctypes.c_void_p()
    rr = np.ones(8)
    dp = rr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.lb_init(ctypes.byref(ctx), 0, 2, 4, lbsc.LB_F32, dp, dp, None) == lbsc.LB_ERR_ARG
    assert b"dimensions" in lib.lb_last_error(None)
    assert lib.lb_init(ctypes.byref(ctx), 2, 2, 2, 7, dp, dp, None) == lbsc.LB_ERR_ARG
    assert lib.lb_init(ctypes.byref(ctx), 2, 2, 2, lbsc.LB_F32, None, dp, None) == lbsc.LB_ERR_ARG
    bad = np.array([1.0, np.nan, 1, 1, 1, 1, 1, 1])
    assert lib.lb_init(ctypes.byref(ctx), 2, 2, 2, lbsc.LB_F32,
                       bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), dp, None) == lbsc.LB_ERR_ARG
    assert ctx.value is None
    assert lib.lb_step(None, 1) == lbsc.LB_ERR_ARG
    assert lib.lb_set_params(None, None) == lbsc.LB_ERR_ARG
    assert lib.lb_moments(None, None, None, None, None) == lbsc.LB_ERR_ARG
    nb = ctypes.c_size_t()
    assert lib.lb_required_bytes(128, 128, 128, lbsc.LB_F32, ctypes.byref(nb)) == lbsc.LB_OK
    # two population buffers of 38 planes dominate: 304 B per node in FP32
    assert 304 * 128 ** 3 < nb.value < 600 * 128 ** 3  # aligned rows and spare rows pad the planes
    assert lib.lb_required_bytes(128, 128, 128, lbsc.LB_BF16, ctypes.byref(nb)) == lbsc.LB_OK
    assert nb.value < 360 * 128 ** 3  # 16-bit: half the population bytes of FP32
    lib.lb_free(None)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_0910_3915_gb300 import lbsc
    saved = lbsc._lib
    try:
        lbsc._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            lbsc.load(str(tmp_path / "missing.so"))
    finally:
        lbsc._lib = saved


def test_closed_form_angles_host(lib):
    """Young's equation and Huang's closed form are host-only entry points."""
    import math
    from paper_0910_3915_gb300 import lbsc
    import oracle
    assert lbsc.young_theta(1.0, 1.0, 0.5) == 90.0
    assert lbsc.young_theta(0.0, 1.0, 0.5) == 180.0 and lbsc.young_theta(1.0, 0.0, 0.5) == 0.0
    rng = np.random.default_rng(3)
    for _ in range(20):
        sg, sl, lg = rng.uniform(-0.02, 0.02), rng.uniform(-0.02, 0.02), rng.uniform(0.01, 0.1)
        assert math.isclose(lbsc.young_theta(sg, sl, lg), oracle.young_theta(sg, sl, lg), rel_tol=1e-14)
    with pytest.raises(lbsc.LBError):
        lbsc.young_theta(0.1, 0.0, 0.0)
    with pytest.raises(lbsc.LBError):
        lbsc.young_theta(float("nan"), 0.0, 0.1)
    # Huang (Eq. huangSigmaLG): a neutral wall gives 90 deg; w > 0 (eta_r = -w, eta_b = +w) repels r
    assert lbsc.huang_theta(0.0, 0.0, 0.7, 0.04) == 90.0
    w = 0.05
    c = -(2 * w) / ((0.7 - 0.04) / 2)
    assert math.isclose(lbsc.huang_theta(-w, w, 0.7, 0.04), math.degrees(math.acos(c)), rel_tol=1e-14)
    assert lbsc.huang_theta(-w, w, 0.7, 0.04) > 90.0 > lbsc.huang_theta(w, -w, 0.7, 0.04)
    with pytest.raises(lbsc.LBError):
        lbsc.huang_theta(0.0, 0.0, 0.04, 0.7)


def test_huang_theta_hand_worked_values(lib):
    """Eq. huangSigmaLG against values worked by hand as exact fractions
    (tests/golden/paper_values.json), including the clamp at |cos| > 1."""
    import json
    import math
    import os
    from paper_0910_3915_gb300 import lbsc
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
        ex = json.load(f)["huang_examples"]
    assert len(ex) >= 4
    for e in ex:
        num, den = (int(t) for t in e["cos_theta"].split("/"))
        c = num / den
        assert math.isclose(c, (e["eta_wall_r"] - e["eta_wall_b"]) / ((e["rho_in"] - e["rho_out"]) / 2),
                            rel_tol=1e-12, abs_tol=1e-15)
        th = lbsc.huang_theta(e["eta_wall_r"], e["eta_wall_b"], e["rho_in"], e["rho_out"])
        assert math.isclose(th, e["theta_deg"], rel_tol=0, abs_tol=1e-9), e


def test_reset_and_slab_argument_errors_before_cuda(lib):
    """lb_reset and the z-slab entry points reject bad arguments before any CUDA call."""
    from paper_0910_3915_gb300 import lbsc
    ctx = ctypes.c_void_p()
    rr = np.ones(2 * 2 * 4)
    dp = rr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.lb_reset(None, dp, dp) == lbsc.LB_ERR_ARG
    # halo flags beyond LB_HALO_BELOW | LB_HALO_ABOVE, a slab without an owned plane, a negative base
    assert lib.lb_init_slab(ctypes.byref(ctx), 2, 2, 4, lbsc.LB_F32, dp, dp, None, 4, 0, None) == lbsc.LB_ERR_ARG
    assert lib.lb_init_slab(ctypes.byref(ctx), 2, 2, 2, lbsc.LB_F32, dp, dp, None, 1, 0, None) == lbsc.LB_ERR_ARG
    assert lib.lb_init_slab(ctypes.byref(ctx), 2, 2, 4, lbsc.LB_F32, dp, dp, None, 1, -1, None) == lbsc.LB_ERR_ARG
    bad_ref = np.array([np.nan, 0.1])
    assert lib.lb_init_slab(ctypes.byref(ctx), 2, 2, 4, lbsc.LB_BF16, dp, dp, None, 1, 0,
                            bad_ref.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == lbsc.LB_ERR_ARG
    assert ctx.value is None
    assert lib.lb_halo_exchange(None, None) == lbsc.LB_ERR_ARG
    assert lib.lb_halo_pack(None, 0, None) == lbsc.LB_ERR_ARG
    assert lib.lb_halo_unpack(None, 1, None) == lbsc.LB_ERR_ARG
    assert lib.lb_slabs_step(None, 0, 1) == lbsc.LB_ERR_ARG
    nb = ctypes.c_size_t()
    assert lib.lb_halo_bytes(None, ctypes.byref(nb)) == lbsc.LB_ERR_ARG


def test_slab_split_covers_the_fluid_planes():
    """slabs.split: even, contiguous, every fluid plane owned exactly once, at
    least one plane a slab; halo flags on the inner faces only."""
    from paper_0910_3915_gb300 import lbsc, slabs
    for nz, n in ((128, 2), (37, 3), (19, 8), (8, 3), (5, 1)):
        b = slabs.split(nz, n)
        assert b[0][0] == 1 and b[-1][1] == nz - 1
        assert all(b[i][1] == b[i + 1][0] for i in range(n - 1))
        sizes = [z1 - z0 for z0, z1 in b]
        assert min(sizes) >= (2 if n > 1 else 1) and max(sizes) - min(sizes) <= 1
        flags = [slabs.halo_flags(i, n) for i in range(n)]
        assert flags[0] == (lbsc.LB_HALO_ABOVE if n > 1 else 0)
        assert flags[-1] == (lbsc.LB_HALO_BELOW if n > 1 else 0)
        assert all(f == lbsc.LB_HALO_BELOW | lbsc.LB_HALO_ABOVE for f in flags[1:-1])
    with pytest.raises(ValueError):
        slabs.split(5, 2)  # three fluid planes: two slabs would leave one with a single plane
    with pytest.raises(ValueError):
        slabs.split(8, 4)
