"""GPU parity of the pressure tensor (Sec. 4.1) and of the surface-tension
reductions (Eq. gammaMechDef, Eq. mechRadGamma) against the FP64 oracle.

The GPU lattice is loaded with the oracle's own populations, so both sides
evaluate the tensor on the same state (up to the storage rounding of the
populations); the reductions are then compared bin by bin.
"""
import math

import numpy as np
import pytest

import oracle
from paper_0910_3915_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CONTACT = dict(g_br=0.08, force_weights=1, force_scale=1.25)


@pytest.fixture(scope="module")
def lbsc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_3915_gb300 import lbsc as m
    m.load()
    return m


def _pair(lbsc, rr, rb, solid, prm, steps, precision="f32", general=False):
    st = oracle.State(rr, rb, solid, oracle.Params(**prm)).step(steps)
    lat = lbsc.Lattice(rr, rb, precision)
    if general:
        lat.set_geometry(solid)
    lat.set_params(**prm).set_populations(st.n)
    return st, lat


@pytest.mark.parametrize("precision,tol", [("f32", 2e-6), ("bf16", 2e-2)])
def test_pressure_tensor_matches_oracle(lbsc, precision, tol):
    nx, ny, nz = 26, 21, 15
    rr, rb = W.droplet_fields(nx, ny, nz, 7.0, seed=5)
    prm = dict(CONTACT, eta_wall_r=-0.04, eta_wall_b=0.04)
    st, lat = _pair(lbsc, rr, rb, W.wall_mask(nx, ny, nz), prm, 150, precision)
    g = lat.pressure_tensor()
    lat.close()
    o = st.pressure_tensor()
    assert np.all(g[:, 0] == 0) and np.all(g[:, -1] == 0)
    scale = np.abs(o).max()
    assert np.abs(g - o).max() <= tol * scale, np.abs(g - o).max() / scale


def test_pressure_tensor_general_geometry(lbsc):
    nx, ny, nz = 20, 18, 14
    solid = W.wall_mask(nx, ny, nz)
    solid[1:5, 6:10, 4:8] = 1
    rr, rb = W.droplet_fields(nx, ny, nz, 6.0, seed=6)
    prm = dict(CONTACT, eta_wall_r=0.03, eta_wall_b=-0.03, tau_r=0.9, tau_b=0.9)
    st, lat = _pair(lbsc, rr, rb, solid, prm, 100, general=True)
    g = lat.pressure_tensor()
    lat.close()
    o = st.pressure_tensor()
    assert np.all(g[:, solid == 1] == 0)
    assert np.abs(g - o).max() <= 2e-6 * np.abs(o).max()


@pytest.mark.parametrize("geometry", ["lamella", "walls"])
def test_pressure_profile_matches_oracle(lbsc, geometry):
    if geometry == "lamella":
        nx, ny, nz = 4, 5, 48
        rr, rb = W.lamella_fields(nx, ny, nz, seed=1, noise=1e-3)
        solid, prm, general = W.periodic_mask(nx, ny, nz), dict(CONTACT), True
    else:
        nx, ny, nz = 4, 5, 34
        rr, rb = W.slab_fields(nx, ny, nz, "liquid")
        solid, prm, general = W.wall_mask(nx, ny, nz), dict(CONTACT, eta_wall_r=-0.05, eta_wall_b=0.05), False
    st, lat = _pair(lbsc, rr, rb, solid, prm, 800, general=general)
    prof, gsum = lat.pressure_profile()
    lat.close()
    r, b, _, _ = st.moments()
    oprof, ogsum = oracle.pressure_profile(st.pressure_tensor(), solid, r, b)
    assert np.array_equal(prof[:, 7], oprof[:, 7])
    assert np.abs(prof[:, :7] - oprof[:, :7]).max() < 2e-6
    assert abs(gsum - ogsum) < 2e-6 * max(1.0, abs(ogsum)) and abs(gsum - ogsum) < 1e-5 * nz


@pytest.mark.parametrize("geometry", ["free", "sessile"])
def test_pressure_radial_matches_oracle(lbsc, geometry):
    if geometry == "free":
        n = 24
        centre = (12.3, 11.7, 12.2)
        rr, rb = W.droplet_fields(n, n, n, 6.0, seed=2, centre=centre)
        solid, prm, general, zmin = W.periodic_mask(n, n, n), dict(CONTACT), True, 0.0
        dims = (n, n, n)
    else:
        dims = (28, 26, 18)
        centre = (14.0, 13.0, 0.5)
        rr, rb = W.droplet_fields(*dims, 8.0, seed=3)
        solid = W.wall_mask(*dims)
        prm, general, zmin = dict(CONTACT, eta_wall_r=-0.05, eta_wall_b=0.05), False, 3.0
    st, lat = _pair(lbsc, rr, rb, solid, prm, 300, general=general)
    bins, gamma, R_s = lat.pressure_radial(centre, 1.0, 20, zmin, 9.0)
    lat.close()
    r, b, _, _ = st.moments()
    obins, ogamma, oR = oracle.pressure_radial(st.pressure_tensor(), solid, r, b, centre, 1.0, 20, zmin, 9.0,
                                               periodic_z=general)
    assert np.array_equal(bins[:, 3], obins[:, 3])
    assert np.abs(bins[:, :3] - obins[:, :3]).max() < 2e-6
    assert math.isfinite(oR) and abs(R_s - oR) < 1e-4
    assert abs(gamma - ogamma) < 1e-5


def test_radial_bins_argument_checks(lbsc):
    rr, rb = W.droplet_fields(16, 16, 10, 4.0)
    lat = lbsc.Lattice(rr, rb)
    for args in (((8, 8, 1), 0.0, 10), ((8, 8, 1), 1.0, 0), ((8, 8, 1), 1.0, 1025), ((math.nan, 8, 1), 1.0, 10)):
        with pytest.raises(lbsc.LBError):
            lat.pressure_radial(args[0], args[1], args[2])
    lat.close()


def _gamma_gpu(lbsc, rr, rb, solid, prm, steps, interfaces, general):
    lat = lbsc.Lattice(rr, rb)
    if general:
        lat.set_geometry(solid)
    lat.set_params(**prm)
    lat.step(steps)
    _, g = lat.pressure_profile()
    lat.close()
    return g / interfaces


def _gamma_oracle(rr, rb, solid, prm, steps, interfaces):
    st = oracle.State(rr, rb, solid, oracle.Params(**prm)).step(steps)
    r, b, _, _ = st.moments()
    return oracle.pressure_profile(st.pressure_tensor(), solid, r, b)[1] / interfaces


def test_young_planar_tensions_match_oracle(lbsc):
    """The planar-interface route to Young's angle (Sec. 4.1): gamma_LG from two
    lamellae, gamma_SL and gamma_SG from slabs of each phase between the walls,
    each evolved on the GPU and by the oracle from the same start."""
    w = 0.05
    er, eb = W.wall_split(w)
    wall = dict(CONTACT, eta_wall_r=er, eta_wall_b=eb)
    rr, rb = W.lamella_fields(2, 2, 48)
    lg = (_gamma_gpu(lbsc, rr, rb, W.periodic_mask(2, 2, 48), CONTACT, 3000, 2, True),
          _gamma_oracle(rr, rb, W.periodic_mask(2, 2, 48), CONTACT, 3000, 2))
    out = {}
    for phase in ("liquid", "gas"):
        rr, rb = W.slab_fields(2, 2, 30, phase)
        out[phase] = (_gamma_gpu(lbsc, rr, rb, W.wall_mask(2, 2, 30), wall, 3000, 2, False),
                      _gamma_oracle(rr, rb, W.wall_mask(2, 2, 30), wall, 3000, 2))
    for g, o in (lg, out["liquid"], out["gas"]):
        assert math.isclose(g, o, rel_tol=2e-3, abs_tol=1e-6), (g, o)
    tg = lbsc.young_theta(out["gas"][0], out["liquid"][0], lg[0])
    to = oracle.young_theta(out["gas"][1], out["liquid"][1], lg[1])
    assert abs(tg - to) < 0.1 and tg > 90.0


def test_laplace_law_free_droplets_3d(lbsc):
    """Free droplets in a periodic box (Sec. 4.2 set-up, on the GPU): the
    pressure jump is linear in 1/R with no intercept, its slope is twice the
    planar surface tension (Eq. gammaMechDef on two lamellae) within 15%, and
    the radial tension of the largest drop (Eq. mechRadGamma) agrees with the
    planar one within 10%."""
    n, steps = 48, 4000
    c = (n / 2, n / 2, n / 2)
    inv_r, dp = [], []
    for R in (8.0, 10.0, 12.0, 14.0):
        rr, rb = W.droplet_fields(n, n, n, R, seed=1, centre=c)
        lat = lbsc.Lattice(rr, rb).set_geometry(W.periodic_mask(n, n, n)).set_params(**CONTACT)
        lat.step(steps)
        P = lat.pressure_tensor()
        r, b, _, _ = lat.moments()
        p = (P[0] + P[1] + P[2]) / 3
        dp.append(p[n // 2, n // 2, n // 2] - p[0, 0, 0])
        inv_r.append(1.0 / (3.0 * float(((r - b) > 0).sum()) / (4.0 * math.pi)) ** (1.0 / 3.0))
        if R == 14.0:
            _, g_rad, R_s = lat.pressure_radial(c, 1.0, n // 2, 0.0, n / 2 - 5)
        lat.close()
    inv_r, dp = np.array(inv_r), np.array(dp)
    slope, icpt = np.polyfit(inv_r, dp, 1)
    fit = slope * inv_r + icpt
    r2 = 1 - ((dp - fit) ** 2).sum() / ((dp - dp.mean()) ** 2).sum()
    assert r2 > 0.99 and abs(icpt) < 0.1 * dp.max()
    rr, rb = W.lamella_fields(4, 4, 64)
    lam = lbsc.Lattice(rr, rb).set_geometry(W.periodic_mask(4, 4, 64)).set_params(**CONTACT)
    lam.step(steps)
    gamma = 0.5 * lam.pressure_profile()[1]
    lam.close()
    assert gamma > 0
    assert math.isclose(slope / 2, gamma, rel_tol=0.15), (slope / 2, gamma)
    assert math.isclose(g_rad, gamma, rel_tol=0.10) and abs(R_s - 1 / inv_r[-1]) < 1.0, (g_rad, gamma, R_s)
