"""Pins for the FP64 oracle: facts fixed by the paper and by the mathematics.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails it. No expected value here
comes from the CUDA path.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_0910_3915_gb300 import workloads as W

from hand_stepper import VEL, from_oracle_layout, step as hand_step

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- lattice table
def test_d3q19_table_isotropy():
    """zeta_k and c_s^2 = 1/3 (Sec. 2, D3Q19): moments up to fourth order."""
    c, zeta, opp = oracle.lattice()
    assert len({tuple(v) for v in c}) == 19
    assert np.array_equal(c[opp], -c)
    assert math.isclose(zeta.sum(), 1.0, abs_tol=1e-15)
    assert np.allclose(zeta @ c, 0, atol=1e-16)
    m2 = np.einsum("k,ki,kj->ij", zeta, c, c)
    assert np.allclose(m2, np.eye(3) / 3, atol=1e-15)
    # fourth-order isotropy: sum zeta c_x^4 = 3 cs^4, sum zeta c_x^2 c_y^2 = cs^4
    assert math.isclose(zeta @ c[:, 0] ** 4, 1 / 3, abs_tol=1e-15)
    assert math.isclose(zeta @ (c[:, 0] ** 2 * c[:, 1] ** 2), 1 / 9, abs_tol=1e-15)


# ---------------------------------------------------------------- equilibrium
@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments_exact(seed):
    """Eq. Equil conserves mass and momentum exactly on D3Q19: the two cubic
    terms cancel in the first moment, so sum n^eq = rho and sum n^eq c = rho u;
    the second moment is rho (c_s^2 delta + u u)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.05, 1.0)
    u = rng.uniform(-0.12, 0.12, 3)
    c, zeta, _ = oracle.lattice()
    neq = oracle.equilibrium(rho, u)
    assert math.isclose(neq.sum(), rho, rel_tol=1e-14)
    assert np.allclose(neq @ c, rho * u, atol=1e-15)
    m2 = np.einsum("k,ki,kj->ij", neq, c, c)
    assert np.allclose(m2, rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)


def test_equilibrium_axis_special_case():
    """For u along +x, Eq. Equil on the +x velocity reduces to zeta rho (1 + 3u + 3u^2)
    (the cubic terms 4.5 u^3 - 4.5 u^3 cancel)."""
    c, zeta, _ = oracle.lattice()
    k = int(np.flatnonzero((c == [1, 0, 0]).all(1))[0])
    for u in (0.01, 0.05, 0.1):
        neq = oracle.equilibrium(0.7, [u, 0, 0])
        assert math.isclose(neq[k], 0.7 / 18 * (1 + 3 * u + 3 * u * u), rel_tol=1e-14)
        kd = int(np.flatnonzero((c == [1, 1, 0]).all(1))[0])
        # diagonal (1,1,0): c.u = u, u^2 = u^2: same polynomial with zeta = 1/36
        assert math.isclose(neq[kd], 0.7 / 36 * (1 + 3 * u + 3 * u * u), rel_tol=1e-14)


# ---------------------------------------------------------------- step invariants
def test_rest_state_is_fixed_point():
    rr = np.full((6, 5, 4), 0.3)
    rb = np.full((6, 5, 4), 0.2)
    st = oracle.State(rr, rb, W.periodic_mask(4, 5, 6), Params(g_br=0.1))
    n0 = st.n.copy()
    st.step(7)
    assert np.allclose(st.n, n0, rtol=0, atol=1e-15)


def test_mass_conserved_with_walls_and_forces():
    """BGK conserves each component's mass per node; bounce-back conserves it
    globally: per-component total mass is constant."""
    rr, rb = W.droplet_fields(16, 14, 12, 5.0, seed=3)
    er, eb = W.wall_split(0.07)
    st = oracle.State(rr, rb, W.wall_mask(16, 14, 12),
                      Params(g_br=0.1, eta_wall_r=er, eta_wall_b=eb, tau_r=0.9, tau_b=1.3))
    m0 = st.moments()[3][:2].copy()
    st.step(300)
    m1 = st.moments()[3][:2]
    assert np.allclose(m1, m0, rtol=1e-13, atol=0)


@pytest.mark.parametrize("g", [0.0, 0.12])
def test_momentum_conserved_periodic(g):
    """In a periodic box, sum over nodes and components of F^a vanishes (the
    x -> x - c_k antisymmetry of Eq. SCforce with cross-coupling), and BGK with
    the shifted velocity adds exactly F^a: total momentum is constant."""
    n = W.random_populations(6, 5, 7, seed=11)
    st = oracle.State(np.ones((7, 5, 6)), np.ones((7, 5, 6)), W.periodic_mask(6, 5, 7),
                      Params(g_br=g, tau_r=0.8, tau_b=1.4))
    st.n[:] = n
    p0 = st.moments()[3][2:5].copy()
    F = st.force()
    assert np.allclose(F.sum(axis=(0, 2, 3, 4)), 0, atol=1e-13)
    st.step(50)
    p1 = st.moments()[3][2:5]
    assert np.allclose(p1, p0, atol=1e-12)
    assert abs(p0).max() > 1e-3  # the state does carry momentum


@pytest.mark.parametrize("weights,lam", [(0, 10.0), (1, 12.0)])
def test_force_on_linear_psi(weights, lam):
    """Eq. SCforce on a linear psi^b field: sum_k G_k psi(x + c_k) c_k = lambda grad psi
    exactly, lambda = sum_k G_k c_kx^2 (10 unweighted, 12 for G_k = 36 zeta_k),
    and the force on r points down the gradient of psi^b (repulsion, g > 0)."""
    nx, ny, nz = 8, 8, 8
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = np.array([0.011, -0.007, 0.004])
    psi_b = 0.2 + s[0] * x + s[1] * y + s[2] * z
    rho_b = -np.log1p(-psi_b)
    rho_r = np.full_like(rho_b, 0.5)
    g, kappa = 0.09, 1.7
    st = oracle.State(rho_r, rho_b, W.periodic_mask(nx, ny, nz),
                      Params(g_br=g, force_weights=weights, force_scale=kappa))
    F = st.force()
    psi_r = 1 - math.exp(-0.5)
    inner = (slice(1, -1),) * 3
    for d in range(3):
        expect = -kappa * g * psi_r * lam * s[d]
        assert np.allclose(F[0, d][inner], expect, rtol=1e-10, atol=1e-16)
    # the force on b uses grad psi^r = 0 here
    assert np.allclose(F[1][(slice(None),) + inner], 0, atol=1e-15)


def test_wall_force_direction():
    """A wall with a positive b-like pseudo-density repels r (Sec. 2, the wall
    as a species with g > 0): the force on r next to the bottom wall points +z."""
    rr = np.full((6, 4, 4), 0.5)
    rb = np.full((6, 4, 4), 0.0)
    st = oracle.State(rr, rb, W.wall_mask(4, 4, 6), Params(g_br=0.1, eta_wall_b=0.2))
    F = st.force()
    assert (F[0, 2, 1] > 0).all() and (F[0, 2, -2] < 0).all()
    assert np.allclose(F[0, :2], 0, atol=1e-16)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("dims,walls", [((4, 4, 4), False), ((4, 3, 6), True)])
def test_matches_independent_pull_stepper(dims, walls):
    """The oracle (push) against an independent per-node pull stepper, 3 steps,
    off-equilibrium populations, forces and walls on, unequal tau."""
    nx, ny, nz = dims
    solid = W.wall_mask(nx, ny, nz) if walls else W.periodic_mask(nx, ny, nz)
    prm = Params(g_br=0.15, tau_r=0.85, tau_b=1.25, eta_wall_r=-0.05, eta_wall_b=0.12,
                 force_weights=1, force_scale=1.3)
    st = oracle.State(np.ones((nz, ny, nx)), np.ones((nz, ny, nx)), solid, prm)
    st.n[:] = W.random_populations(nx, ny, nz, seed=5) * (1 - solid)[None, None]
    c, _, _ = oracle.lattice()
    h = from_oracle_layout(st.n, c)
    for _ in range(3):
        st.step(1)
        h = hand_step(h, solid, (prm.tau_r, prm.tau_b), prm.g_br,
                      (prm.eta_wall_r, prm.eta_wall_b), prm.force_weights, prm.force_scale)
        ho = from_oracle_layout(st.n, c)
        for a in (0, 1):
            assert np.allclose(ho[a], h[a], rtol=1e-13, atol=1e-15)


def test_mirror_symmetry_r_b():
    """Swapping the components and the wall's two pseudo-densities swaps the
    result exactly: the method treats r and b alike."""
    rr, rb = W.droplet_fields(12, 10, 9, 4.0, seed=2)
    solid = W.wall_mask(12, 10, 9)
    a = oracle.State(rr, rb, solid, Params(g_br=0.1, eta_wall_r=-0.04, eta_wall_b=0.04, force_weights=1))
    b = oracle.State(rb, rr, solid, Params(g_br=0.1, eta_wall_r=0.04, eta_wall_b=-0.04, force_weights=1))
    a.step(40)
    b.step(40)
    assert np.array_equal(a.n[0], b.n[1]) and np.array_equal(a.n[1], b.n[0])


# ---------------------------------------------------------------- physics the paper fixes
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_shear_wave_viscosity(tau):
    """Sec. 4: kinematic viscosity nu = (2 tau - 1)/6, i.e. 1/6 at tau = 1.
    A shear wave u_x = A sin(k z) decays as exp(-nu k^2 t)."""
    gold = golden("paper_values.json")["kinematic_viscosity"]
    nu = (2 * tau - 1) / 6
    if tau == 1.0:
        assert math.isclose(nu, gold["value_at_tau_1"], rel_tol=1e-15)
    nz, A = 64, 1e-4
    kw = 2 * math.pi / nz
    st = oracle.State(np.ones((nz, 1, 1)), np.zeros((nz, 1, 1)), W.periodic_mask(1, 1, nz),
                      Params(g_br=0.0, tau_r=tau, tau_b=tau))
    for z in range(nz):
        st.n[0, :, z, 0, 0] = oracle.equilibrium(1.0, [A * math.sin(kw * z), 0, 0])
    T = 400
    st.step(T)
    _, _, u, _ = st.moments()
    amp = 2 / nz * np.sum(u[0, :, 0, 0] * np.sin(kw * np.arange(nz)))
    assert math.isclose(amp / A, math.exp(-nu * kw * kw * T), rel_tol=2e-3)


CONTACT = Params(g_br=0.08, force_weights=1, force_scale=1.25)


def _lamella(nz=64, steps=6000, prm=CONTACT):
    rr, rb = W.lamella_fields(1, 1, nz)
    st = oracle.State(rr, rb, W.periodic_mask(1, 1, nz), prm)
    st.step(steps)
    return st


def test_flat_interface_mechanical_equilibrium():
    """Sec. 4.1, flat lamellae at rest: the normal component P_zz of the
    pressure tensor is constant across the interface (d/dz P_zz = 0), the two
    components mirror each other, and the bulk pressure equals the tensor's
    bulk value c_s^2 (rho_r + rho_b) + g kappa lambda psi^r psi^b."""
    st = _lamella()
    rr, rb, u, _ = st.moments()
    P = st.pressure_tensor()
    pzz = P[2, :, 0, 0]
    assert np.ptp(pzz) / pzz.mean() < 2e-3
    r, b = rr[:, 0, 0], rb[:, 0, 0]
    assert np.allclose(r, np.roll(b, 32), atol=1e-12)
    assert np.abs(u).max() < 1e-6
    zb = 16  # bulk of the r-rich lamella
    psr, psb = 1 - math.exp(-r[zb]), 1 - math.exp(-b[zb])
    bulk = (r[zb] + b[zb]) / 3 + CONTACT.g_br * CONTACT.force_scale * 12 * psr * psb
    assert math.isclose(pzz[zb], bulk, rel_tol=1e-6)  # bulk uniform to ~1e-8 after 6000 steps
    assert r[zb] > 0.7 and b[zb] < 0.05


def _surface_tension_flat(st):
    """gamma = int (P_N - P_T) dz over one interface (Eq. gammaMechDef)."""
    P = st.pressure_tensor()
    d = P[2, :, 0, 0] - P[0, :, 0, 0]
    return 0.5 * d.sum()  # the periodic box holds two interfaces


def test_laplace_law_cylinders():
    """Laplace's law for columns of r in b (quasi-2D, periodic): the pressure
    jump is linear in 1/R with no intercept, and its slope is the surface
    tension of the flat interface from Eq. gammaMechDef."""
    nx = ny = 48
    inv_r, dp = [], []
    for R in (8.0, 10.0, 12.0, 15.0):
        z, y, x = np.meshgrid(np.arange(1), np.arange(ny), np.arange(nx), indexing="ij")
        inside = (x - nx / 2) ** 2 + (y - ny / 2) ** 2 <= R * R
        rr = np.where(inside, 0.7, 0.04)
        rb = np.where(inside, 0.04, 0.7)
        st = oracle.State(rr, rb, W.periodic_mask(nx, ny, 1), CONTACT)
        st.step(3000)
        P = st.pressure_tensor()
        p = (P[0] + P[1]) / 2
        dp.append(p[0, ny // 2, nx // 2] - p[0, 0, 0])
        rr2, rb2, _, _ = st.moments()
        # equivalent radius of the phi > 0 region
        inv_r.append(1 / math.sqrt(float(((rr2 - rb2) > 0).sum()) / math.pi))
    inv_r, dp = np.array(inv_r), np.array(dp)
    slope, icpt = np.polyfit(inv_r, dp, 1)
    fit = slope * inv_r + icpt
    r2 = 1 - ((dp - fit) ** 2).sum() / ((dp - dp.mean()) ** 2).sum()
    assert r2 > 0.99
    assert abs(icpt) < 0.1 * dp.max()
    gamma = _surface_tension_flat(_lamella())
    assert gamma > 0
    assert math.isclose(slope, gamma, rel_tol=0.15)


# ---------------------------------------------------------------- geometry of the measurement
def _cap_field(theta_deg, R=20.0, n=72, nz=48, width=2.0):
    """Synthetic phi = tanh((R - |p - c|)/width) of a sphere cut by the wall plane
    z = 0.5 at angle theta (centre height 0.5 - R cos theta)."""
    zc = 0.5 - R * math.cos(math.radians(theta_deg))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    d = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - zc) ** 2)
    phi = np.tanh((R - d) / width)
    solid = W.wall_mask(n, n, nz)
    rr = 0.37 + 0.33 * phi
    rb = 0.37 - 0.33 * phi
    return rr, rb, solid, zc


@pytest.mark.parametrize("theta", [45.0, 60.0, 90.0, 120.0, 150.0])
def test_contact_angle_on_analytic_caps(theta):
    """Sec. 3, Eq. geoCA with r = (4h^2 + b^2)/(8h): a spherical cap of known angle
    is recovered within 0.5 deg by the reference-plane construction (1 deg by
    the sphere fit); h, b, r satisfy the cap relation."""
    rr, rb, solid, zc = _cap_field(theta)
    ca = oracle.contact_angle(rr, rb, solid, offset=5.0)
    assert ca["ok"] == 1
    assert abs(ca["theta_deg"] - theta) < 0.5
    # the fit (a cross-check, not the paper's construction) sees few points on shallow caps
    assert abs(ca["theta_fit_deg"] - theta) < 1.0
    h, b, r = ca["h"], ca["b"], ca["r"]
    assert math.isclose(r, (4 * h * h + b * b) / (8 * h), rel_tol=1e-12)
    assert abs(ca["r_fit"] - 20.0) < 0.5 and abs(ca["zc"] - zc) < 0.5


def test_contact_angle_small_cap_with_small_offset():
    """A 30-degree cap of radius 20 is only 2.7 high: measured from a plane 1 above the wall."""
    rr, rb, solid, _ = _cap_field(30.0)
    ca = oracle.contact_angle(rr, rb, solid, offset=1.0)
    assert ca["ok"] == 1 and abs(ca["theta_deg"] - 30.0) < 1.0


@pytest.mark.parametrize("theta", [60.0, 120.0])
@pytest.mark.parametrize("frac", [-0.5, 0.5])
def test_contact_angle_at_level_on_analytic_caps(theta, frac):
    """Sec. 3 construction at phi = level (Fig. 4's half-max error bars): on the
    cap phi = A tanh((R - d)/w) the level set phi = c is the sphere of radius
    R - w atanh(c/A) about the same centre, so the angle at that level is
    acos((0.5 - z_c)/R_c). The two signs of c give angles about 3.6 deg apart,
    so taking the level with the wrong sign fails."""
    R, width, A = 20.0, 2.0, 0.66
    rr, rb, solid, zc = _cap_field(theta, R=R, width=width)
    level = frac * A
    R_c = R - width * math.atanh(frac)
    theta_c = math.degrees(math.acos((0.5 - zc) / R_c))
    ca = oracle.contact_angle(rr, rb, solid, offset=5.0, level=level)
    assert ca["ok"] == 1
    assert abs(ca["theta_deg"] - theta_c) < 0.5
    assert abs(ca["r_fit"] - R_c) < 0.1
    assert abs(ca["zc"] - zc) < 0.2
    assert abs(theta_c - theta) > 1.5  # the level moves the angle by more than the tolerance


def test_cap_relation_worked_example():
    """Fig. 2 caption: r = (4h^2 + b^2)/(8h); hand-worked values in the golden file."""
    for ex in golden("paper_values.json")["cap_relation_examples"]:
        h, b = ex["h"], ex["b"]
        assert math.isclose((4 * h * h + b * b) / (8 * h), ex["r"], rel_tol=1e-12)
        th = math.degrees(math.atan2(b / 2, ex["r"] - h))
        assert math.isclose(th, ex["theta_deg"], abs_tol=1e-9)


# ---------------------------------------------------------------- surface tension reductions
@pytest.mark.parametrize("plane", ["xy", "xz", "yz"])
def test_pressure_tensor_off_diagonal_on_tilted_lamella(plane):
    """Sec. 4.1 pressure tensor, off-diagonal entries. Lamellae whose normal
    n = (e_i + e_j)/sqrt(2) lies on a face diagonal of the lattice (periodic
    N x N box, densities a function of s = x_i + x_j only). With the W36
    weights (G_k = 36 zeta_k) and tau = 1, every population, weight and
    neighbour psi depends on a velocity only through c.n and zeta_k, and within
    each group of equal c.n the D3Q19 sums of (c.t)^2 and c_k^2 coincide for the
    in-plane tangent t = (e_i - e_j)/sqrt(2) and the third axis e_k. So:
    P_ii = P_jj (the i <-> j mirror), P_ik = P_jk = 0 (the k mirror), and the
    in-plane tangential stress t.P.t = (P_ii + P_jj)/2 - P_ij equals P_kk
    exactly. A wrong index, sign or factor in P_ij breaks the last identity.
    The normal-minus-tangential excess integrated along n is the lamella's
    surface tension (Eq. gammaMechDef), within the lattice's anisotropy of the
    axis-aligned value."""
    N, steps = 48, 2000
    i, j = {"xy": (0, 1), "xz": (0, 2), "yz": (1, 2)}[plane]
    k = 3 - i - j
    dims = [1, 1, 1]
    dims[i] = dims[j] = N
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = (x, y, z)
    s = (c[i] + c[j]) % N
    inside = s < N // 2
    rr, rb = np.where(inside, 0.7, 0.04), np.where(inside, 0.04, 0.7)
    st = oracle.State(rr, rb, W.periodic_mask(nx, ny, nz), CONTACT)
    st.step(steps)
    P = st.pressure_tensor()
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (0, 2): 4, (1, 2): 5}
    Pii, Pjj, Pkk = P[comp[(i, i)]], P[comp[(j, j)]], P[comp[(k, k)]]
    Pij = P[comp[(i, j)]]
    Pik, Pjk = P[comp[tuple(sorted((i, k)))]], P[comp[tuple(sorted((j, k)))]]
    scale = np.abs(Pii).max()
    assert np.abs(Pij).max() > 1e-3 * scale  # the shear entry is far from zero across the interfaces
    assert np.abs(Pii - Pjj).max() < 1e-13 * scale
    assert np.abs(Pik).max() < 1e-13 * scale and np.abs(Pjk).max() < 1e-13 * scale
    PT = 0.5 * (Pii + Pjj) - Pij
    PN = 0.5 * (Pii + Pjj) + Pij
    assert np.abs(PT - Pkk).max() < 1e-13 * scale
    # Eq. gammaMechDef along n: one unit of s is 1/sqrt(2) along the normal; two interfaces
    sf = s.ravel()
    excess = np.array([(PN - PT).ravel()[sf == v].mean() for v in range(N)])
    gamma_tilted = 0.5 * excess.sum() / math.sqrt(2)
    gamma_axis = _surface_tension_flat(_lamella())
    assert math.isclose(gamma_tilted, gamma_axis, rel_tol=0.1)


def test_pressure_profile_on_analytic_planar_field():
    """Eq. gammaMechDef on a synthetic tensor field whose P_N - P_T along z is a
    Gaussian of known integral: the plane means drop in-plane variations of
    zero mean, solid planes are skipped, and the integral is recovered."""
    nx, ny, nz = 6, 5, 40
    A, w, z0, p0 = 0.013, 1.7, 19.3, 0.31
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = A * np.exp(-((z - z0) ** 2) / (2 * w * w))
    P = np.zeros((6, nz, ny, nx))
    P[0] = p0 - s / 3 + 0.02 * np.cos(2 * np.pi * x / nx)
    P[1] = p0 - s / 3 - 0.03 * np.sin(2 * np.pi * y / ny)
    P[2] = p0 + 2 * s / 3
    P[3] = 0.01 * np.cos(2 * np.pi * x / nx)
    solid = W.wall_mask(nx, ny, nz)
    P[:, solid == 1] = 5.0  # must not enter
    phi = np.tanh((z - z0) / 2.0)
    rr, rb = 0.37 + 0.33 * phi, 0.37 - 0.33 * phi
    prof, gsum = oracle.pressure_profile(P, solid, rr, rb)
    assert np.all(prof[[0, -1]] == 0)
    assert np.allclose(prof[1:-1, 7], nx * ny)
    assert np.allclose(prof[1:-1, 3], 0, atol=1e-15)
    assert np.allclose(prof[1:-1, 6], 0.66 * np.tanh((np.arange(1, nz - 1) - z0) / 2.0), atol=1e-14)
    assert math.isclose(gsum, A * w * math.sqrt(2 * math.pi), rel_tol=1e-6)


def _spherical_field(n=40, R=10.0, centre=(20.3, 19.8, 20.1), A=0.01, w=1.5, p0=0.3):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    d = [x - centre[0], y - centre[1], z - centre[2]]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    nv = [di / r for di in d]
    s = A * np.exp(-((r - R) ** 2) / (2 * w * w))
    P = np.zeros((6, n, n, n))
    for c, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        P[c] = s * nv[i] * nv[j] + (p0 - s / 3 if i == j else 0.0)
    phi = np.tanh((R - r) / 2.0)
    return P, 0.37 + 0.33 * phi, 0.37 - 0.33 * phi


def test_pressure_radial_on_analytic_spherical_field():
    """Eq. mechRadGamma on P = p0 I + s(r) (n n - I/3), for which P_N - P_T = s(r)
    exactly: the binned normal/transversal split, the phi = 0 radius and the
    (r/R_s)^2-weighted integral are recovered; the minimum image makes the
    result independent of where the periodic box is cut."""
    n, R, A, w = 40, 10.0, 0.01, 1.5
    c = (20.3, 19.8, 20.1)
    P, rr, rb = _spherical_field(n, R, c, A, w)
    solid = W.periodic_mask(n, n, n)
    bins, gamma, R_s = oracle.pressure_radial(P, solid, rr, rb, c, 1.0, 20, 0.0, 15.0, periodic_z=True)
    assert abs(R_s - R) < 0.05
    rq = np.linspace(0, 15.0, 30001)
    exact = np.trapezoid((rq / R) ** 2 * A * np.exp(-((rq - R) ** 2) / (2 * w * w)), rq)
    assert math.isclose(gamma, exact, rel_tol=0.01)
    assert np.all(bins[:, 0] - bins[:, 1] >= 0)
    # cut the periodic box elsewhere: roll the fields and the centre together
    sh = (7, -5, 11)
    P2 = np.roll(P, sh, axis=(3, 2, 1))
    rr2, rb2 = (np.roll(a, sh, axis=(2, 1, 0)) for a in (rr, rb))
    c2 = ((c[0] + sh[0]) % n, (c[1] + sh[1]) % n, (c[2] + sh[2]) % n)
    bins2, gamma2, R2 = oracle.pressure_radial(P2, solid, rr2, rb2, c2, 1.0, 20, 0.0, 15.0, periodic_z=True)
    assert np.allclose(bins2, bins, rtol=1e-12, atol=1e-15) and math.isclose(gamma2, gamma, rel_tol=1e-12)


def _wall_gamma(phase, w, steps=3000, nz=34):
    """gamma of a fluid-wall interface: a slab of one bulk phase between the two
    walls (two identical interfaces), Eq. gammaMechDef."""
    rr, rb = W.slab_fields(4, 4, nz, phase)
    er, eb = W.wall_split(w)
    st = oracle.State(rr, rb, W.wall_mask(4, 4, nz), Params(g_br=0.08, force_weights=1, force_scale=1.25,
                                                              eta_wall_r=er, eta_wall_b=eb))
    st.step(steps)
    r, b, _, _ = st.moments()
    _, gsum = oracle.pressure_profile(st.pressure_tensor(), st.solid, r, b)
    return 0.5 * gsum


def test_young_planar_wall_tensions_mirror_and_sign():
    """Young's equation with planar tensions (Sec. 4.1): swapping the
    components and the sign of the wall parameter maps liquid-wall onto
    gas-wall exactly, a neutral wall gives gamma_SL = gamma_SG (theta = 90 deg),
    and a wall parameter w > 0, which repels the r-rich liquid, gives theta > 90."""
    w = 0.05
    sl, sg = _wall_gamma("liquid", w), _wall_gamma("gas", w)
    assert math.isclose(_wall_gamma("gas", -w), sl, rel_tol=1e-9, abs_tol=1e-13)
    assert math.isclose(_wall_gamma("liquid", -w), sg, rel_tol=1e-9, abs_tol=1e-13)
    s0l, s0g = _wall_gamma("liquid", 0.0), _wall_gamma("gas", 0.0)
    assert math.isclose(s0l, s0g, rel_tol=1e-9, abs_tol=1e-13)
    assert sl > sg
    assert oracle.young_theta(sg, sl, 0.01) > 90.0
    assert oracle.young_theta(1.0, 1.0, 0.5) == 90.0
    assert oracle.young_theta(0.0, 1.0, 0.5) == 180.0 and oracle.young_theta(1.0, 0.0, 0.5) == 0.0


def test_oracle_counts_non_finite_populations():
    """A NaN fed to the oracle is counted in the conservation sums' non-finite
    slot (the GPU reduction reports the same count as LB_ERR_NAN)."""
    rr, rb = W.droplet_fields(6, 5, 6, 2.0)
    st = oracle.State(rr, rb, W.wall_mask(6, 5, 6), Params())
    st.n[1, 7, 2, 3, 4] = np.nan
    st.n[0, 0, 3, 1, 1] = np.inf
    assert st.moments()[3][5] == 2
    st.n[0, 0, 0, 1, 1] = np.nan  # a solid node holds no populations and is not counted
    assert st.moments()[3][5] == 2
