"""The hand-written adjoint (lb_step_backward): the gradient of a droplet
observable with respect to the wall pseudo-densities, against central finite
differences of the FP64 oracle (the FP64 CPU reference gradient), against
finite differences of the GPU forward run, and independent of the
checkpoint interval."""
import math

import numpy as np
import pytest

import oracle
from paper_0910_3915_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CONTACT = dict(g_br=0.08, force_weights=1, force_scale=1.25)
EPS = 0.05


@pytest.fixture(scope="module")
def lbsc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_3915_gb300 import lbsc as m
    m.load()
    return m


def observable(rr, rb, obs):
    """The three observables, written out in numpy from their definitions."""
    nz = rr.shape[0]
    z = np.arange(nz)[:, None, None] - 0.5 + 0 * rr
    fl = np.zeros_like(rr, dtype=bool)
    fl[1:-1] = True
    if obs == "com":
        return float((z * rr)[fl].sum() / rr[fl].sum())
    w = 1.0 / (1.0 + np.exp(-(rr - rb) / EPS))
    if obs == "com_soft":
        return float((z * w)[fl].sum() / w[fl].sum())
    return float(w[1].sum())


def oracle_J(rr, rb, prm, steps, obs):
    st = oracle.State(rr, rb, W.wall_mask(*rr.shape[::-1]), oracle.Params(**prm)).step(steps)
    r, b, _, _ = st.moments()
    return observable(r, b, obs)


@pytest.mark.parametrize("obs", ["com_soft", "com", "wetted"])
def test_adjoint_against_fp64_oracle_central_differences(lbsc, obs):
    nx, ny, nz, steps = 20, 18, 14, 40
    rr, rb = W.droplet_fields(nx, ny, nz, 5.0, seed=2)
    w = 0.03
    prm = dict(CONTACT, eta_wall_r=-w, eta_wall_b=w)
    lat = lbsc.Lattice(rr, rb).set_params(**prm)
    J, g = lat.step_backward(steps, ckpt_every=15, observable=obs)
    lat.close()
    assert math.isclose(J, oracle_J(rr, rb, prm, steps, obs), rel_tol=1e-5)
    h = 1e-4
    fd = []
    for comp in ("eta_wall_r", "eta_wall_b"):
        jp = oracle_J(rr, rb, dict(prm, **{comp: prm[comp] + h}), steps, obs)
        jm = oracle_J(rr, rb, dict(prm, **{comp: prm[comp] - h}), steps, obs)
        fd.append((jp - jm) / (2 * h))
    fd = np.array(fd)
    assert np.abs(fd).max() > 1e-4  # the observable does depend on the wall
    assert np.allclose(g, fd, rtol=1e-3, atol=1e-3 * np.abs(fd).max())


def test_adjoint_with_unequal_tau_and_checkpoint_independence(lbsc):
    nx, ny, nz, steps = 16, 16, 12, 30
    rr, rb = W.droplet_fields(nx, ny, nz, 4.5, seed=7)
    prm = dict(CONTACT, tau_r=0.85, tau_b=1.2, eta_wall_r=0.02, eta_wall_b=-0.02)
    grads = []
    for ck in (7, 30, 100):
        lat = lbsc.Lattice(rr, rb).set_params(**prm)
        grads.append(lat.step_backward(steps, ckpt_every=ck, observable="com_soft"))
        lat.close()
    for J, g in grads[1:]:
        assert J == grads[0][0] and np.array_equal(g, grads[0][1])
    h = 1e-4
    fd = []
    for comp in ("eta_wall_r", "eta_wall_b"):
        jp = oracle_J(rr, rb, dict(prm, **{comp: prm[comp] + h}), steps, "com_soft")
        jm = oracle_J(rr, rb, dict(prm, **{comp: prm[comp] - h}), steps, "com_soft")
        fd.append((jp - jm) / (2 * h))
    assert np.allclose(grads[0][1], fd, rtol=1e-3, atol=1e-3 * np.abs(fd).max())


def test_adjoint_against_gpu_finite_differences_full_config(lbsc):
    """64^3, R = 16, 200 steps with checkpoints every 100: the adjoint against
    FP32 central differences of the GPU forward run (h = 1e-2: FP32 noise)."""
    nx = ny = nz = 64
    rr, rb = W.droplet_fields(nx, ny, nz, 16.0, seed=0)
    prm = dict(CONTACT, eta_wall_r=0.0, eta_wall_b=0.0)
    lat = lbsc.Lattice(rr, rb).set_params(**prm)
    s0 = lat.save()
    J, g = lat.step_backward(200, ckpt_every=100, observable="com_soft")
    h = 1e-2
    fd = []
    for comp in ("eta_wall_r", "eta_wall_b"):
        js = []
        for sgn in (1, -1):
            lat.load(s0)
            lat.set_params(**dict(prm, **{comp: prm[comp] + sgn * h}))
            lat.step(200)
            js.append(lat.observable("com_soft"))
        fd.append((js[0] - js[1]) / (2 * h))
    lat.close()
    assert np.allclose(g, fd, rtol=2e-2, atol=2e-2 * np.abs(fd).max())


@pytest.mark.slow
def test_adjoint_full_config_against_fp64_oracle_central_differences(lbsc):
    """The adjoint calibration configuration itself: 64^3, R = 16, g_br = 0.08,
    wall parameters at 0, 2000 steps with checkpoints every 100. The gradient
    of the droplet's centre-of-mass height with respect to both wall
    pseudo-densities against central differences (h = 1e-4) of the FP64 oracle
    over the same 2000 steps: within 1e-3 relative."""
    nx = ny = nz = 64
    steps, ckpt, obs = 2000, 100, "com"
    rr, rb = W.droplet_fields(nx, ny, nz, 16.0, seed=0)
    prm = dict(CONTACT, eta_wall_r=0.0, eta_wall_b=0.0)
    lat = lbsc.Lattice(rr, rb).set_params(**prm)
    J, g = lat.step_backward(steps, ckpt_every=ckpt, observable=obs)
    lat.close()
    h = 1e-4
    fd = []
    for comp in ("eta_wall_r", "eta_wall_b"):
        jp = oracle_J(rr, rb, dict(prm, **{comp: prm[comp] + h}), steps, obs)
        jm = oracle_J(rr, rb, dict(prm, **{comp: prm[comp] - h}), steps, obs)
        fd.append((jp - jm) / (2 * h))
    fd = np.array(fd)
    j0 = oracle_J(rr, rb, prm, steps, obs)
    assert math.isclose(J, j0, rel_tol=1e-4), (J, j0)
    assert np.abs(fd).max() > 1e-3  # the centre of mass does move with the wall
    rel = float(np.max(np.abs(np.asarray(g) - fd)) / np.max(np.abs(fd)))
    print(f"adjoint 64^3 x 2000 steps: gradient {list(g)}, FP64 oracle central differences {list(fd)}, "
          f"max relative difference {rel:.2e}")
    assert np.allclose(g, fd, rtol=1e-3, atol=1e-3 * np.abs(fd).max()), (g, fd)


def test_autograd_function_chain_rule(lbsc):
    torch = pytest.importorskip("torch")
    nx, ny, nz = 16, 16, 12
    rr, rb = W.droplet_fields(nx, ny, nz, 4.5, seed=3)
    lat = lbsc.Lattice(rr, rb).set_params(**CONTACT)
    s0 = lat.save()
    f = lbsc.wall_gradient(lat, s0, lbsc.Params(**CONTACT), nsteps=20, ckpt_every=10)
    w = torch.tensor(0.02, dtype=torch.float64, requires_grad=True)
    J = f(w)
    J.backward()
    lat.load(s0)
    lat.set_params(**dict(CONTACT, eta_wall_r=-0.02, eta_wall_b=0.02))
    J2, g = lat.step_backward(20, 10, "com_soft")
    assert J.item() == J2
    assert math.isclose(w.grad.item(), g[1] - g[0], rel_tol=1e-12)
    lat.close()
