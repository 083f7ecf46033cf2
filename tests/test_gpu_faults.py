"""Failure detection without a GPU fault: bad inputs and bad states injected
on the host come back as status codes (through LBError), and the context
stays usable afterwards. (The bounded device wait is covered by
test_bounded_wait_reports_timeout_and_context_survives.)"""
import numpy as np
import pytest

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


def _code(lbsc, fn):
    with pytest.raises(lbsc.LBError) as e:
        fn()
    return e.value.code


def test_bad_parameters_and_geometry_are_refused(lbsc):
    rr, rb = W.droplet_fields(16, 12, 10, 4.0)
    lat = lbsc.Lattice(rr, rb).set_params(**CONTACT)
    assert _code(lbsc, lambda: lat.set_params(**CONTACT, tau_r=0.5)) == lbsc.LB_ERR_ARG
    assert _code(lbsc, lambda: lat.set_params(**CONTACT, tau_b=0.3)) == lbsc.LB_ERR_ARG
    assert _code(lbsc, lambda: lat.set_params(**dict(CONTACT, g_br=float("nan")))) == lbsc.LB_ERR_ARG
    assert _code(lbsc, lambda: lat.set_params(**dict(CONTACT, force_weights=7))) == lbsc.LB_ERR_ARG
    assert _code(lbsc, lambda: lat.set_geometry(np.ones((10, 12, 16), np.uint8))) == lbsc.LB_ERR_ARG
    assert _code(lbsc, lambda: lat.set_tiling(8, 1, 0)) == lbsc.LB_ERR_ARG  # 12 rows in one 8-row tile
    assert _code(lbsc, lambda: lat.set_tiling(6, 0, 0)) == lbsc.LB_ERR_ARG
    assert _code(lbsc, lambda: lat.step(-1)) == lbsc.LB_ERR_ARG
    # the context still works, with the last accepted parameters
    lat.step(10)
    assert lat.conservation()[7] == 10
    lat.close()


def test_non_finite_state_is_reported_and_recovered(lbsc):
    rr, rb = W.droplet_fields(16, 12, 10, 4.0)
    lat = lbsc.Lattice(rr, rb).set_params(**CONTACT)
    lat.step(5)
    good = lat.save()
    n = lat.populations()
    n[0, 3, 4, 5, 6] = np.nan
    lat.set_populations(n)
    assert _code(lbsc, lambda: lat.conservation()) == lbsc.LB_ERR_NAN
    lat.load(good)
    cons = lat.conservation()
    assert cons[5] == 0 and cons[7] == 5
    # a truncated or foreign checkpoint is refused and leaves the state alone
    assert _code(lbsc, lambda: lat.load(good[:64])) == lbsc.LB_ERR_ARG
    assert _code(lbsc, lambda: lat.load(b"X" * len(good))) == lbsc.LB_ERR_ARG
    assert np.array_equal(lat.conservation(), cons)
    lat.close()


def test_unsupported_requests_are_refused(lbsc):
    nx, ny, nz = 16, 12, 10
    solid = W.wall_mask(nx, ny, nz)
    solid[1:3, 4:6, 4:6] = 1
    rr, rb = W.droplet_fields(nx, ny, nz, 4.0)
    lat = lbsc.Lattice(rr, rb).set_geometry(solid).set_params(**CONTACT)
    assert _code(lbsc, lambda: lat.step_backward(10, 5)) == lbsc.LB_ERR_UNSUPPORTED
    lat.close()
