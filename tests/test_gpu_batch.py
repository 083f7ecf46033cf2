"""The batched sweep: many droplet lattices of uneven sizes and parameters in
one persistent launch per step must give exactly what each lattice gives on
its own, and match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_0910_3915_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbsc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_3915_gb300 import lbsc as m
    m.load()
    return m


def _boxes(n=6, edges=(24, 33, 40, 48), seed=3):
    boxes = W.sweep_boxes(n, seed=seed, edges=edges)
    fields, params = [], []
    for bx in boxes:
        fields.append(W.droplet_fields(bx.edge, bx.edge, bx.edge, bx.radius, seed=bx.seed))
        er, eb = W.wall_split(bx.w)
        params.append(dict(g_br=bx.g_br, eta_wall_r=er, eta_wall_b=eb, force_weights=1, force_scale=1.25))
    return boxes, fields, params


@pytest.mark.parametrize("variant", ["auto", "ldg"])
@pytest.mark.parametrize("precision", ["f32", "f16", "bf16"])
def test_batch_equals_individual_lattices_bitwise(lbsc, precision, variant):
    """The TMA-staged batch kernel (auto) and the load-from-global one, for
    each storage precision, against each box stepped alone."""
    boxes, fields, params = _boxes()
    batch = lbsc.Batch(fields, [lbsc.Params(**p) for p in params], precision).set_step_variant(variant)
    batch.step(70)  # two graph replays of 32 steps plus 6 single launches
    for i, ((rr, rb), p) in enumerate(zip(fields, params)):
        lat = lbsc.Lattice(rr, rb, precision).set_params(**p)
        lat.step(70)
        ref = lat.populations()
        got = batch.box(i).populations()
        e = boxes[i].edge
        fl = (W.wall_mask(e, e, e) == 0)[None, None]
        assert np.array_equal(np.where(fl, got, 0), np.where(fl, ref, 0)), i
        lat.close()
    batch.close()


def test_batch_schedules_agree_and_match_oracle(lbsc):
    boxes, fields, params = _boxes(n=4, edges=(20, 27), seed=5)
    a = lbsc.Batch(fields, [lbsc.Params(**p) for p in params])
    b = lbsc.Batch(fields, [lbsc.Params(**p) for p in params]).set_schedule(4, 7, 1)
    c = lbsc.Batch(fields, [lbsc.Params(**p) for p in params]).set_step_variant("ldg").set_schedule(16, 40)
    a.step(100)
    b.step(100)
    c.step(100)
    for i in range(len(boxes)):
        ra, rb_, rc = a.box(i).moments()[:2], b.box(i).moments()[:2], c.box(i).moments()[:2]
        assert np.array_equal(ra[0], rb_[0]) and np.array_equal(ra[1], rb_[1])
        assert np.array_equal(ra[0], rc[0]) and np.array_equal(ra[1], rc[1])
    c.close()
    i = 1
    e = boxes[i].edge
    solid = W.wall_mask(e, e, e)
    o = oracle.State(*fields[i], solid, oracle.Params(**params[i])).step(100).moments()
    fl = solid == 0
    ra = a.box(i).moments()
    err = max(np.max(np.abs(ra[k] - o[k])[fl] / np.abs(o[k])[fl]) for k in (0, 1))
    assert err <= 1e-5
    cons = a.conservation()
    assert cons.shape == (4, 8) and np.all(cons[:, 7] == 100)
    angles = a.contact_angles(3.0)
    assert len(angles) == 4
    a.close()
    b.close()


def test_batch_refuses_a_box_stepped_alone(lbsc):
    _, fields, params = _boxes(n=2, edges=(16,), seed=1)
    batch = lbsc.Batch(fields, [lbsc.Params(**p) for p in params])
    with pytest.raises(lbsc.LBError):
        batch.box(0).step(1)
    batch.step(3)
    batch.close()
