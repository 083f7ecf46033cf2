"""The z-slab decomposition on the GPU (through the C ABI): slabs stepped one
step at a time with their faces exchanged after each step hold exactly the
whole lattice's populations (bitwise, FP32 and BF16 storage), match the FP64
oracle within the parity bar, and the message path (pack into a device
buffer, unpack from it; also host-staged between two processes over gloo)
equals the lattice-to-lattice exchange."""
import ctypes
import os
import socket

import numpy as np
import pytest

import oracle
from paper_0910_3915_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CONTACT = dict(g_br=0.08, force_weights=1, force_scale=1.25, eta_wall_r=-0.05, eta_wall_b=0.05)


@pytest.fixture(scope="module")
def lbsc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_3915_gb300 import lbsc as m
    m.load()
    return m


def _whole(lbsc, rr, rb, steps, precision="f32"):
    lat = lbsc.Lattice(rr, rb, precision).set_params(**CONTACT)
    lat.step(steps)
    n = lat.populations()
    m = lat.moments()
    lat.close()
    return n, m


@pytest.mark.parametrize("nslab", [2, 3])
def test_slabs_bitwise_equal_whole_lattice_and_oracle(lbsc, nslab):
    from paper_0910_3915_gb300.slabs import Slabs
    nx, ny, nz, steps = 48, 40, 37, 100
    rr, rb = W.droplet_fields(nx, ny, nz, 11.0, seed=4)
    n_whole, m_whole = _whole(lbsc, rr, rb, steps)
    with Slabs(rr, rb, nslab).set_params(**CONTACT) as s:
        s.step(steps)
        n = s.populations()
        m = s.moments()
    fl = W.wall_mask(nx, ny, nz) == 0
    assert np.array_equal(n[:, :, 1:-1], n_whole[:, :, 1:-1])
    assert np.array_equal(m[0][fl], m_whole[0][fl]) and np.array_equal(m[1][fl], m_whole[1][fl])
    assert m[3][6] == m_whole[3][6] == nx * ny * (nz - 2)
    assert np.allclose(m[3][:5], m_whole[3][:5], rtol=1e-12, atol=1e-12 * m_whole[3][1])
    o = oracle.State(rr, rb, W.wall_mask(nx, ny, nz), oracle.Params(**CONTACT)).step(steps).moments()
    err = max(np.max(np.abs(m[a] - o[a])[fl] / np.abs(o[a])[fl]) for a in (0, 1))
    assert err <= 1e-5, err


def test_bf16_slabs_bitwise_equal_whole_lattice(lbsc):
    """16-bit storage: the slabs share the whole lattice's deviation references
    and key the rounding dither by the node's place in the whole lattice."""
    from paper_0910_3915_gb300.slabs import Slabs
    nx, ny, nz, steps = 40, 32, 30, 60
    rr, rb = W.droplet_fields(nx, ny, nz, 9.0, seed=6)
    n_whole, _ = _whole(lbsc, rr, rb, steps, "bf16")
    with Slabs(rr, rb, 2, "bf16").set_params(**CONTACT) as s:
        s.step(steps)
        n = s.populations()
    assert np.array_equal(n[:, :, 1:-1], n_whole[:, :, 1:-1])


def test_message_path_equals_direct_exchange(lbsc):
    """lb_halo_pack into a device buffer and lb_halo_unpack from it, face by
    face, give the same state as the one-kernel lattice-to-lattice exchange."""
    import torch
    from paper_0910_3915_gb300.slabs import Slabs
    nx, ny, nz, steps = 36, 20, 25, 30
    rr, rb = W.droplet_fields(nx, ny, nz, 8.0, seed=9)
    lib = lbsc.load()
    with Slabs(rr, rb, 3).set_params(**CONTACT) as direct, Slabs(rr, rb, 3).set_params(**CONTACT) as msgs:
        direct.step(steps)
        nb = ctypes.c_size_t()
        assert lib.lb_halo_bytes(msgs.slabs[0]._ctx, ctypes.byref(nb)) == lbsc.LB_OK
        assert nb.value == 38 * nx * ny * 4
        up = [torch.empty(nb.value, dtype=torch.uint8, device="cuda") for _ in range(2)]
        dn = [torch.empty(nb.value, dtype=torch.uint8, device="cuda") for _ in range(2)]
        for _ in range(steps):
            for s in msgs.slabs:
                s.step(1)
            for i in range(2):
                a, b = msgs.slabs[i]._ctx, msgs.slabs[i + 1]._ctx
                assert lib.lb_halo_pack(a, 1, ctypes.c_void_p(up[i].data_ptr())) == lbsc.LB_OK
                assert lib.lb_halo_pack(b, 0, ctypes.c_void_p(dn[i].data_ptr())) == lbsc.LB_OK
            for i in range(2):
                a, b = msgs.slabs[i]._ctx, msgs.slabs[i + 1]._ctx
                assert lib.lb_halo_unpack(b, 0, ctypes.c_void_p(up[i].data_ptr())) == lbsc.LB_OK
                assert lib.lb_halo_unpack(a, 1, ctypes.c_void_p(dn[i].data_ptr())) == lbsc.LB_OK
        assert np.array_equal(msgs.populations(), direct.populations())
        # a face without a neighbour has no halo plane to pack
        assert lib.lb_halo_pack(msgs.slabs[0]._ctx, 0, ctypes.c_void_p(up[0].data_ptr())) == lbsc.LB_ERR_STATE


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        from paper_0910_3915_gb300.slabs import DistributedSlab
        nx, ny, nz = 32, 24, 26
        rr, rb = W.droplet_fields(nx, ny, nz, 7.0, seed=12)
        s = DistributedSlab(rr, rb, "f32", staged=True).set_params(**CONTACT)
        s.step(40)
        cons = s.conservation()
        n = s.lat.populations()[:, :, 1:-1]
        parts = [None] * world
        dist.all_gather_object(parts, n)
        s.close()
        out[rank] = (cons, parts)
    finally:
        dist.destroy_process_group()


def test_distributed_slabs_host_staged_two_processes(lbsc):
    """Two processes, one slab each, on this GPU; the faces go through host
    memory over gloo (no kernel waits on another process). The gathered owned
    planes equal the whole lattice's; the FP64 sums are the same bits on both ranks."""
    import torch.multiprocessing as mp
    nx, ny, nz = 32, 24, 26
    rr, rb = W.droplet_fields(nx, ny, nz, 7.0, seed=12)
    n_whole, m_whole = _whole(lbsc, rr, rb, 40)
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    got = np.concatenate(res[0][1], axis=2)
    assert np.array_equal(got, n_whole[:, :, 1:-1])
    assert np.array_equal(res[0][0], res[1][0])
    assert np.allclose(res[0][0][:2], m_whole[3][:2], rtol=1e-12, atol=0)


def test_single_slab_and_thin_slabs(lbsc):
    """Degenerate splits: one slab (no halo planes: the whole lattice) and slabs
    of two owned planes each (the thinnest a slab with two neighbours may be)
    stay bitwise equal to the whole lattice; a one-plane slab between two
    neighbours is refused."""
    from paper_0910_3915_gb300.slabs import Slabs
    nx, ny, nz, steps = 32, 20, 8, 25
    rr, rb = W.droplet_fields(nx, ny, nz, 5.0, seed=14)
    n_whole, _ = _whole(lbsc, rr, rb, steps)
    with pytest.raises(lbsc.LBError):
        lbsc.Lattice(rr[:3], rb[:3], slab=(lbsc.LB_HALO_BELOW | lbsc.LB_HALO_ABOVE, 2, None))
    for nslab in (1, (nz - 2) // 2):
        with Slabs(rr, rb, nslab).set_params(**CONTACT) as s:
            s.step(steps)
            assert np.array_equal(s.populations()[:, :, 1:-1], n_whole[:, :, 1:-1]), nslab


def test_reset_restarts_bitwise_and_rejects_bad_densities(lbsc):
    """lb_reset: a lattice restarted from its initial densities repeats its run
    bit for bit (the step counter, which keys 16-bit rounding, restarts too); a
    negative or non-finite density is rejected and a later reset still works."""
    nx, ny, nz = 36, 28, 20
    rr, rb = W.droplet_fields(nx, ny, nz, 6.0, seed=8)
    for precision in ("f32", "bf16"):
        lat = lbsc.Lattice(rr, rb, precision).set_params(**CONTACT)
        lat.step(30)
        first = lat.populations()
        lat.reset(rr, rb)
        assert lat.conservation()[7] == 0
        lat.step(30)
        assert np.array_equal(lat.populations(), first)
        bad = rr.copy()
        bad[3, 4, 5] = -0.1
        with pytest.raises(lbsc.LBError) as e:
            lat.reset(bad, rb)
        assert e.value.code == lbsc.LB_ERR_ARG
        bad[3, 4, 5] = np.nan
        with pytest.raises(lbsc.LBError):
            lat.reset(rr, bad)
        lat.reset(rr, rb).step(30)
        assert np.array_equal(lat.populations(), first)
        lat.close()
