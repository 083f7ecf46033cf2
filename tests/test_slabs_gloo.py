"""Host logic of the z-slab decomposition on CPU ranks (gloo, world size 2 and 3).

Every rank steps its slab with the FP64 oracle: the slab's planes with the
wall layers of the whole lattice where it has them and fluid halo planes where
it has neighbours, in a z-periodic box. The oracle then updates the halo
planes too, but everything a halo plane's own update writes (into itself and
into the crossing slots of the owned boundary plane) is overwritten by the
exchange, exactly as the slab kernel leaves those values to it. The faces
travel as host messages (pack_host / unpack_host, the message layout of
lb_halo_pack) by point-to-point send and receive; the FP64 conservation sums
are added in rank order. The gathered owned planes must equal the oracle's
whole-lattice run bit for bit. No GPU is involved.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_0910_3915_gb300 import slabs  # noqa: E402
from paper_0910_3915_gb300 import workloads as W  # noqa: E402

PRM = dict(g_br=0.08, force_weights=1, force_scale=1.25, eta_wall_r=-0.04, eta_wall_b=0.04)
DIMS = (14, 12, 19)  # nx, ny, nz: 17 fluid planes, uneven slabs
STEPS = 12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fields():
    nx, ny, nz = DIMS
    return W.droplet_fields(nx, ny, nz, 4.5, seed=11)


def _rank_main(rank, world_size, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        nx, ny, nz = DIMS
        rr, rb = _fields()
        z0, z1 = slabs.split(nz, world_size)[rank]
        solid = np.zeros((z1 - z0 + 2, ny, nx), np.uint8)
        if rank == 0:
            solid[0] = 1
        if rank == world_size - 1:
            solid[-1] = 1
        st = oracle.State(rr[z0 - 1:z1 + 1], rb[z0 - 1:z1 + 1], solid, oracle.Params(**PRM))
        for _ in range(STEPS):
            st.step(1)
            send = [torch.from_numpy(slabs.pack_host(st.n, f)) for f in (0, 1)]
            got = slabs.exchange_messages(send[0], send[1], rank, world_size)
            for f in (0, 1):
                if got[f] is not None:
                    slabs.unpack_host(st.n, f, got[f].numpy())
        # each rank's FP64 masses over its owned planes (the halo planes are the neighbours')
        own = st.n[:, :, 1:-1]
        cons = slabs.sum_in_rank_order(np.array([own[0].sum(), own[1].sum()]))
        parts = [None] * world_size
        dist.all_gather_object(parts, (z0, z1, st.n[:, :, 1:-1].copy()))
        out[rank] = (cons, parts)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world_size", [2, 3])
def test_slab_exchange_matches_whole_lattice_bitwise(world_size):
    nx, ny, nz = DIMS
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world_size, port, out), nprocs=world_size, join=True)
        res = dict(out)
    rr, rb = _fields()
    ref = oracle.State(rr, rb, W.wall_mask(nx, ny, nz), oracle.Params(**PRM)).step(STEPS)
    whole = ref.n[:, :, 1:-1]
    cons0, parts = res[0]
    got = np.concatenate([p[2] for p in parts], axis=2)
    assert [p[:2] for p in parts] == slabs.split(nz, world_size)
    assert np.array_equal(got, whole)
    rcons = ref.moments()[3]
    assert np.allclose(cons0, rcons[:2], rtol=1e-12, atol=0)
    for r in range(1, world_size):  # every rank holds the same bits
        assert np.array_equal(res[r][0], cons0)


def test_messages_carry_the_crossing_populations_and_the_boundary_plane():
    """Message layout on a labelled array: the outgoing message of a face holds
    the crossing velocities from the halo plane and the boundary plane's
    non-opposing values; applying it to the neighbour fills exactly the slots
    its own step leaves to the exchange."""
    nz, ny, nx = 6, 3, 4
    n = np.arange(2 * 19 * nz * ny * nx, dtype=np.float64).reshape(2, 19, nz, ny, nx)
    up = slabs.pack_host(n, 1)
    assert up.shape == (slabs.ENTRIES, ny, nx)
    assert np.array_equal(up[0], n[0, 5, nz - 1]) and np.array_equal(up[9], n[1, 18, nz - 1])
    assert np.array_equal(up[10], n[0, 0, nz - 2]) and np.array_equal(up[37], n[1, 18, nz - 2])
    dn = slabs.pack_host(n, 0)
    assert np.array_equal(dn[0], n[0, 6, 0]) and np.array_equal(dn[23], n[0, 17, 1])
    # the receiver above: first owned plane takes the up-crossing, bottom halo the c_z >= 0 values
    m = np.zeros_like(n)
    slabs.unpack_host(m, 0, up)
    written = np.argwhere(m.reshape(2, 19, nz, -1).any(axis=3))
    cz = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1])
    for a, k, z in written:
        assert (z == 1 and cz[k] == 1) or (z == 0 and cz[k] >= 0)
    assert len(written) == slabs.ENTRIES
    # velocity sets: the two crossing sets are opposite, flat has c_z = 0
    assert all(cz[k] == 1 for k in slabs.UP) and all(cz[k] == -1 for k in slabs.DOWN)
    assert all(cz[k] == 0 for k in slabs.FLAT) and len(set(slabs.FLAT + slabs.UP + slabs.DOWN)) == 19
