"""A lattice decomposed into z slabs, with one exchange per step.

The update of a node needs only its nearest neighbours (Sec. 2), so the
lattice splits into slabs of whole z planes. A slab is a library context
whose planes 1..nz-2 it owns; its plane 0 and plane nz-1 are the lattice's
solid wall layers or halo planes, copies of the neighbouring slab's boundary
plane (include/lbsc.h, "z-slab decomposition"). After every step each face
carries one message each way: the 5 populations per component that crossed
it, and the 28 values of the sender's boundary plane that the receiver's halo
plane takes (its other 10 it holds already: the populations it pushed across
itself). Each node then computes exactly what it computes in the whole
lattice, so the decomposed run is bitwise equal to it.

- ``Slabs``: all slabs on the current device in one process, stepped by
  lb_slabs_step (every slab steps, then every face is exchanged lattice to
  lattice by one kernel).
- ``DistributedSlab``: one slab per rank of a torch.distributed group; the
  faces travel as messages (lb_halo_pack / lb_halo_unpack) by point-to-point
  send and receive, device buffers for NCCL or host-staged for gloo. The FP64
  conservation sums are gathered and added in rank order, so every rank gets
  the same bits.
- ``pack_host`` / ``unpack_host``: the same messages on host arrays in the
  layout of lb_get_populations ([component][k][z][y][x]), entry for entry.
"""
from __future__ import annotations

import ctypes

import numpy as np

UP = (5, 11, 14, 15, 18)      # c_z = +1: (0,0,1), (1,0,1), (-1,0,1), (0,1,1), (0,-1,1)
DOWN = (6, 12, 13, 16, 17)    # c_z = -1: the opposites, in the same order
FLAT = (0, 1, 2, 3, 4, 7, 8, 9, 10)  # c_z = 0
ENTRIES = 38                  # 2 x 5 crossing + 2 x 14 boundary-plane values per face node


def split(nz: int, nslab: int):
    """Owned plane ranges [z0, z1) of the whole lattice's fluid planes 1..nz-2,
    as even as possible. Every slab owns at least two planes when there are
    more than one: a slab sends its boundary plane right after its own step, so
    that plane's populations must all come from the slab itself (or the wall)."""
    nf = nz - 2
    if nslab < 1 or (nslab > 1 and 2 * nslab > nf) or nslab > nf:
        raise ValueError("need 1 <= nslab and at least two fluid planes per slab")
    return [(1 + i * nf // nslab, 1 + (i + 1) * nf // nslab) for i in range(nslab)]


def halo_flags(i: int, nslab: int) -> int:
    from .lbsc import LB_HALO_ABOVE, LB_HALO_BELOW
    return (LB_HALO_BELOW if i > 0 else 0) | (LB_HALO_ABOVE if i + 1 < nslab else 0)


def references(rho_r, rho_b):
    """The whole lattice's 16-bit deviation references: the mean initial
    density of each component over the fluid planes, summed node after node in
    storage order (as lb_init forms them), so every slab encodes alike."""
    rr, rb = np.asarray(rho_r, np.float64), np.asarray(rho_b, np.float64)
    cnt = rr[1:-1].size
    return (float(np.cumsum(rr[1:-1].ravel())[-1] / cnt), float(np.cumsum(rb[1:-1].ravel())[-1] / cnt))


def _entries(nz: int, face: int, unpack: bool):
    """(plane, component, velocity) of each message entry, in message order."""
    if face == 0:
        zc, zp, d = (1, 0, +1) if unpack else (0, 1, -1)
    else:
        zc, zp, d = (nz - 2, nz - 1, -1) if unpack else (nz - 1, nz - 2, +1)
    cross = UP if d > 0 else DOWN
    out = [(zc, a, cross[i]) for a in (0, 1) for i in range(5)]
    out += [(zp, a, k) for a in (0, 1) for k in FLAT + cross]
    return out


def pack_host(n: np.ndarray, face: int) -> np.ndarray:
    """Outgoing message (38, ny, nx) of face 0 (below) or 1 (above) from a slab's
    populations n (2, 19, nz, ny, nx)."""
    return np.stack([n[a, k, z] for z, a, k in _entries(n.shape[2], face, False)])


def unpack_host(n: np.ndarray, face: int, msg: np.ndarray) -> None:
    """Apply the neighbour's message on face 0 (below) or 1 (above) to n in place."""
    for j, (z, a, k) in enumerate(_entries(n.shape[2], face, True)):
        n[a, k, z] = msg[j]


def exchange_messages(send_below, send_above, rank: int, world: int, group=None):
    """Send each message to the neighbour on its face and receive theirs:
    returns (from_below, from_above), None where there is no neighbour. The
    sends and receives of a rank are posted together (batch_isend_irecv), so no
    rank waits on a send whose receive is not yet posted."""
    import torch
    import torch.distributed as dist

    ops, from_below, from_above = [], None, None
    if rank > 0:
        from_below = torch.empty_like(send_below)
        ops += [dist.P2POp(dist.isend, send_below, rank - 1, group),
                dist.P2POp(dist.irecv, from_below, rank - 1, group)]
    if rank + 1 < world:
        from_above = torch.empty_like(send_above)
        ops += [dist.P2POp(dist.isend, send_above, rank + 1, group),
                dist.P2POp(dist.irecv, from_above, rank + 1, group)]
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    return from_below, from_above


def sum_in_rank_order(local: np.ndarray, group=None, device=None) -> np.ndarray:
    """FP64 sum over the ranks of a vector, added in rank order (the same bits on every rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return np.asarray(local, np.float64).copy()
    t = torch.as_tensor(np.asarray(local, np.float64), device=device)
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    out = np.zeros_like(np.asarray(local, np.float64))
    for p in parts:
        out = out + p.cpu().numpy()
    return out


class Slabs:
    """A lattice split into `nslab` z slabs on the current device (one process).

    rho_r, rho_b: the whole lattice's initial densities (nz, ny, nx), walls at
    z = 0 and nz-1. Each slab holds its owned planes plus a halo or wall plane
    on each side; ``step`` runs lb_slabs_step."""

    def __init__(self, rho_r, rho_b, nslab: int, precision: str = "f32", stream=None):
        from .lbsc import Lattice

        rr, rb = np.asarray(rho_r, np.float64), np.asarray(rho_b, np.float64)
        self.nz, self.ny, self.nx = rr.shape
        self.bounds = split(self.nz, nslab)
        ref = references(rr, rb) if precision != "f32" else None
        self.slabs = []
        for i, (z0, z1) in enumerate(self.bounds):
            self.slabs.append(Lattice(rr[z0 - 1:z1 + 1], rb[z0 - 1:z1 + 1], precision, stream,
                                      slab=(halo_flags(i, nslab), z0 - 1, ref)))
        self.precision = precision
        self._arr = (ctypes.c_void_p * nslab)(*[s._ctx.value for s in self.slabs])

    @property
    def shape(self):
        return self.nz, self.ny, self.nx

    def set_params(self, params=None, **kw) -> "Slabs":
        for s in self.slabs:
            s.set_params(params, **kw)
        return self

    def set_tiling(self, tile_y: int, y_tiles: int = 0, z_segments: int = 0) -> "Slabs":
        for s in self.slabs:
            s.set_tiling(tile_y, y_tiles, z_segments)
        return self

    def step(self, n: int = 1) -> "Slabs":
        from .lbsc import _check, load
        _check(load().lb_slabs_step(self._arr, len(self.slabs), int(n)), self.slabs[0]._ctx)
        return self

    def sync(self):
        for s in self.slabs:
            s.sync()

    def _gather(self, parts):
        """Whole-lattice array from per-slab arrays (..., nz_slab, ny, nx): the owned
        planes of every slab, the wall planes from the end slabs."""
        out = [parts[0][..., :1, :, :]]
        out += [p[..., 1:-1, :, :] for p in parts]
        out.append(parts[-1][..., -1:, :, :])
        return np.concatenate(out, axis=-3)

    def moments(self):
        """(rho_r, rho_b, None, cons[8]) of the whole lattice."""
        ms = [s.moments() for s in self.slabs]
        return self._gather([m[0] for m in ms]), self._gather([m[1] for m in ms]), None, self.conservation()

    def populations(self) -> np.ndarray:
        return self._gather([s.populations() for s in self.slabs])

    def conservation(self) -> np.ndarray:
        """FP64 sums over the owned planes of the slabs, added in slab order."""
        out = np.zeros(8)
        for s in self.slabs:
            c = s.conservation()
            out[:7] += c[:7]
            out[7] = c[7]
        return out

    def close(self):
        for s in self.slabs:
            s.close()
        self.slabs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class DistributedSlab:
    """This rank's slab of a lattice split over a torch.distributed group, one
    slab per rank (and per GPU). ``staged``: messages go through host memory
    (for the gloo backend); otherwise they stay in device buffers (NCCL)."""

    def __init__(self, rho_r, rho_b, precision: str = "f32", group=None, staged: bool = False, stream=None):
        import torch
        import torch.distributed as dist

        from .lbsc import Lattice, load

        self.group = group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        rr, rb = np.asarray(rho_r, np.float64), np.asarray(rho_b, np.float64)
        self.nz, self.ny, self.nx = rr.shape
        self.bounds = split(self.nz, self.world)
        z0, z1 = self.bounds[self.rank]
        ref = references(rr, rb) if precision != "f32" else None
        self.lat = Lattice(rr[z0 - 1:z1 + 1], rb[z0 - 1:z1 + 1], precision, stream,
                           slab=(halo_flags(self.rank, self.world), z0 - 1, ref))
        nbytes = ctypes.c_size_t()
        load().lb_halo_bytes(self.lat._ctx, ctypes.byref(nbytes))
        self.staged = staged
        self._out = [torch.empty(nbytes.value, dtype=torch.uint8, device="cuda") for _ in range(2)]
        self._dev = None if staged else "cuda"

    def set_params(self, params=None, **kw) -> "DistributedSlab":
        self.lat.set_params(params, **kw)
        return self

    def step(self, n: int = 1) -> "DistributedSlab":
        import torch

        from .lbsc import _check, load

        lib = load()
        ctx = self.lat._ctx
        has = (self.rank > 0, self.rank + 1 < self.world)
        for _ in range(int(n)):
            self.lat.step(1)
            for face in (0, 1):
                if has[face]:
                    _check(lib.lb_halo_pack(ctx, face, ctypes.c_void_p(self._out[face].data_ptr())), ctx)
            if self.staged:
                self.lat.sync()
                send = [t.cpu() for t in self._out]
            else:
                torch.cuda.current_stream().synchronize()  # the packs ran on the lattice's stream
                send = self._out
            got = exchange_messages(send[0], send[1], self.rank, self.world, self.group)
            for face in (0, 1):
                if has[face]:
                    m = got[face].to("cuda") if self.staged else got[face]
                    _check(lib.lb_halo_unpack(ctx, face, ctypes.c_void_p(m.data_ptr())), ctx)
                    if self.staged:
                        self.lat.sync()  # the host copy of the message must outlive the unpack
        return self

    def conservation(self) -> np.ndarray:
        c = self.lat.conservation()
        tot = sum_in_rank_order(c[:7], self.group, self._dev)
        return np.concatenate([tot, c[7:]])

    def owned_moments(self):
        """(rho_r, rho_b) of this rank's owned planes."""
        r, b, _, _ = self.lat.moments()
        return r[1:-1], b[1:-1]

    def close(self):
        self.lat.close()
