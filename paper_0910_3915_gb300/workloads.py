"""Seeded synthetic inputs: droplet-on-wall lattices and parameter draws.

This module generates inputs only: geometry masks, initial density fields
and parameter samples. It holds none of the method's arithmetic, so both the
CUDA path and the FP64 oracle take their inputs from here.

Setup (Sec. 2, the droplet experiment): a cap of component r sits on the
bottom wall, surrounded by component b. Node (x, y, z) is inside the droplet
when (x - nx/2)^2 + (y - ny/2)^2 + (z - 0.5)^2 <= R^2, i.e. the sphere's
centre lies on the mid-grid wall plane z = 0.5. Inside rho_r = 0.7,
rho_b = 0.04; outside the two are swapped. Each node and component gets an
independent uniform perturbation in [-1e-3, 1e-3] from numpy's PCG64.
Solid layers are z = 0 and z = nz - 1; x and y are periodic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

RHO_MAJOR = 0.7
RHO_MINOR = 0.04
NOISE = 1e-3


def wall_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    """uint8 mask (nz, ny, nx) with solid layers at z = 0 and z = nz - 1."""
    s = np.zeros((nz, ny, nx), np.uint8)
    s[0] = 1
    s[-1] = 1
    return s


def periodic_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    return np.zeros((nz, ny, nx), np.uint8)


def droplet_fields(nx: int, ny: int, nz: int, radius: float, seed: int = 0,
                   noise: float = NOISE, inside=(RHO_MAJOR, RHO_MINOR),
                   centre=None):
    """Initial (rho_r, rho_b), each float64 (nz, ny, nx), for a cap on z = 0.5."""
    cx, cy, cz = centre if centre is not None else (nx / 2, ny / 2, 0.5)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside_mask = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= radius ** 2
    rr = np.where(inside_mask, inside[0], inside[1]).astype(np.float64)
    rb = np.where(inside_mask, inside[1], inside[0]).astype(np.float64)
    if noise:
        rng = np.random.Generator(np.random.PCG64(seed))
        d = rng.uniform(-noise, noise, size=(2, nz, ny, nx))
        rr += d[0]
        rb += d[1]
    return rr, rb


def lamella_fields(nx: int, ny: int, nz: int, seed: int = 0, noise: float = 0.0,
                   dens=(RHO_MAJOR, RHO_MINOR)):
    """Two lamellae of nz/2 layers each, normal to z, periodic: r-rich in the lower half."""
    rr = np.full((nz, ny, nx), dens[1])
    rb = np.full((nz, ny, nx), dens[0])
    rr[: nz // 2] = dens[0]
    rb[: nz // 2] = dens[1]
    if noise:
        rng = np.random.Generator(np.random.PCG64(seed))
        d = rng.uniform(-noise, noise, size=(2, nz, ny, nx))
        rr += d[0]
        rb += d[1]
    return rr, rb


def slab_fields(nx: int, ny: int, nz: int, phase: str, dens=(RHO_MAJOR, RHO_MINOR)):
    """A box filled with one bulk phase: "liquid" (r-rich) or "gas" (b-rich),
    for the fluid-wall surface tensions of the planar-interface measurement."""
    hi, lo = dens
    a, b = (hi, lo) if phase == "liquid" else (lo, hi)
    return np.full((nz, ny, nx), float(a)), np.full((nz, ny, nx), float(b))


def random_populations(nx: int, ny: int, nz: int, seed: int, lo: float = 0.01, hi: float = 0.06):
    """Arbitrary positive populations (2, 19, nz, ny, nx) for tests that start off-equilibrium."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(2, 19, nz, ny, nx))


def wall_split(w: float):
    """Signed wall parameter w -> (eta_wall_r, eta_wall_b) = (-w, +w).

    w > 0 gives the wall a b-like pseudo-density (repelling the r droplet) and a
    negative r-like one (attracting b); w = 0 is a neutral wall."""
    return -w, w


@dataclass(frozen=True)
class Box:
    """One droplet problem of the batched sweep."""
    edge: int
    radius: float
    g_br: float
    w: float
    seed: int


def sweep_boxes(n: int = 64, seed: int = 3, edges=(48, 64, 80, 96)) -> list[Box]:
    """Batched sweep: cubic boxes with edges drawn from `edges`, radius 0.3 edge,
    g_br ~ U[0.06, 0.12], w ~ U[-0.1, 0.1]; noise seed = box index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    e = rng.choice(np.asarray(edges), size=n)
    g = rng.uniform(0.06, 0.12, size=n)
    w = rng.uniform(-0.1, 0.1, size=n)
    return [Box(int(e[i]), 0.3 * float(e[i]), float(g[i]), float(w[i]), i) for i in range(n)]


def small_wall_params(n: int = 5, seed: int = 1):
    """Wall parameters of the 32^3 case: n values U[-0.05, 0.05] from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [float(v) for v in rng.uniform(-0.05, 0.05, size=n)]


# The workloads, by shape (nx, ny, nz), droplet radius and step counts.
SMALL = dict(name="droplet 32x32x32 R=8", dims=(32, 32, 32), radius=8.0, g_br=0.08, steps=2000)
SINGLE = dict(name="droplet 128x128x128 R=30", dims=(128, 128, 128), radius=30.0, g_br=0.08, steps=20000)
PRECISION = dict(name="droplet 256x256x128 R=60", dims=(256, 256, 128), radius=60.0, g_br=0.08, steps=10000)
PRECISION_DOWN = dict(name="droplet 64x64x32 R=15", dims=(64, 64, 32), radius=15.0, g_br=0.08)
ADJOINT = dict(name="droplet 64x64x64 R=16", dims=(64, 64, 64), radius=16.0, g_br=0.08, steps=2000, ckpt=100)
