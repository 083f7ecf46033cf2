"""Independent brute-force stepper for tiny lattices (a pin for the C oracle).

Written separately from the oracle and in a different formulation: its own
velocity table built by enumeration, per-node Python loops, and a PULL
stream (each node gathers n_k from x - c_k, or its own reversed post-collision
value when x - c_k is solid), where the oracle pushes. It follows the same
method (Sec. 2: moments, psi = 1 - exp(-rho), Eq. SCforce with the wall as a
species, the force-shifted cubic equilibrium of Eq. Equil, BGK, Eq. LBeqs with
mid-grid bounce-back). Only for lattices of a few hundred nodes.
"""
from __future__ import annotations

import itertools

import numpy as np

# every integer velocity with |c|^2 <= 2 in 3D: 1 + 6 + 12 = 19
VEL = np.array([c for c in itertools.product((-1, 0, 1), repeat=3) if sum(v * v for v in c) <= 2])
W = np.array([{0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[int(c @ c)] for c in VEL])
OPP = np.array([int(np.flatnonzero((VEL == -c).all(1))[0]) for c in VEL])


def step(n, solid, tau, g, eta_wall, weights=0, kappa=1.0):
    """One step. n: dict a -> array (nz, ny, nx, 19) in this module's velocity order."""
    nz, ny, nx = solid.shape
    cs2 = 1 / 3
    G = 36 * W if weights == 1 else np.ones(19)
    rho = {a: n[a].sum(-1) for a in (0, 1)}
    mom = {a: n[a] @ VEL for a in (0, 1)}
    psi = {}
    for a in (0, 1):
        psi[a] = np.where(solid == 1, eta_wall[a], 1 - np.exp(-rho[a]))
    post = {a: np.zeros_like(n[a]) for a in (0, 1)}
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if solid[z, y, x]:
            continue
        F = {}
        for a in (0, 1):
            acc = np.zeros(3)
            for k, c in enumerate(VEL):
                if not c.any():
                    continue
                zz, yy, xx = (z + c[2]) % nz, (y + c[1]) % ny, (x + c[0]) % nx
                acc += G[k] * psi[1 - a][zz, yy, xx] * c
            F[a] = -kappa * g * psi[a][z, y, x] * acc
        num = sum(mom[a][z, y, x] / tau[a] for a in (0, 1))
        den = sum(rho[a][z, y, x] / tau[a] for a in (0, 1))
        ubar = num / den if den > 0 else np.zeros(3)
        for a in (0, 1):
            r = rho[a][z, y, x]
            u = ubar + tau[a] * F[a] / r if r > 1e-12 else ubar
            cu = VEL @ u
            uu = u @ u
            neq = W * r * (1 + cu / cs2 + cu ** 2 / (2 * cs2 ** 2) - uu / (2 * cs2)
                           + cu ** 3 / (6 * cs2 ** 3) - uu * cu / (2 * cs2 ** 2))
            post[a][z, y, x] = n[a][z, y, x] - (n[a][z, y, x] - neq) / tau[a]
    out = {a: np.zeros_like(n[a]) for a in (0, 1)}
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if solid[z, y, x]:
            continue
        for k, c in enumerate(VEL):
            zs, ys, xs = (z - c[2]) % nz, (y - c[1]) % ny, (x - c[0]) % nx
            for a in (0, 1):
                if solid[zs, ys, xs]:
                    out[a][z, y, x, k] = post[a][z, y, x, OPP[k]]
                else:
                    out[a][z, y, x, k] = post[a][zs, ys, xs, k]
    return out


def from_oracle_layout(n_oracle, c_oracle):
    """(2, 19, nz, ny, nx) in the oracle's order -> dict a -> (nz, ny, nx, 19) in VEL order."""
    perm = [int(np.flatnonzero((c_oracle == c).all(1))[0]) for c in VEL]
    return {a: np.moveaxis(n_oracle[a][perm], 0, -1).copy() for a in (0, 1)}
