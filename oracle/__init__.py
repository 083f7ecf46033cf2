"""FP64 CPU oracle of the two-component Shan-Chen D3Q19 step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the CPU
baseline leg of ``bench.py`` may import this package; the product path never
does. It shares no code with the CUDA library.

The arithmetic lives in ``lb_oracle.c`` (plain C, double precision, one pass
per stage of the method in the paper's order). This module only compiles it
with gcc and marshals numpy arrays.

Array conventions: fields are numpy arrays of shape (nz, ny, nx) (x fastest);
populations have shape (2, 19, nz, ny, nx).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIB = os.path.join(_HERE, "liblb_oracle.so")

Q = 19


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lb_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double * 2), ("g", ctypes.c_double),
                ("eta_wall", ctypes.c_double * 2), ("force_scale", ctypes.c_double),
                ("weights", ctypes.c_int)]


class _Droplet(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("theta_deg", "theta_fit_deg", "h", "b", "r", "base_ref", "xc", "yc", "zc", "r_fit")] + \
               [("ok", ctypes.c_int), ("n_points", ctypes.c_int)]


@dataclass
class Params:
    """Method parameters. ``eta_wall_r`` is the wall's pseudo-density standing in
    for psi^r (felt by component b); ``eta_wall_b`` stands in for psi^b (felt by r)."""
    tau_r: float = 1.0
    tau_b: float = 1.0
    g_br: float = 0.08
    eta_wall_r: float = 0.0
    eta_wall_b: float = 0.0
    force_weights: int = 0
    force_scale: float = 1.0

    def c(self) -> _Params:
        p = _Params()
        p.tau[0], p.tau[1] = self.tau_r, self.tau_b
        p.g = self.g_br
        p.eta_wall[0], p.eta_wall[1] = self.eta_wall_r, self.eta_wall_b
        p.force_scale = self.force_scale
        p.weights = self.force_weights
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        u8 = ctypes.POINTER(ctypes.c_uint8)
        i = ctypes.c_int
        _lib.lbo_lattice.argtypes = [ctypes.POINTER(ctypes.c_int)] * 3 + [d, ctypes.POINTER(ctypes.c_int)]
        _lib.lbo_equilibrium.argtypes = [ctypes.c_double, d, d]
        _lib.lbo_init_equilibrium.argtypes = [i, i, i, u8, d, d, d]
        _lib.lbo_density.argtypes = [i, i, i, u8, d, d, d]
        _lib.lbo_force.argtypes = [ctypes.POINTER(_Params), i, i, i, u8, d, d]
        _lib.lbo_run.argtypes = [ctypes.POINTER(_Params), i, i, i, u8, d, i]
        _lib.lbo_run.restype = ctypes.c_int
        _lib.lbo_moments.argtypes = [ctypes.POINTER(_Params), i, i, i, u8, d, d, d, d, d]
        _lib.lbo_contact_angle.argtypes = [i, i, i, u8, d, d, ctypes.c_double, ctypes.POINTER(_Droplet)]
        _lib.lbo_contact_angle.restype = ctypes.c_int
        _lib.lbo_contact_angle_level.argtypes = [i, i, i, u8, d, d, ctypes.c_double, ctypes.c_double,
                                                 ctypes.POINTER(_Droplet)]
        _lib.lbo_contact_angle_level.restype = ctypes.c_int
        _lib.lbo_pressure_tensor.argtypes = [ctypes.POINTER(_Params), i, i, i, u8, d, d]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def lattice():
    """(c [19,3] int, zeta [19], opp [19]) of the oracle's D3Q19 table."""
    cx, cy, cz, opp = (np.zeros(Q, np.int32) for _ in range(4))
    zeta = np.zeros(Q)
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    lib().lbo_lattice(ip(cx), ip(cy), ip(cz), _dp(zeta), ip(opp))
    return np.stack([cx, cy, cz], 1), zeta, opp


def equilibrium(rho: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    lib().lbo_equilibrium(float(rho), _dp(u), _dp(out))
    return out


class State:
    """A lattice held by the oracle: populations n (2, 19, nz, ny, nx), solid mask, params."""

    def __init__(self, rho_r: np.ndarray, rho_b: np.ndarray, solid: np.ndarray, params: Params):
        self.nz, self.ny, self.nx = rho_r.shape
        self.solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.params = params
        self.n = np.zeros((2, Q) + rho_r.shape)
        rr = np.ascontiguousarray(rho_r, dtype=np.float64)
        rb = np.ascontiguousarray(rho_b, dtype=np.float64)
        lib().lbo_init_equilibrium(self.nx, self.ny, self.nz, _u8(self.solid), _dp(rr), _dp(rb), _dp(self.n))

    @property
    def dims(self):
        return self.nx, self.ny, self.nz

    def step(self, steps: int = 1) -> "State":
        p = self.params.c()
        rc = lib().lbo_run(ctypes.byref(p), *self.dims, _u8(self.solid), _dp(self.n), int(steps))
        if rc != 0:
            raise ValueError("oracle: bad argument")
        return self

    def density(self):
        rho = np.zeros((2,) + self.n.shape[2:])
        j = np.zeros((2, 3) + self.n.shape[2:])
        lib().lbo_density(*self.dims, _u8(self.solid), _dp(self.n), _dp(rho), _dp(j))
        return rho, j

    def force(self) -> np.ndarray:
        F = np.zeros((2, 3) + self.n.shape[2:])
        p = self.params.c()
        lib().lbo_force(ctypes.byref(p), *self.dims, _u8(self.solid), _dp(self.n), _dp(F))
        return F

    def moments(self):
        """(rho_r, rho_b, u[3,...], cons[8])"""
        shp = self.n.shape[2:]
        rr, rb, u, cons = np.zeros(shp), np.zeros(shp), np.zeros((3,) + shp), np.zeros(8)
        p = self.params.c()
        lib().lbo_moments(ctypes.byref(p), *self.dims, _u8(self.solid), _dp(self.n),
                          _dp(rr), _dp(rb), _dp(u), _dp(cons))
        return rr, rb, u, cons

    def pressure_tensor(self) -> np.ndarray:
        P = np.zeros((6,) + self.n.shape[2:])
        p = self.params.c()
        lib().lbo_pressure_tensor(ctypes.byref(p), *self.dims, _u8(self.solid), _dp(self.n), _dp(P))
        return P

    def contact_angle(self, offset: float = 5.0) -> dict:
        rr, rb, _, _ = self.moments()
        return contact_angle(rr, rb, self.solid, offset)


def contact_angle(rho_r: np.ndarray, rho_b: np.ndarray, solid: np.ndarray, offset: float = 5.0,
                  level: float = 0.0) -> dict:
    nz, ny, nx = rho_r.shape
    out = _Droplet()
    rr = np.ascontiguousarray(rho_r, dtype=np.float64)
    rb = np.ascontiguousarray(rho_b, dtype=np.float64)
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    lib().lbo_contact_angle_level(nx, ny, nz, _u8(s), _dp(rr), _dp(rb), float(offset), float(level),
                                  ctypes.byref(out))
    return {f: getattr(out, f) for f, _ in _Droplet._fields_}


# ---------------------------------------------------------------- surface tension (Sec. 4.1-4.2)
def pressure_profile(P: np.ndarray, solid: np.ndarray, rho_r: np.ndarray, rho_b: np.ndarray):
    """Plane averages of the pressure tensor along z and the planar surface
    tension integral of Eq. gammaMechDef (normal z, dz = 1).

    P: (6, nz, ny, nx) with components xx, yy, zz, xy, xz, yz (``State.pressure_tensor``).
    Returns (prof, gamma_sum): prof[z] = (mean P_xx, P_yy, P_zz, P_xy, P_xz, P_yz,
    mean phi, fluid count) over the plane's fluid nodes (zeros for a solid plane),
    and gamma_sum = sum over planes with fluid of P_N - P_T, P_N = P_zz,
    P_T = (P_xx + P_yy)/2. A periodic box with two interfaces holds 2 gamma."""
    nz = P.shape[1]
    fl = solid == 0
    phi = rho_r - rho_b
    prof = np.zeros((nz, 8))
    for z in range(nz):
        m = fl[z]
        n = int(m.sum())
        if n == 0:
            continue
        for c in range(6):
            prof[z, c] = P[c, z][m].sum() / n
        prof[z, 6] = phi[z][m].sum() / n
        prof[z, 7] = n
    has = prof[:, 7] > 0
    gamma_sum = float(np.sum(prof[has, 2] - 0.5 * (prof[has, 0] + prof[has, 1])))
    return prof, gamma_sum


def pressure_radial(P: np.ndarray, solid: np.ndarray, rho_r: np.ndarray, rho_b: np.ndarray, centre,
                    dr: float, nbins: int, zmin: float, r_max: float, periodic_z: bool = False):
    """Radial profile of the normal and transversal pressure about `centre`
    (x, y, z) and the curved-interface surface tension of Eq. mechRadGamma.

    For a fluid node at distance r (minimum image along x, y, and z when
    periodic_z) with unit vector n = (x - centre)/r: P_N = n.P.n and
    P_T = (tr P - P_N)/2. Nodes with z < zmin or r = 0 are skipped; node r
    falls in bin floor(r/dr). Returns (bins, gamma, R_s): bins[b] = (mean P_N,
    mean P_T, mean phi, count); R_s the radius where the bin-mean phi first
    changes sign going outward (linear interpolation between bin centres
    r_b = (b + 1/2) dr); gamma = sum over bins with r_b <= r_max of
    (r_b/R_s)^2 (P_N - P_T) dr (0 and R_s = nan when phi never changes sign)."""
    nz, ny, nx = rho_r.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def sep(a, c, n, periodic):
        d = a - c
        if periodic:
            d = d - n * np.round(d / n)
        return d

    dx = sep(x, centre[0], nx, True)
    dy = sep(y, centre[1], ny, True)
    dz = sep(z, centre[2], nz, periodic_z)
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    use = (solid == 0) & (z >= zmin) & (r > 0)
    b = np.floor(r / dr).astype(np.int64)
    use &= b < nbins
    rs = np.where(r > 0, r, 1.0)
    n = [dx / rs, dy / rs, dz / rs]
    T = [[P[0], P[3], P[4]], [P[3], P[1], P[5]], [P[4], P[5], P[2]]]
    pn = sum(n[i] * T[i][j] * n[j] for i in range(3) for j in range(3))
    pt = 0.5 * (P[0] + P[1] + P[2] - pn)
    phi = rho_r - rho_b
    bins = np.zeros((nbins, 4))
    for k in range(nbins):
        m = use & (b == k)
        cnt = int(m.sum())
        if cnt:
            bins[k] = (pn[m].sum() / cnt, pt[m].sum() / cnt, phi[m].sum() / cnt, cnt)
    R_s = float("nan")
    prev = None
    for k in range(nbins):
        if bins[k, 3] == 0:
            continue
        if prev is not None and (bins[prev, 2] > 0) != (bins[k, 2] > 0):
            r0, r1 = (prev + 0.5) * dr, (k + 0.5) * dr
            p0, p1 = bins[prev, 2], bins[k, 2]
            R_s = r0 + (r1 - r0) * p0 / (p0 - p1)
            break
        prev = k
    gamma = 0.0
    if R_s == R_s:
        for k in range(nbins):
            rb = (k + 0.5) * dr
            if bins[k, 3] and rb <= r_max:
                gamma += (rb / R_s) ** 2 * (bins[k, 0] - bins[k, 1]) * dr
    return bins, gamma, R_s


def young_theta(gamma_sg: float, gamma_sl: float, gamma_lg: float) -> float:
    """Young's equation (Eq. young): cos theta = (gamma_SG - gamma_SL)/gamma_LG,
    in degrees; 0 or 180 when the ratio leaves [-1, 1] (complete wetting or drying)."""
    c = (gamma_sg - gamma_sl) / gamma_lg
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))
