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
