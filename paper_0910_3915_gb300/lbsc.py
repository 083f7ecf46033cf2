"""Python binding of the lbsc C ABI (include/lbsc.h): argument marshalling only.

Every computation runs in the CUDA library ``liblbsc.so`` next to this file;
this module converts numpy arrays to pointers, passes a CUDA stream handle
and turns status codes into exceptions. There is no CPU fallback: if the
library is missing or cannot be loaded, ``load()`` raises.

Field arrays are numpy arrays of shape (nz, ny, nx) (x fastest), i.e. the
C ABI's index x + nx*(y + ny*z).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

# LBSC_LIBRARY selects another build of the library (e.g. the bounds-checked liblbsc_debug.so)
_LIB_PATH = os.environ.get("LBSC_LIBRARY") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblbsc.so")

LB_OK = 0
LB_ERR_ARG = -1
LB_ERR_CUDA = -2
LB_ERR_NAN = -3
LB_ERR_BARRIER_TIMEOUT = -4
LB_ERR_STATE = -5
LB_ERR_UNSUPPORTED = -6

LB_F32, LB_F16, LB_BF16 = 0, 1, 2
PRECISIONS = {"f32": LB_F32, "f16": LB_F16, "bf16": LB_BF16}
LB_WEIGHTS_UNIT, LB_WEIGHTS_W36 = 0, 1
LB_STEP_AUTO, LB_STEP_LDG, LB_STEP_TMA = 0, 1, 2
LB_OBS_COM, LB_OBS_COM_SOFT, LB_OBS_WETTED = 0, 1, 2
LB_BUILD_BOUNDS_CHECKED = 1
LB_HALO_BELOW, LB_HALO_ABOVE = 1, 2
LB_DROP_OK, LB_DROP_BAD_PLANE, LB_DROP_NO_PHASE, LB_DROP_NO_APEX, LB_DROP_LOW_APEX, LB_DROP_NO_BASE = range(6)
DROP_STATUS = {LB_DROP_OK: "ok", LB_DROP_BAD_PLANE: "reference plane outside the lattice",
               LB_DROP_NO_PHASE: "no droplet phase (dissolved)", LB_DROP_NO_APEX: "no apex crossing",
               LB_DROP_LOW_APEX: "apex below the reference plane",
               LB_DROP_NO_BASE: "no base at the reference plane (detached)"}
OBSERVABLES = {"com": LB_OBS_COM, "com_soft": LB_OBS_COM_SOFT, "wetted": LB_OBS_WETTED}
STEP_VARIANTS = {"auto": LB_STEP_AUTO, "ldg": LB_STEP_LDG, "tma": LB_STEP_TMA}


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lbsc error {code}: {msg}")
        self.code = code


class lb_params(ctypes.Structure):
    _fields_ = [("tau_r", ctypes.c_double), ("tau_b", ctypes.c_double), ("g_br", ctypes.c_double),
                ("eta_wall_r", ctypes.c_double), ("eta_wall_b", ctypes.c_double),
                ("force_weights", ctypes.c_int), ("force_scale", ctypes.c_double)]


class lb_droplet(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("theta_deg", "theta_fit_deg", "h", "b", "r", "base_ref", "xc", "yc", "zc", "r_fit")] + \
               [("ok", ctypes.c_int), ("n_points", ctypes.c_int), ("phi_max", ctypes.c_double),
                ("phi_min", ctypes.c_double), ("status", ctypes.c_int)]


@dataclass
class Params:
    """Model parameters (lb_params). ``eta_wall_r`` stands in for psi^r at solid
    nodes (felt by b), ``eta_wall_b`` for psi^b (felt by r)."""
    tau_r: float = 1.0
    tau_b: float = 1.0
    g_br: float = 0.0
    eta_wall_r: float = 0.0
    eta_wall_b: float = 0.0
    force_weights: int = LB_WEIGHTS_UNIT
    force_scale: float = 1.0

    def c(self) -> lb_params:
        return lb_params(self.tau_r, self.tau_b, self.g_br, self.eta_wall_r, self.eta_wall_b,
                         int(self.force_weights), self.force_scale)


_lib = None

_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int

# (name, restype, argtypes) of every entry point declared in include/lbsc.h
SIGNATURES = [
    ("lb_init", _I, [ctypes.POINTER(_VP), _I, _I, _I, _I, _DP, _DP, _VP]),
    ("lb_required_bytes", _I, [_I, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    ("lb_init_external", _I, [ctypes.POINTER(_VP), _I, _I, _I, _I, _DP, _DP, _VP, _VP, ctypes.c_size_t]),
    ("lb_set_geometry", _I, [_VP, ctypes.POINTER(ctypes.c_uint8)]),
    ("lb_set_params", _I, [_VP, ctypes.POINTER(lb_params)]),
    ("lb_step", _I, [_VP, _I]),
    ("lb_sync", _I, [_VP]),
    ("lb_selftest_bounded_wait", _I, [_VP, ctypes.c_uint]),
    ("lb_selftest_psi", _I, [ctypes.POINTER(ctypes.c_float), _I, ctypes.POINTER(ctypes.c_float)]),
    ("lb_selftest_round", _I, [_I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint), _I,
                               ctypes.POINTER(ctypes.c_uint)]),
    ("lb_moments", _I, [_VP, _DP, _DP, _DP, _DP]),
    ("lb_conservation", _I, [_VP, _DP]),
    ("lb_reset", _I, [_VP, _DP, _DP]),
    ("lb_init_slab", _I, [ctypes.POINTER(_VP), _I, _I, _I, _I, _DP, _DP, _VP, _I, _I, _DP]),
    ("lb_halo_bytes", _I, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    ("lb_halo_pack", _I, [_VP, _I, _VP]),
    ("lb_halo_unpack", _I, [_VP, _I, _VP]),
    ("lb_halo_exchange", _I, [_VP, _VP]),
    ("lb_slabs_step", _I, [ctypes.POINTER(_VP), _I, _I]),
    ("lb_contact_angle", _I, [_VP, ctypes.c_double, ctypes.POINTER(lb_droplet)]),
    ("lb_contact_angle_at", _I, [_VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(lb_droplet)]),
    ("lb_measure", _I, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.POINTER(lb_droplet)]),
    ("lb_state_bytes", _I, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    ("lb_save", _I, [_VP, _VP, ctypes.c_size_t]),
    ("lb_load", _I, [_VP, _VP, ctypes.c_size_t]),
    ("lb_get_populations", _I, [_VP, _DP]),
    ("lb_set_populations", _I, [_VP, _DP]),
    ("lb_set_schedule", _I, [_VP, _I, _I]),
    ("lb_build_flags", _I, [ctypes.POINTER(_I)]),
    ("lb_set_tiling", _I, [_VP, _I, _I, _I]),
    ("lb_pressure_tensor", _I, [_VP, _DP]),
    ("lb_pressure_profile", _I, [_VP, _DP, _DP]),
    ("lb_pressure_radial", _I, [_VP, _DP, ctypes.c_double, _I, ctypes.c_double, ctypes.c_double, _DP, _DP, _DP]),
    ("lb_young_theta", _I, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _DP]),
    ("lb_huang_theta", _I, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _DP]),
    ("lb_set_step_variant", _I, [_VP, _I, _I]),
    ("lb_step_backward", _I, [_VP, _I, _I, _I, _DP, _DP]),
    ("lb_observable", _I, [_VP, _I, _DP]),
    ("lb_batch_create", _I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(_I), _DP, _DP, ctypes.POINTER(lb_params), _I, _VP]),
    ("lb_batch_set_params", _I, [_VP, _I, ctypes.POINTER(lb_params)]),
    ("lb_batch_set_schedule", _I, [_VP, _I, _I, _I]),
    ("lb_batch_set_step_variant", _I, [_VP, _I]),
    ("lb_batch_step", _I, [_VP, _I]),
    ("lb_batch_box", _I, [_VP, _I, ctypes.POINTER(_VP)]),
    ("lb_batch_conservation", _I, [_VP, _DP]),
    ("lb_batch_contact_angles", _I, [_VP, ctypes.c_double, ctypes.POINTER(lb_droplet)]),
    ("lb_batch_last_error", ctypes.c_char_p, [_VP]),
    ("lb_batch_free", None, [_VP]),
    ("lb_conservation_static", _I, [_VP, _VP, _I, _I, _I, _VP, _VP]),
    ("lb_last_error", ctypes.c_char_p, [_VP]),
    ("lb_free", None, [_VP]),
]


def young_theta(gamma_sg: float, gamma_sl: float, gamma_lg: float) -> float:
    """Young's equation in degrees (clamped at 0 / 180)."""
    t = ctypes.c_double()
    _check(load().lb_young_theta(float(gamma_sg), float(gamma_sl), float(gamma_lg), ctypes.byref(t)))
    return t.value


def huang_theta(eta_wall_r: float, eta_wall_b: float, rho_in: float, rho_out: float) -> float:
    """Huang's closed-form contact angle of the r droplet in degrees."""
    t = ctypes.c_double()
    _check(load().lb_huang_theta(float(eta_wall_r), float(eta_wall_b), float(rho_in), float(rho_out),
                                 ctypes.byref(t)))
    return t.value


def build_flags() -> int:
    f = ctypes.c_int()
    _check(load().lb_build_flags(ctypes.byref(f)))
    return f.value


def load(path: str = _LIB_PATH):
    """Load the CUDA library (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"lbsc CUDA library not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int, ctx=None):
    if rc != LB_OK:
        msg = load().lb_last_error(ctx)
        raise LBError(rc, msg.decode() if msg else "")


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(None)


def conservation_static(populations_ptr: int, solid_ptr: int | None, nx: int, ny: int, nz: int,
                        cons_ptr: int, stream: int | None = None) -> None:
    """lb_conservation_static: FP64 conservation sums of a dense device
    population array into a device array of 8 doubles, with no allocation
    (its scratch is a fixed device array of the library). Asynchronous on
    ``stream`` (default: torch's current stream)."""
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    rc = load().lb_conservation_static(ctypes.c_void_p(populations_ptr),
                                       ctypes.c_void_p(solid_ptr) if solid_ptr else None,
                                       nx, ny, nz, ctypes.c_void_p(cons_ptr), st)
    _check(rc)


class Lattice:
    """One lattice on the current CUDA device (a ``lb_ctx``).

    rho_r, rho_b: initial densities (nz, ny, nx). precision: "f32", "f16" or "bf16".
    stream: a CUDA stream handle (int) or None for torch's current stream.
    torch_memory: place the lattice in a torch-allocated device buffer
    (lb_init_external); otherwise the library allocates it (lb_init).
    """

    def __init__(self, rho_r, rho_b, precision: str = "f32", stream=None, torch_memory: bool = False,
                 slab=None):
        lib = load()
        rr, rb = _f64(rho_r), _f64(rho_b)
        if rr.shape != rb.shape or rr.ndim != 3:
            raise ValueError("rho_r and rho_b must have the same 3-D shape (nz, ny, nx)")
        self.nz, self.ny, self.nx = rr.shape
        self.precision = precision
        st = _current_stream() if stream is None else ctypes.c_void_p(stream)
        ctx = ctypes.c_void_p()
        self._buf = None
        if slab is not None:
            # a z slab of a decomposed lattice: slab = (halo flags, zbase, references or None)
            halo, zbase, ref = slab
            ref_a = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64)
            rc = lib.lb_init_slab(ctypes.byref(ctx), self.nx, self.ny, self.nz, PRECISIONS[precision], _dp(rr),
                                  _dp(rb), st, int(halo), int(zbase), None if ref_a is None else _dp(ref_a))
        elif torch_memory:
            import torch
            nbytes = ctypes.c_size_t()
            _check(lib.lb_required_bytes(self.nx, self.ny, self.nz, PRECISIONS[precision], ctypes.byref(nbytes)))
            self._buf = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
            ptr = (self._buf.data_ptr() + 255) // 256 * 256
            rc = lib.lb_init_external(ctypes.byref(ctx), self.nx, self.ny, self.nz, PRECISIONS[precision],
                                      _dp(rr), _dp(rb), st, ctypes.c_void_p(ptr), nbytes.value)
        else:
            rc = lib.lb_init(ctypes.byref(ctx), self.nx, self.ny, self.nz, PRECISIONS[precision],
                             _dp(rr), _dp(rb), st)
        _check(rc)
        self._ctx = ctx
        self._params = Params()

    # ------------------------------------------------------------ configuration
    @property
    def shape(self):
        return self.nz, self.ny, self.nx

    @property
    def params(self) -> Params:
        return self._params

    def set_params(self, params: Params | None = None, **kw) -> "Lattice":
        p = params if params is not None else Params(**{**self._params.__dict__, **kw})
        cp = p.c()
        _check(load().lb_set_params(self._ctx, ctypes.byref(cp)), self._ctx)
        self._params = p
        return self

    def reset(self, rho_r, rho_b) -> "Lattice":
        """Start again from new initial densities (lb_reset): no allocation; the
        step count returns to 0, geometry, parameters and schedule stay."""
        rr, rb = _f64(rho_r), _f64(rho_b)
        if rr.shape != self.shape or rb.shape != self.shape:
            raise ValueError("rho_r and rho_b must have the lattice's shape (nz, ny, nx)")
        _check(load().lb_reset(self._ctx, _dp(rr), _dp(rb)), self._ctx)
        return self

    def set_geometry(self, solid) -> "Lattice":
        s = np.ascontiguousarray(solid, dtype=np.uint8)
        if s.shape != self.shape:
            raise ValueError("solid mask must have shape (nz, ny, nx)")
        _check(load().lb_set_geometry(self._ctx, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), self._ctx)
        return self

    def set_schedule(self, tile_y: int = 8, z_segments: int = 0) -> "Lattice":
        _check(load().lb_set_schedule(self._ctx, tile_y, z_segments), self._ctx)
        return self

    def set_tiling(self, tile_y: int = 8, y_tiles: int = 0, z_segments: int = 0) -> "Lattice":
        """Tile height, number of y-tiles (even row split; 0 = ceil(ny / tile_y)) and z segments."""
        _check(load().lb_set_tiling(self._ctx, tile_y, y_tiles, z_segments), self._ctx)
        return self

    def set_step_variant(self, variant: str = "auto", stages: int = 0) -> "Lattice":
        _check(load().lb_set_step_variant(self._ctx, STEP_VARIANTS[variant], int(stages)), self._ctx)
        return self

    # ------------------------------------------------------------ stepping
    def step(self, n: int = 1) -> "Lattice":
        _check(load().lb_step(self._ctx, int(n)), self._ctx)
        return self

    def sync(self) -> "Lattice":
        _check(load().lb_sync(self._ctx), self._ctx)
        return self

    # ------------------------------------------------------------ readback
    def moments(self, velocity: bool = False):
        """(rho_r, rho_b, u or None, cons[8])"""
        rr = np.empty(self.shape)
        rb = np.empty(self.shape)
        u = np.empty((3,) + self.shape) if velocity else None
        cons = np.empty(8)
        _check(load().lb_moments(self._ctx, _dp(rr), _dp(rb), _dp(u) if u is not None else None, _dp(cons)),
               self._ctx)
        return rr, rb, u, cons

    def conservation(self) -> np.ndarray:
        cons = np.empty(8)
        _check(load().lb_conservation(self._ctx, _dp(cons)), self._ctx)
        return cons

    def contact_angle(self, offset: float = 5.0, level: float = 0.0) -> dict:
        d = lb_droplet()
        _check(load().lb_contact_angle_at(self._ctx, float(offset), float(level), ctypes.byref(d)), self._ctx)
        return {f: getattr(d, f) for f, _ in lb_droplet._fields_}

    def measure(self, offset: float = 5.0):
        """(conservation sums, contact angle at level 0) in one pass over the
        populations: the results of conservation() and contact_angle(offset)."""
        cons = np.empty(8)
        d = lb_droplet()
        _check(load().lb_measure(self._ctx, _dp(cons), float(offset), ctypes.byref(d)), self._ctx)
        return cons, {f: getattr(d, f) for f, _ in lb_droplet._fields_}

    def pressure_tensor(self) -> np.ndarray:
        """P (6, nz, ny, nx): xx, yy, zz, xy, xz, yz of the pressure tensor (Sec. 4.1)."""
        P = np.empty((6,) + self.shape)
        _check(load().lb_pressure_tensor(self._ctx, _dp(P)), self._ctx)
        return P

    def pressure_profile(self):
        """(prof (nz, 8), gamma_sum): plane means of P and phi, fluid counts, and
        sum_z (P_N - P_T) (Eq. gammaMechDef, normal z)."""
        prof = np.empty((self.shape[0], 8))
        g = ctypes.c_double()
        _check(load().lb_pressure_profile(self._ctx, _dp(prof), ctypes.byref(g)), self._ctx)
        return prof, g.value

    def pressure_radial(self, centre, dr: float = 1.0, nbins: int = 64, zmin: float = 0.0, r_max: float = 1e30):
        """(bins (nbins, 4), gamma, R_s): radial means of P_N, P_T, phi and counts
        about `centre` (x, y, z) and the surface tension of Eq. mechRadGamma."""
        c = np.ascontiguousarray(centre, dtype=np.float64)
        bins = np.empty((int(nbins), 4))
        g, rs = ctypes.c_double(), ctypes.c_double()
        _check(load().lb_pressure_radial(self._ctx, _dp(c), float(dr), int(nbins), float(zmin), float(r_max),
                                         _dp(bins), ctypes.byref(g), ctypes.byref(rs)), self._ctx)
        return bins, g.value, rs.value

    def populations(self) -> np.ndarray:
        n = np.empty((2, 19) + self.shape)
        _check(load().lb_get_populations(self._ctx, _dp(n)), self._ctx)
        return n

    def set_populations(self, n) -> "Lattice":
        a = _f64(n)
        if a.shape != (2, 19) + self.shape:
            raise ValueError("populations must have shape (2, 19, nz, ny, nx)")
        _check(load().lb_set_populations(self._ctx, _dp(a)), self._ctx)
        return self

    # ------------------------------------------------------------ adjoint
    def step_backward(self, nsteps: int, ckpt_every: int = 100, observable: str = "com_soft"):
        """Advance nsteps; return (J, dJ/d(eta_wall_r, eta_wall_b)) by the discrete adjoint."""
        g = np.zeros(2)
        J = ctypes.c_double()
        _check(load().lb_step_backward(self._ctx, int(nsteps), int(ckpt_every), OBSERVABLES[observable],
                                       _dp(g), ctypes.byref(J)), self._ctx)
        return J.value, g

    def observable(self, observable: str = "com_soft") -> float:
        J = ctypes.c_double()
        _check(load().lb_observable(self._ctx, OBSERVABLES[observable], ctypes.byref(J)), self._ctx)
        return J.value

    # ------------------------------------------------------------ checkpoints
    def save(self) -> bytes:
        nb = ctypes.c_size_t()
        _check(load().lb_state_bytes(self._ctx, ctypes.byref(nb)), self._ctx)
        buf = ctypes.create_string_buffer(nb.value)
        _check(load().lb_save(self._ctx, buf, nb.value), self._ctx)
        return buf.raw

    def load(self, state: bytes) -> "Lattice":
        _check(load().lb_load(self._ctx, state, len(state)), self._ctx)
        return self

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            load().lb_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _bcheck(rc: int, b=None):
    if rc != LB_OK:
        msg = load().lb_batch_last_error(b)
        raise LBError(rc, msg.decode() if msg else "")


class _BoxView(Lattice):
    """A borrowed box context of a Batch: readers only (moments, contact angle, save)."""

    def __init__(self, ctx, shape, precision, batch):
        self.nz, self.ny, self.nx = shape
        self.precision = precision
        self._ctx = ctx
        self._buf = None
        self._params = Params()
        self._batch = batch

    def step(self, n: int = 1):
        raise LBError(LB_ERR_STATE, "a batch box is stepped through its Batch")

    def close(self):
        self._ctx = ctypes.c_void_p()  # owned by the batch


class Batch:
    """Many independent droplet lattices advanced together (lb_batch_*).

    fields: list of (rho_r, rho_b) pairs, each (nz, ny, nx); params: list of Params."""

    def __init__(self, fields, params, precision: str = "f32", stream=None):
        lib = load()
        self.n = len(fields)
        if self.n != len(params) or self.n == 0:
            raise ValueError("one Params per box")
        dims = []
        rr_all, rb_all = [], []
        self.shapes = []
        for rr, rb in fields:
            rr, rb = _f64(rr), _f64(rb)
            nz, ny, nx = rr.shape
            dims += [nx, ny, nz]
            self.shapes.append((nz, ny, nx))
            rr_all.append(rr.ravel())
            rb_all.append(rb.ravel())
        d = (ctypes.c_int * len(dims))(*dims)
        rr = np.ascontiguousarray(np.concatenate(rr_all))
        rb = np.ascontiguousarray(np.concatenate(rb_all))
        pa = (lb_params * self.n)(*[p.c() for p in params])
        st = _current_stream() if stream is None else ctypes.c_void_p(stream)
        b = ctypes.c_void_p()
        _bcheck(lib.lb_batch_create(ctypes.byref(b), self.n, d, _dp(rr), _dp(rb), pa, PRECISIONS[precision], st))
        self._b = b
        self.precision = precision
        self.params = list(params)

    def set_schedule(self, tile_y: int = 8, planes_per_item: int = 32, ctas_per_sm: int = 0) -> "Batch":
        _bcheck(load().lb_batch_set_schedule(self._b, tile_y, planes_per_item, ctas_per_sm), self._b)
        return self

    def set_step_variant(self, variant: str = "auto") -> "Batch":
        """"auto"/"tma": the TMA-staged persistent kernel (4- or 8-row tiles),
        "ldg": the load-from-global one; both give identical results."""
        _bcheck(load().lb_batch_set_step_variant(self._b, STEP_VARIANTS[variant]), self._b)
        return self

    def set_params(self, i: int, params: Params) -> "Batch":
        cp = params.c()
        _bcheck(load().lb_batch_set_params(self._b, i, ctypes.byref(cp)), self._b)
        self.params[i] = params
        return self

    def step(self, n: int = 1) -> "Batch":
        _bcheck(load().lb_batch_step(self._b, int(n)), self._b)
        return self

    def box(self, i: int) -> Lattice:
        c = ctypes.c_void_p()
        _bcheck(load().lb_batch_box(self._b, i, ctypes.byref(c)), self._b)
        return _BoxView(c, self.shapes[i], self.precision, self)

    def conservation(self) -> np.ndarray:
        out = np.empty((self.n, 8))
        _bcheck(load().lb_batch_conservation(self._b, _dp(out)), self._b)
        return out

    def contact_angles(self, offset: float = 5.0) -> list:
        recs = (lb_droplet * self.n)()
        _bcheck(load().lb_batch_contact_angles(self._b, float(offset), recs), self._b)
        return [{f: getattr(r, f) for f, _ in lb_droplet._fields_} for r in recs]

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            load().lb_batch_free(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wall_gradient(lattice: Lattice, initial_state: bytes, base: Params, nsteps: int, ckpt_every: int = 100,
                  observable: str = "com_soft"):
    """Torch autograd Function over the signed wall parameter w, (eta_r, eta_b) = (-w, +w).

    Returns a function f(w_tensor) -> J_tensor whose backward uses the adjoint
    gradient dJ/dw = dJ/deta_b - dJ/deta_r. Each call restarts from
    ``initial_state`` (a checkpoint from Lattice.save())."""
    import torch

    class LBStepFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, w):
            wv = float(w.detach().cpu())
            lattice.load(initial_state)
            lattice.set_params(Params(**{**base.__dict__, "eta_wall_r": -wv, "eta_wall_b": wv}))
            J, g = lattice.step_backward(nsteps, ckpt_every, observable)
            ctx.dJdw = g[1] - g[0]
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            return grad * ctx.dJdw

    return LBStepFn.apply
