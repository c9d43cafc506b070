"""GB300 (sm_103a) split-operator Dirac stepper: Python binding of libdirac.

Thin ctypes binding of the C ABI in include/dirac.h, with the same function names.  It only
marshals arguments: numpy arrays are passed as host pointers, torch CUDA tensors as device
pointers, and every step of the scheme runs in libdirac's CUDA kernels.  There is no CPU
fallback: when libdirac.so is missing or fails to load, every call raises.

Build the library with ``python -m paper_1107_4650_gb300.build`` (or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdirac.so")

DIRAC_OK, DIRAC_ERR_ARG, DIRAC_ERR_OOM, DIRAC_ERR_CUDA, DIRAC_ERR_NONFINITE, DIRAC_ERR_TIMEOUT, DIRAC_ERR_STATE = range(7)
DIRAC_FP64, DIRAC_FP32, DIRAC_FX64 = 0, 1, 2
DIRAC_BC_ZERO, DIRAC_BC_PERIODIC = 0, 1
DIRAC_V_NONE, DIRAC_V_X_ONLY, DIRAC_V_FULL = 0, 1, 2
DIRAC_LIE, DIRAC_STRANG = 0, 1
DIRAC_PLAN_STEP_2D, DIRAC_PLAN_STRANG_2D, DIRAC_PLAN_FIELD_2D, DIRAC_PLAN_SHIFT_2D = 0, 1, 2, 3
DIRAC_PLAN_3D_TWO_PASS, DIRAC_PLAN_3D_FUSED, DIRAC_PLAN_3D_STRANG, DIRAC_PLAN_STRANG_FIELD_2D = 4, 5, 6, 7
DIRAC_PLAN_3D_STRANG_FUSED, DIRAC_PLAN_SHIFT_SWEEPS, DIRAC_PLAN_FIELD_SWEEPS = 8, 9, 10
DIRAC_PLAN_3D_STRANG_ZPASS = 11

STATUS_NAMES = {0: "DIRAC_OK", 1: "DIRAC_ERR_ARG", 2: "DIRAC_ERR_OOM", 3: "DIRAC_ERR_CUDA",
                4: "DIRAC_ERR_NONFINITE", 5: "DIRAC_ERR_TIMEOUT", 6: "DIRAC_ERR_STATE"}


class DiracError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class dirac_config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("dx", ctypes.c_double),
                ("c", ctypes.c_double), ("m", ctypes.c_double), ("x_min", ctypes.c_double * 3),
                ("precision", ctypes.c_int), ("boundary", ctypes.c_int), ("flux_face", ctypes.c_int64),
                ("stream", ctypes.c_void_p), ("device", ctypes.c_int), ("steps_per_launch", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("points_per_lane", ctypes.c_int), ("splitting", ctypes.c_int),
                ("char_shift", ctypes.c_int), ("ext_state", ctypes.c_void_p * 2)]


class dirac_obs(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_double), ("norm_right", ctypes.c_double), ("flux_cum", ctypes.c_double),
                ("centroid", ctypes.c_double * 3), ("step", ctypes.c_int64)]


class dirac_info(ctypes.Structure):
    _fields_ = [("steps_per_launch", ctypes.c_int), ("points_per_lane", ctypes.c_int),
                ("launch_warps", ctypes.c_int64), ("strip_width", ctypes.c_int64),
                ("segment_rows", ctypes.c_int64), ("graphs", ctypes.c_int),
                ("kernel_launches", ctypes.c_int64), ("device_bytes", ctypes.c_size_t), ("plan", ctypes.c_int),
                ("fx_shift", ctypes.c_int), ("state_index", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libdirac.so; raises RuntimeError if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdirac.so not found at %s: build it first (paper_1107_4650_gb300.build)" % path)
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "dirac_default_config": (None, [ctypes.POINTER(dirac_config)]),
        "dirac_create_grid": (I, [ctypes.POINTER(dirac_config), ctypes.POINTER(P)]),
        "dirac_destroy": (I, [P]),
        "dirac_set_potential": (I, [P, P, I, I64]),
        "dirac_set_state": (I, [P, P, I]),
        "dirac_get_state": (I, [P, P, I]),
        "dirac_state_ptr": (I, [P, ctypes.POINTER(P)]),
        "dirac_set_state_fx": (I, [P, P, I, I]),
        "dirac_get_state_fx": (I, [P, P, ctypes.POINTER(I), I]),
        "dirac_step": (I, [P, I64]),
        "dirac_observables": (I, [P, ctypes.POINTER(dirac_obs), P, I]),
        "dirac_set_counters": (I, [P, I64, D]),
        "dirac_set_absorber": (I, [P, P, I64]),
        "dirac_set_vector_potential": (I, [P, P, I64]),
        "dirac_set_field": (I, [P, P, P, P, I64]),
        "dirac_get_info": (I, [P, ctypes.POINTER(dirac_info)]),
        "dirac_autotune": (I, [P]),
        "dirac_last_error": (ctypes.c_char_p, [P]),
        "dirac_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int, handle=None):
    if st != DIRAC_OK:
        msg = load_library().dirac_last_error(handle)
        raise DiracError(st, msg.decode() if msg else "")


def _ptr(buf, want_elem_bytes: int):
    """(pointer, on_device) for a numpy array or a torch tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return buf.ctypes.data, 0
    if hasattr(buf, "data_ptr") and hasattr(buf, "is_cuda"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr(), 1 if buf.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def dirac_version() -> str:
    return load_library().dirac_version().decode()


def dirac_default_config() -> dirac_config:
    cfg = dirac_config()
    load_library().dirac_default_config(ctypes.byref(cfg))
    return cfg


def dirac_create_grid(cfg: dirac_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().dirac_create_grid(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def dirac_destroy(h) -> None:
    _check(load_library().dirac_destroy(h))


def dirac_set_potential(h, V, layout: int) -> None:
    if layout == DIRAC_V_NONE:
        _check(load_library().dirac_set_potential(h, None, layout, 0), h)
        return
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
    _check(load_library().dirac_set_potential(h, V.ctypes.data, layout, V.size), h)


def dirac_set_state(h, psi) -> None:
    p, dev = _ptr(psi, 8)
    _check(load_library().dirac_set_state(h, p, dev), h)


def dirac_get_state(h, out) -> None:
    p, dev = _ptr(out, 8)
    _check(load_library().dirac_get_state(h, p, dev), h)


def dirac_set_state_fx(h, q, shift: int) -> None:
    """DIRAC_FX64: set the int64 fixed-point state q (psi = q 2^-shift) without conversion."""
    p, dev = _ptr(q, 8)
    _check(load_library().dirac_set_state_fx(h, p, int(shift), dev), h)


def dirac_get_state_fx(h, out) -> int:
    """DIRAC_FX64: copy the int64 fixed-point state into out; returns its shift."""
    p, dev = _ptr(out, 8)
    sh = ctypes.c_int()
    _check(load_library().dirac_get_state_fx(h, p, ctypes.byref(sh), dev), h)
    return sh.value


def dirac_state_ptr(h) -> int:
    p = ctypes.c_void_p()
    _check(load_library().dirac_state_ptr(h, ctypes.byref(p)), h)
    return p.value


def dirac_step(h, nsteps: int) -> None:
    _check(load_library().dirac_step(h, int(nsteps)), h)


def dirac_observables(h, density=None) -> dict:
    obs = dirac_obs()
    if density is None:
        st = load_library().dirac_observables(h, ctypes.byref(obs), None, 0)
    else:
        p, dev = _ptr(density, 8)
        st = load_library().dirac_observables(h, ctypes.byref(obs), p, dev)
    _check(st, h)
    return {"norm": obs.norm, "norm_right": obs.norm_right, "flux_cum": obs.flux_cum,
            "centroid": tuple(obs.centroid), "step": obs.step}


def dirac_set_absorber(h, a) -> None:
    """Per-x-column damping factors in (0, 1] (None: remove)."""
    if a is None:
        _check(load_library().dirac_set_absorber(h, None, 0), h)
        return
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    _check(load_library().dirac_set_absorber(h, a.ctypes.data, a.size), h)


def dirac_set_vector_potential(h, A_tilde) -> None:
    """Uniform vector-potential field integrals, an (nsteps, 3) array (None: remove the field)."""
    if A_tilde is None:
        _check(load_library().dirac_set_vector_potential(h, None, 0), h)
        return
    At = np.ascontiguousarray(A_tilde, dtype=np.float64).reshape(-1, 3)
    _check(load_library().dirac_set_vector_potential(h, At.ctypes.data, At.shape[0]), h)


def dirac_set_field(h, a, w, F) -> None:
    """Separable space-time field: a (3 per cell, or None), w (1 per cell, or None) and the (nsteps, 4) envelope
    integrals F = (F_x, F_y, F_z, F_V) per step (None: remove the field)."""
    if F is None:
        _check(load_library().dirac_set_field(h, None, None, None, 0), h)
        return
    Fa = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, 4)
    aa = None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    _check(load_library().dirac_set_field(h, None if aa is None else aa.ctypes.data,
                                          None if ww is None else ww.ctypes.data, Fa.ctypes.data, Fa.shape[0]), h)


def dirac_set_counters(h, step: int, flux_cum: float) -> None:
    _check(load_library().dirac_set_counters(h, int(step), float(flux_cum)), h)


def dirac_get_info(h) -> dict:
    info = dirac_info()
    _check(load_library().dirac_get_info(h, ctypes.byref(info)), h)
    return {f: getattr(info, f) for f, _ in dirac_info._fields_}


def dirac_autotune(h) -> None:
    _check(load_library().dirac_autotune(h), h)


def dirac_last_error(h=None) -> str:
    return load_library().dirac_last_error(h).decode()


def make_config(n, ndim: int = 2, dx: float | None = None, precision: int = DIRAC_FP64,
                boundary: int = DIRAC_BC_ZERO, x_min=None, flux_face: int = -1, stream=None,
                device: int = 0, steps_per_launch: int = 0, use_graphs: bool = True,
                c: float | None = None, m: float | None = None, points_per_lane: int = 0,
                splitting: int = 0, char_shift: int = 0, ext_state=None) -> dirac_config:
    """dirac_default_config() with the given fields replaced (n = (nx, ny, nz)).  ext_state: two caller-owned
    device buffers (torch CUDA tensors or raw device addresses) the grid uses as its ping-pong state buffers."""
    cfg = dirac_default_config()
    cfg.ndim = ndim
    for d in range(3):
        cfg.n[d] = int(n[d])
    if dx is not None:
        cfg.dx = dx
    if c is not None:
        cfg.c = c
    if m is not None:
        cfg.m = m
    if x_min is None:
        x_min = tuple(-0.5 * n[d] * cfg.dx for d in range(3))
    for d in range(3):
        cfg.x_min[d] = x_min[d]
    cfg.precision = precision
    cfg.boundary = boundary
    cfg.flux_face = flux_face
    cfg.stream = stream
    cfg.device = device
    cfg.steps_per_launch = steps_per_launch
    cfg.use_graphs = 1 if use_graphs else 0
    cfg.points_per_lane = points_per_lane
    cfg.splitting = splitting
    cfg.char_shift = char_shift
    if ext_state is not None:
        if len(ext_state) != 2:
            raise ValueError("ext_state takes two buffers")
        for i, b in enumerate(ext_state):
            cfg.ext_state[i] = b.data_ptr() if hasattr(b, "data_ptr") else b
    return cfg


# ----------------------------------------------------------------------------- batched ensemble

class dirac_klein_run(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int64), ("face", ctypes.c_int64), ("nsteps", ctypes.c_int64),
                ("V0", ctypes.c_double), ("L", ctypes.c_double), ("p0", ctypes.c_double),
                ("width", ctypes.c_double), ("x0", ctypes.c_double), ("absorb", ctypes.c_int64),
                ("eta", ctypes.c_double)]


class dirac_batch_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("dx", ctypes.c_double), ("c", ctypes.c_double),
                ("m", ctypes.c_double), ("stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("steps_per_launch", ctypes.c_int), ("points_per_lane", ctypes.c_int),
                ("segment_rows", ctypes.c_int64), ("use_graphs", ctypes.c_int)]


class dirac_batch_info(ctypes.Structure):
    _fields_ = [("steps_per_launch", ctypes.c_int), ("points_per_lane", ctypes.c_int),
                ("segment_rows", ctypes.c_int64), ("launches", ctypes.c_int64), ("max_tasks", ctypes.c_int64),
                ("point_steps", ctypes.c_int64), ("blocks", ctypes.c_int), ("device_bytes", ctypes.c_size_t)]


def _batch_lib():
    lib = load_library()
    if getattr(lib, "_batch_sigs", False):
        return lib
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    DP = ctypes.POINTER(ctypes.c_double)
    sig = {
        "dirac_batch_default_config": (None, [ctypes.POINTER(dirac_batch_config)]),
        "dirac_batch_create": (I, [ctypes.POINTER(dirac_klein_run), I, ctypes.POINTER(dirac_batch_config),
                                   ctypes.POINTER(P)]),
        "dirac_batch_destroy": (I, [P]),
        "dirac_batch_reset": (I, [P]),
        "dirac_batch_set_state": (I, [P, I, P, I]),
        "dirac_batch_set_potential": (I, [P, I, P, I64]),
        "dirac_batch_set_absorber": (I, [P, I, P, I64]),
        "dirac_batch_run": (I, [P]),
        "dirac_batch_results": (I, [P, DP, DP, DP]),
        "dirac_batch_get_state": (I, [P, I, P, I]),
        "dirac_batch_autotune": (I, [P]),
        "dirac_batch_get_info": (I, [P, ctypes.POINTER(dirac_batch_info)]),
        "dirac_batch_last_error": (ctypes.c_char_p, [P]),
        "dirac_batch_klein": (I, [ctypes.POINTER(dirac_klein_run), I, ctypes.POINTER(dirac_batch_config), DP, DP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    lib._batch_sigs = True
    return lib


def _bcheck(st: int, handle=None):
    if st != DIRAC_OK:
        msg = _batch_lib().dirac_batch_last_error(handle)
        raise DiracError(st, msg.decode() if msg else "")


def klein_runs_array(runs) -> "ctypes.Array":
    """ctypes array of dirac_klein_run from objects with side, face, nsteps, V0, L, p0, width, x0 (or dicts)."""
    arr = (dirac_klein_run * len(runs))()
    for i, r in enumerate(runs):
        get = (lambda k: r.get(k, 0)) if isinstance(r, dict) else (lambda k: getattr(r, k, 0))
        for f, _ in dirac_klein_run._fields_:
            setattr(arr[i], f, get(f))
    return arr


def dirac_batch_default_config() -> dirac_batch_config:
    cfg = dirac_batch_config()
    _batch_lib().dirac_batch_default_config(ctypes.byref(cfg))
    return cfg


def dirac_batch_create(runs, cfg: dirac_batch_config) -> ctypes.c_void_p:
    arr = runs if isinstance(runs, ctypes.Array) else klein_runs_array(runs)
    h = ctypes.c_void_p()
    _bcheck(_batch_lib().dirac_batch_create(arr, len(arr), ctypes.byref(cfg), ctypes.byref(h)))
    return h


def dirac_batch_destroy(h) -> None:
    _bcheck(_batch_lib().dirac_batch_destroy(h))


def dirac_batch_reset(h) -> None:
    _bcheck(_batch_lib().dirac_batch_reset(h), h)


def dirac_batch_set_state(h, run: int, psi) -> None:
    p, dev = _ptr(psi, 8)
    _bcheck(_batch_lib().dirac_batch_set_state(h, int(run), p, dev), h)


def dirac_batch_set_potential(h, run: int, V) -> None:
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
    _bcheck(_batch_lib().dirac_batch_set_potential(h, int(run), V.ctypes.data, V.size), h)


def dirac_batch_set_absorber(h, run: int, a) -> None:
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    _bcheck(_batch_lib().dirac_batch_set_absorber(h, int(run), a.ctypes.data, a.size), h)


def dirac_batch_run(h) -> None:
    _bcheck(_batch_lib().dirac_batch_run(h), h)


def dirac_batch_results(h, nruns: int) -> dict:
    T = np.zeros(nruns)
    F = np.zeros(nruns)
    N = np.zeros(nruns)
    dp = ctypes.POINTER(ctypes.c_double)
    _bcheck(_batch_lib().dirac_batch_results(h, T.ctypes.data_as(dp), F.ctypes.data_as(dp), N.ctypes.data_as(dp)), h)
    return {"T": T, "flux": F, "norm0": N}


def dirac_batch_get_state(h, run: int, out) -> None:
    p, dev = _ptr(out, 8)
    _bcheck(_batch_lib().dirac_batch_get_state(h, int(run), p, dev), h)


def dirac_batch_autotune(h) -> None:
    _bcheck(_batch_lib().dirac_batch_autotune(h), h)


def dirac_batch_get_info(h) -> dict:
    info = dirac_batch_info()
    _bcheck(_batch_lib().dirac_batch_get_info(h, ctypes.byref(info)), h)
    return {f: getattr(info, f) for f, _ in dirac_batch_info._fields_}


def dirac_batch_klein(runs, cfg: dirac_batch_config):
    """(T, R) arrays for the runs, in one call."""
    arr = runs if isinstance(runs, ctypes.Array) else klein_runs_array(runs)
    T = np.zeros(len(arr))
    R = np.zeros(len(arr))
    dp = ctypes.POINTER(ctypes.c_double)
    _bcheck(_batch_lib().dirac_batch_klein(arr, len(arr), ctypes.byref(cfg), T.ctypes.data_as(dp), R.ctypes.data_as(dp)))
    return T, R


# ----------------------------------------------------------------------------- transmission surrogate

def _sur_lib():
    lib = _batch_lib()
    if getattr(lib, "_sur_sigs", False):
        return lib
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "dirac_surrogate_create": (I, [P, P, ctypes.c_uint64, I, P, I, ctypes.POINTER(P)]),
        "dirac_surrogate_destroy": (I, [P]),
        "dirac_surrogate_train": (I, [P, P, P, I64, I, I, D, P]),
        "dirac_surrogate_predict": (I, [P, P, I64, P]),
        "dirac_surrogate_gradient": (I, [P, P, P, I64, P, P]),
        "dirac_surrogate_num_params": (I64, []),
        "dirac_surrogate_get_params": (I, [P, P]),
        "dirac_surrogate_set_params": (I, [P, P]),
        "dirac_surrogate_save": (I, [P, ctypes.c_char_p]),
        "dirac_surrogate_load": (I, [P, ctypes.c_char_p]),
        "dirac_surrogate_query": (I, [P, P, I64, ctypes.POINTER(dirac_batch_config), P, P]),
        "dirac_klein_run_from_reduced": (I, [P, D, D, D, ctypes.POINTER(dirac_klein_run)]),
        "dirac_surrogate_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    lib._sur_sigs = True
    return lib


def _scheck(st, handle=None):
    if st != DIRAC_OK:
        msg = _sur_lib().dirac_surrogate_last_error(handle)
        raise DiracError(st, msg.decode() if msg else "")


def _f64(a, cols=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def dirac_surrogate_create(lo, hi, seed: int = 0, max_batch: int = 4096, stream=None, device: int = 0):
    lo, hi = _f64(lo), _f64(hi)
    h = ctypes.c_void_p()
    _scheck(_sur_lib().dirac_surrogate_create(lo.ctypes.data, hi.ctypes.data, seed, max_batch, stream, device,
                                              ctypes.byref(h)))
    return h


def dirac_surrogate_destroy(h) -> None:
    _scheck(_sur_lib().dirac_surrogate_destroy(h))


def dirac_surrogate_train(h, X, T, epochs: int, batch: int, lr: float) -> float:
    X, T = _f64(X), _f64(T)
    loss = ctypes.c_double()
    _scheck(_sur_lib().dirac_surrogate_train(h, X.ctypes.data, T.ctypes.data, len(T), epochs, batch, lr,
                                             ctypes.addressof(loss)), h)
    return loss.value


def dirac_surrogate_predict(h, X) -> np.ndarray:
    X = _f64(X)
    out = np.zeros(X.shape[0])
    _scheck(_sur_lib().dirac_surrogate_predict(h, X.ctypes.data, X.shape[0], out.ctypes.data), h)
    return out


def dirac_surrogate_gradient(h, X, T):
    X, T = _f64(X), _f64(T)
    g = np.zeros(_sur_lib().dirac_surrogate_num_params(), dtype=np.float32)
    loss = ctypes.c_double()
    _scheck(_sur_lib().dirac_surrogate_gradient(h, X.ctypes.data, T.ctypes.data, len(T), g.ctypes.data,
                                                ctypes.addressof(loss)), h)
    return loss.value, g


def dirac_surrogate_get_params(h) -> np.ndarray:
    p = np.zeros(_sur_lib().dirac_surrogate_num_params(), dtype=np.float32)
    _scheck(_sur_lib().dirac_surrogate_get_params(h, p.ctypes.data), h)
    return p


def dirac_surrogate_set_params(h, params) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    _scheck(_sur_lib().dirac_surrogate_set_params(h, p.ctypes.data), h)


def dirac_surrogate_save(h, path: str) -> None:
    """Checkpoint: box, FP32 parameters and Adam state to the file at path."""
    _scheck(_sur_lib().dirac_surrogate_save(h, os.fsencode(path)), h)


def dirac_surrogate_load(h, path: str) -> None:
    """Restores box, parameters and Adam state from a checkpoint written by dirac_surrogate_save."""
    _scheck(_sur_lib().dirac_surrogate_load(h, os.fsencode(path)), h)


def dirac_surrogate_query(h, X, solver_cfg: dirac_batch_config):
    X = _f64(X)
    T = np.zeros(X.shape[0])
    used = np.zeros(X.shape[0], dtype=np.int32)
    _scheck(_sur_lib().dirac_surrogate_query(h, X.ctypes.data, X.shape[0], ctypes.byref(solver_cfg), T.ctypes.data,
                                             used.ctypes.data), h)
    return T, used.astype(bool)


def dirac_klein_run_from_reduced(q, dx: float, c: float, m: float) -> dict:
    q = _f64(q)
    run = dirac_klein_run()
    _scheck(_sur_lib().dirac_klein_run_from_reduced(q.ctypes.data, dx, c, m, ctypes.byref(run)))
    return {f: getattr(run, f) for f, _ in dirac_klein_run._fields_}
