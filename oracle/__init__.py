"""FP64 CPU oracle of the split-operator Dirac scheme.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports, links or executes anything here, and nothing here imports the product.

``dirac_oracle.c`` holds the scheme itself (sweeps of Eqs. sol_dis_1-3, the
phase of Eq. sol_dis_4 at A = 0, the face flux and the observables).  This
module compiles it with gcc (``-ffp-contract=off``) and wraps it with ctypes.
``klein.py`` holds the Klein-step transmission: the closed form of Eq. trans_co
and a transfer integration of the stationary Dirac equation.

State arrays are complex128 of shape (nz, ny, nx, 4), C-contiguous (ny = 1 for
the 2-D x-z plane).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dirac_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

I64_3 = ctypes.c_int64 * 3
D3 = ctypes.c_double * 3


def build(force: bool = False) -> str:
    """Compile the oracle to oracle/_build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        lib.oracle_sweep.argtypes = [P, I64_3, ctypes.c_int, ctypes.c_int]
        lib.oracle_phase.argtypes = [P, I64_3, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, ctypes.c_int]
        lib.oracle_step.argtypes = [P, I64_3, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P]
        lib.oracle_observables.argtypes = [P, I64_3, ctypes.c_int, ctypes.c_double, D3, ctypes.c_int64, P]
        lib.oracle_step_strang2d.argtypes = [P, I64_3, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P]
        lib.oracle_step_strang3d.argtypes = lib.oracle_step_strang2d.argtypes
        lib.oracle_step_fx.argtypes = [P, I64_3, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, P, ctypes.c_int, ctypes.c_int64]
        lib.oracle_step_strang2d_fx.argtypes = [P, I64_3, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, P, ctypes.c_int, ctypes.c_int64]
        lib.oracle_step_strang3d_fx.argtypes = lib.oracle_step_strang2d_fx.argtypes
        for f in (lib.oracle_sweep, lib.oracle_phase, lib.oracle_step, lib.oracle_observables,
                  lib.oracle_step_strang2d, lib.oracle_step_strang3d, lib.oracle_step_fx, lib.oracle_step_strang2d_fx,
                  lib.oracle_step_strang3d_fx):
            f.restype = ctypes.c_int
        lib.oracle_set_absorber.argtypes = [P]
        lib.oracle_set_absorber.restype = None
        lib.oracle_set_vector_potential.argtypes = [P, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_set_vector_potential.restype = None
        lib.oracle_set_shift.argtypes = [ctypes.c_int64]
        lib.oracle_set_shift.restype = None
        lib.oracle_set_field.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_set_field.restype = None
        _lib = lib
    return _lib


def _as_state(psi: np.ndarray) -> np.ndarray:
    psi = np.asarray(psi)
    if psi.ndim == 3:  # (nz, nx, 4): 2-D x-z plane
        psi = psi[:, None, :, :]
    if psi.ndim != 4 or psi.shape[-1] != 4:
        raise ValueError("state must have shape (nz, ny, nx, 4) or (nz, nx, 4)")
    return np.ascontiguousarray(psi, dtype=np.complex128).copy()


def _dims(psi: np.ndarray):
    nz, ny, nx, _ = psi.shape
    return I64_3(nx, ny, nz)


def _potential(V, psi):
    if V is None:
        return None, 0
    V = np.ascontiguousarray(V, dtype=np.float64)
    nz, ny, nx, _ = psi.shape
    if V.size == nx and V.ndim == 1:
        return V, 1
    if V.size == nx * ny * nz:
        return V.reshape(-1), 2
    raise ValueError("potential must have nx entries (one per x column) or one per cell")


class _Shift:
    """Context: characteristic shift K (c dt = K dx, Sec. 2.3); 1 outside the context."""
    def __init__(self, K):
        if int(K) < 1:
            raise ValueError("the characteristic shift must be >= 1")
        self.K = int(K)

    def __enter__(self):
        _load().oracle_set_shift(self.K)
        return self

    def __exit__(self, *exc):
        _load().oracle_set_shift(1)


def sweep(psi, axis: int, periodic: bool = False, shift: int = 1) -> np.ndarray:
    """One directional sub-step (Eq. sol_dis_1/2/3 for axis 0/1/2) with neighbours at +-shift cells; returns a
    new array."""
    out = _as_state(psi)
    with _Shift(shift):
        rc = _load().oracle_sweep(out.ctypes.data, _dims(out), int(axis), int(bool(periodic)))
    if rc != 0:
        raise MemoryError("oracle_sweep")
    return out


def phase(psi, m: float, c: float, dt: float, V=None) -> np.ndarray:
    """Mass and scalar-potential step (Eq. sol_dis_4 at A = 0); returns a new array."""
    out = _as_state(psi)
    Varr, layout = _potential(V, out)
    _load().oracle_phase(out.ctypes.data, _dims(out), float(m), float(c), float(dt),
                         None if Varr is None else Varr.ctypes.data, layout)
    return out


class _Absorber:
    """Context: per-x-column damping factors a(x) multiplied into the phase coefficients (None: none)."""
    def __init__(self, a, nx):
        self.a = None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        if self.a is not None and self.a.size != nx:
            raise ValueError("absorber needs one factor per x column")

    def __enter__(self):
        _load().oracle_set_absorber(None if self.a is None else self.a.ctypes.data)
        return self

    def __exit__(self, *exc):
        _load().oracle_set_absorber(None)


class _VectorPotential:
    """Context: per-step uniform vector-potential integrals At[n] = (At_x, At_y, At_z) (None: none)."""
    def __init__(self, At, step0):
        self.At = None if At is None else np.ascontiguousarray(At, dtype=np.float64).reshape(-1, 3)
        self.step0 = int(step0)

    def __enter__(self):
        if self.At is None:
            _load().oracle_set_vector_potential(None, 0, 0)
        else:
            _load().oracle_set_vector_potential(self.At.ctypes.data, self.At.shape[0], self.step0)
        return self

    def __exit__(self, *exc):
        _load().oracle_set_vector_potential(None, 0, 0)


class _Field:
    """Context: a separable space-time field (a, w, F) or None.  a: 3 values per cell (the profile of e A,
    [z][y][x][d]) or None; w: 1 value per cell (the profile of the time-dependent part of V) or None; F: (nt, 4)
    per-step integrals (F_x, F_y, F_z, F_V) of the envelopes; step s of a call uses row step0 + s."""
    def __init__(self, field, step0, ncells):
        self.field = field
        self.step0 = int(step0)
        if field is None:
            return
        a, w, F = field
        self.a = None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        self.w = None if w is None else np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
        self.F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, 4)
        if self.a is not None and self.a.size != 3 * ncells:
            raise ValueError("the field profile a needs 3 values per cell")
        if self.w is not None and self.w.size != ncells:
            raise ValueError("the field profile w needs 1 value per cell")

    def __enter__(self):
        if self.field is not None:
            _load().oracle_set_field(None if self.a is None else self.a.ctypes.data,
                                     None if self.w is None else self.w.ctypes.data, self.F.ctypes.data,
                                     self.F.shape[0], self.step0)
        return self

    def __exit__(self, *exc):
        _load().oracle_set_field(None, None, None, 0, 0)


def step(psi, ndim: int, m: float, c: float, dx: float, nsteps: int, V=None,
         periodic: bool = False, flux_face: int = -1, flux_cum: float = 0.0, absorber=None,
         A_tilde=None, step0: int = 0, shift: int = 1, field=None):
    """nsteps first-order split steps (Eqs. split1-4 discretised as sol_dis_1-4), dt = dx/c.

    Returns (psi_out, flux_cum): the cumulative probability carried across the x face
    `flux_face` (between cells flux_face-1 and flux_face), added to the given start value.
    `absorber`: optional per-x-column factors a(x) in (0, 1] applied with the phase (not in the paper).
    `A_tilde`: optional (nt, 3) array of uniform vector-potential integrals e int A dt per step (Eq. field_dis1);
    step s of this call uses row step0 + s, and the phase is the full matrix of Eq. sol_dis_4.
    `shift`: characteristic shift K, c dt = K dx (Sec. 2.3): dt = K dx / c and neighbours at +-K cells.
    `field`: optional separable space-time field (a, w, F) (see _Field): per cell and step the phase matrix of
    Eq. sol_dis_4 with At(i) = F_xyz a(i) and V~(i) = V(i) dt + F_V w(i) (Eqs. field_dis1, field_dis2).
    """
    out = _as_state(psi)
    Varr, layout = _potential(V, out)
    fc = ctypes.c_double(flux_cum)
    with _Absorber(absorber, out.shape[2]), _VectorPotential(A_tilde, step0), _Shift(shift), \
            _Field(field, step0, out.size // 4):
        rc = _load().oracle_step(out.ctypes.data, _dims(out), int(ndim), int(bool(periodic)), float(m), float(c),
                                 float(dx), None if Varr is None else Varr.ctypes.data, layout, int(nsteps),
                                 int(flux_face), ctypes.addressof(fc))
    if rc == -2:
        raise ValueError("the vector-potential table ends before the last step")
    if rc != 0:
        raise MemoryError("oracle_step")
    return out, fc.value


def step_strang2d(psi, m: float, c: float, dx: float, nsteps: int, V=None, periodic: bool = False,
                  flux_face: int = -1, flux_cum: float = 0.0, shift: int = 1, A_tilde=None, step0: int = 0,
                  field=None):
    """nsteps second-order (Strang) steps in the x-z plane (Sec. 2.4): x, z, phase(dt), z, x with
    dt = 2 dx / c.  A_tilde / step0: a uniform vector potential as in step() (the phase matrix over dt); field:
    a separable space-time field as in step(), its integrals spanning the whole step.
    Returns (psi_out, flux_cum) as step()."""
    out = _as_state(psi)
    if out.shape[1] != 1:
        raise ValueError("Strang steps are 2-D (ny = 1)")
    Varr, layout = _potential(V, out)
    fc = ctypes.c_double(flux_cum)
    with _Shift(shift), _VectorPotential(A_tilde, step0), _Field(field, step0, out.size // 4):
        rc = _load().oracle_step_strang2d(out.ctypes.data, _dims(out), int(bool(periodic)), float(m), float(c),
                                          float(dx), None if Varr is None else Varr.ctypes.data, layout, int(nsteps),
                                          int(flux_face), ctypes.addressof(fc))
    if rc == -2:
        raise ValueError("the vector-potential table ends before the last step")
    if rc != 0:
        raise MemoryError("oracle_step_strang2d")
    return out, fc.value


def step_strang3d(psi, m: float, c: float, dx: float, nsteps: int, V=None, periodic: bool = False,
                  flux_face: int = -1, flux_cum: float = 0.0, shift: int = 1, A_tilde=None, step0: int = 0,
                  field=None):
    """nsteps second-order (Strang) steps in 3-D (Sec. 2.4): A(dt/4) B(dt/2) A(dt/4) C(dt/2) D(dt) C(dt/2)
    A(dt/4) B(dt/2) A(dt/4) with c dt / 4 = shift * dx: x sweeps move `shift` cells, y and z sweeps 2 shift.
    A_tilde / step0: a uniform vector potential as in step() (the phase matrix over dt); field: a separable
    space-time field as in step(), its integrals spanning the whole step.
    Returns (psi_out, flux_cum) as step()."""
    out = _as_state(psi)
    Varr, layout = _potential(V, out)
    fc = ctypes.c_double(flux_cum)
    with _Shift(shift), _VectorPotential(A_tilde, step0), _Field(field, step0, out.size // 4):
        rc = _load().oracle_step_strang3d(out.ctypes.data, _dims(out), int(bool(periodic)), float(m), float(c),
                                          float(dx), None if Varr is None else Varr.ctypes.data, layout, int(nsteps),
                                          int(flux_face), ctypes.addressof(fc))
    if rc == -2:
        raise ValueError("the vector-potential table ends before the last step")
    if rc != 0:
        raise MemoryError("oracle_step_strang3d")
    return out, fc.value


def fx_encode(psi, S: int) -> np.ndarray:
    """Fixed-point state q = round(psi 2^S) (nearest, ties to even), int64 of shape (nz, ny, nx, 4, 2)."""
    arr = _as_state(psi)
    x = np.ldexp(arr.view(np.float64).reshape(arr.shape + (2,)), S)
    return np.rint(x).astype(np.int64)


def fx_decode(q, S: int) -> np.ndarray:
    """psi = q 2^-S as complex128 of shape (nz, ny, nx, 4)."""
    q = np.ascontiguousarray(q, dtype=np.int64)
    x = np.ldexp(q.astype(np.float64), -S)
    return x.view(np.complex128).reshape(q.shape[:-1])


def fx_shift(psi, ndim: int = 2, strang: bool = False) -> int:
    """The fixed-point shift for a state: S = 60 - e in 2-D (59 - e for 3-D first-order steps, 57 - e for 3-D
    second-order steps) where the discrete L2 norm sqrt(sum |psi_c|^2) = m 2^e with m in [0.5, 1); 0 for the
    zero state.  Each sweep with its 1/2 and the phase do not raise the norm, so a step's values (2^j times
    it after j sweeps without the 1/2: j = 2, 3, 4 before the phase) stay below 2^62."""
    arr = _as_state(psi)
    A = float(np.sqrt(np.sum(arr.real ** 2 + arr.imag ** 2)))
    top = (57 if strang else 59) if ndim == 3 else 60
    return top - (np.frexp(A)[1] if A > 0 else top)


def step_fx(q, m: float, c: float, dx: float, nsteps: int, V=None, periodic: bool = False, absorber=None,
            ndim: int = 2):
    """nsteps first-order steps on a fixed-point state q (int64, (nz, ny, nx, 4, 2); ny = 1 in 2-D): exact
    integer sweeps without the 1/2 factors, the phase coefficients (carrying 1/4, or 1/8 in 3-D) held as
    round(p/4 2^62) and each output component rounded once after the exact 128-bit product
    (oracle_step_fx).  Returns the new q."""
    out = np.ascontiguousarray(q, dtype=np.int64).copy()
    if out.ndim != 5 or out.shape[3:] != (4, 2) or (ndim == 2 and out.shape[1] != 1):
        raise ValueError("q must have shape (nz, ny, nx, 4, 2), ny = 1 in 2-D")
    nz, ny, nx = out.shape[:3]
    Varr, layout = _potential(V, np.zeros((nz, ny, nx, 4), complex))
    with _Absorber(absorber, nx):
        rc = _load().oracle_step_fx(out.ctypes.data, I64_3(nx, ny, nz), int(ndim), int(bool(periodic)), float(m),
                                    float(c), float(dx), None if Varr is None else Varr.ctypes.data, layout,
                                    int(nsteps))
    if rc != 0:
        raise MemoryError("oracle_step_fx")
    return out


def step_strang2d_fx(q, m: float, c: float, dx: float, nsteps: int, V=None, periodic: bool = False, absorber=None):
    """nsteps second-order 2-D steps (x, z, phase over 2 dx / c, z, x; Sec. 2.4) on a fixed-point state q
    (int64, (nz, 1, nx, 4, 2)): exact integer sweeps, the phase coefficients carrying the four sweeps' halves
    (1/16) as round(p/16 2^62), each output component rounded once (oracle_step_strang2d_fx)."""
    out = np.ascontiguousarray(q, dtype=np.int64).copy()
    if out.ndim != 5 or out.shape[1] != 1 or out.shape[3:] != (4, 2):
        raise ValueError("q must have shape (nz, 1, nx, 4, 2)")
    nz, ny, nx = out.shape[:3]
    Varr, layout = _potential(V, np.zeros((nz, ny, nx, 4), complex))
    with _Absorber(absorber, nx):
        rc = _load().oracle_step_strang2d_fx(out.ctypes.data, I64_3(nx, ny, nz), int(bool(periodic)), float(m),
                                             float(c), float(dx), None if Varr is None else Varr.ctypes.data,
                                             layout, int(nsteps))
    if rc != 0:
        raise MemoryError("oracle_step_strang2d_fx")
    return out


def step_strang3d_fx(q, m: float, c: float, dx: float, nsteps: int, V=None, periodic: bool = False):
    """nsteps second-order 3-D steps (Sec. 2.4: A(1) B(2) A(1) C(2) D C(2) A(1) B(2) A(1), dt = 4 dx / c) on a
    fixed-point state q (int64, (nz, ny, nx, 4, 2)), the eight halves (1/256) in the phase coefficients
    (oracle_step_strang3d_fx)."""
    out = np.ascontiguousarray(q, dtype=np.int64).copy()
    if out.ndim != 5 or out.shape[3:] != (4, 2):
        raise ValueError("q must have shape (nz, ny, nx, 4, 2)")
    nz, ny, nx = out.shape[:3]
    Varr, layout = _potential(V, np.zeros((nz, ny, nx, 4), complex))
    rc = _load().oracle_step_strang3d_fx(out.ctypes.data, I64_3(nx, ny, nz), int(bool(periodic)), float(m),
                                         float(c), float(dx), None if Varr is None else Varr.ctypes.data, layout,
                                         int(nsteps))
    if rc != 0:
        raise MemoryError("oracle_step_strang3d_fx")
    return out


def observables(psi, ndim: int, dx: float, x_min=(0.0, 0.0, 0.0), flux_face: int = -1) -> dict:
    """norm, norm right of the flux face and centroid, summed in index order."""
    arr = _as_state(psi)
    out = (ctypes.c_double * 5)()
    _load().oracle_observables(arr.ctypes.data, _dims(arr), int(ndim), float(dx), D3(*x_min),
                               int(flux_face), ctypes.addressof(out))
    return {"norm": out[0], "norm_right": out[1], "centroid": (out[2], out[3], out[4])}


def density(psi) -> np.ndarray:
    """rho = sum_c |psi_c|^2 per cell, shape (nz, ny, nx)."""
    arr = _as_state(psi)
    return (arr.real ** 2 + arr.imag ** 2).sum(axis=-1)
