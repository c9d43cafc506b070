"""The oracle pins catch plausible mistakes: each mutant below is a copy of the oracle's C source with one
planted error (a flipped sign, swapped neighbours, a dropped factor, a wrong component, a wrong phase
sign, a flux sign, a centroid or face off by a cell or an axis), built into a temporary library; at least one pin check must reject it.  CPU only."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1107_4650_gb300 import workloads as W
from tests import dirac_algebra as A
from tests.test_oracle_pins import _fx_step_bigint, _fx_strang3d_free_periodic

SRC = os.path.join(os.path.dirname(oracle.__file__), "dirac_oracle.c")
C = W.C_AU
DX = W.DX_DEFAULT

MUTANTS = {
    "x_sweep_sign": ("o[3] = c_half(c_add(c_add(L[0], L[3]), c_sub(R[3], R[0])));",
                     "o[3] = c_half(c_add(c_add(L[0], L[3]), c_sub(R[0], R[3])));"),
    "x_sweep_neighbours_swapped": ("o[0] = c_half(c_add(c_add(L[0], L[3]), c_sub(R[0], R[3])));",
                                   "o[0] = c_half(c_add(c_add(R[0], R[3]), c_sub(L[0], L[3])));"),
    "z_sweep_component": ("o[1] = c_half(c_add(c_sub(L[1], L[3]), c_add(R[1], R[3])));",
                          "o[1] = c_half(c_add(c_sub(L[1], L[2]), c_add(R[1], R[3])));"),
    "y_sweep_i_sign": ("o[0] = c_half(c_add(c_sub_ib(L[0], L[3]), c_add_ib(R[0], R[3])));",
                       "o[0] = c_half(c_add(c_add_ib(L[0], L[3]), c_sub_ib(R[0], R[3])));"),
    "dropped_half": ("o[2] = c_half(c_add(c_add(L[0], L[2]), c_sub(R[2], R[0])));",
                     "o[2] = c_add(c_add(L[0], L[2]), c_sub(R[2], R[0]));"),
    "phase_mass_sign": ("double t_dn = vdt - mu;", "double t_dn = vdt + mu;"),
    "phase_conjugate": ("cplx p_up = {cos(t_up), -sin(t_up)};", "cplx p_up = {cos(t_up), sin(t_up)};"),
    "flux_sign": ("f += right - left;", "f += right + left;"),
    "boundary_wrap_off_by_one": ("i = ((i % n[0]) + n[0]) % n[0];", "i = ((i % n[0]) + n[0] + 1) % n[0];"),
    "A_z_entry_sign": ("U[1][3].im = -az; U[3][1].im = -az;", "U[1][3].im = az; U[3][1].im = -az;"),
    "A_y_entry_sign": ("U[0][3].re = ay;  U[0][3].im = ax;", "U[0][3].re = -ay;  U[0][3].im = ax;"),
    "A_mass_term_sign": ("U[0][0].re = cA; U[0][0].im = -ms;", "U[0][0].re = cA; U[0][0].im = ms;"),
    "shift_ignored_in_sweep": ("d[axis] = shift;", "d[axis] = 1;"),
    "shift_flux_window": ("for (int64_t i = face - g_shift; i < face; ++i) {", "for (int64_t i = face - 1; i < face; ++i) {"),
    "shift_time_step": ("double dt = (double)g_shift * dx / c;", "double dt = dx / c;"),
    "strang3d_order": ("const int axes[9] = {0, 1, 0, 2, -1, 2, 0, 1, 0};", "const int axes[9] = {1, 0, 0, 2, -1, 2, 0, 1, 0};"),
    "strang3d_half_step_shift": ("ax == 0 ? g_shift : 2 * g_shift", "ax == 0 ? g_shift : g_shift"),
    "A_row_order": ("acc = c_mac(acc, q[b], c_mul(U[a][b], g));", "acc = c_mac(acc, q[b], c_mul(U[b][a], g));"),
    "fx_rounding_offset": ("return (int64_t)((v + ((__int128)1 << 61)) >> 62);",
                           "return (int64_t)((v + ((__int128)1 << 60)) >> 62);"),
    "fx_z_sweep_sign": ("z[3].re = (L[3].re - L[1].re) + (R[1].re + R[3].re);",
                        "z[3].re = (L[1].re - L[3].re) + (R[1].re + R[3].re);"),
    "fx_coefficient_scale": ("return (int64_t)nearbyint(ldexp(p * halves, 62));",
                             "return (int64_t)nearbyint(ldexp(p * halves, 61));"),
    "fx_x_sweep_neighbour": ("const qcplx *L = qcell(in, n, periodic, i - sh, j, k), *R = qcell(in, n, periodic, i + sh, j, k);",
                             "const qcplx *L = qcell(in, n, periodic, i - sh, j, k), *R = qcell(in, n, periodic, i - sh, j, k);"),
    "fx_y_sweep_i_sign": ("o[0].re = (L[0].re + L[3].im) + (R[0].re - R[3].im);",
                          "o[0].re = (L[0].re - L[3].im) + (R[0].re - R[3].im);"),
    "fx_3d_halves": ("const double halves = ndim == 3 ? 0.125 : 0.25;", "const double halves = 0.25;"),
    "fx_strang_halves": ("fx_phase(q, n, m, c, 2.0 * dx / c, V, layout, 0.0625);", "fx_phase(q, n, m, c, 2.0 * dx / c, V, layout, 0.125);"),
    "fx_strang_order": ("        fx_sweep_z(q, t, n, periodic, 1);\n        fx_sweep_x(t, q, n, periodic, 1);\n    }",
                        "        fx_sweep_x(q, t, n, periodic, 1);\n        fx_sweep_z(t, q, n, periodic, 1);\n    }"),
    "fx_strang3d_final_rounding": ("q_d[e] = (q_d[e] + 8) >> 4;", "q_d[e] = (q_d[e] + 0) >> 4;"),
    "centroid_half_cell": ("sx += (x_min[0] + (i + 0.5) * dx) * rho;", "sx += (x_min[0] + i * dx) * rho;"),
    "centroid_y_index": ("sy += (x_min[1] + (j + 0.5) * dx) * rho;", "sy += (x_min[1] + (k + 0.5) * dx) * rho;"),
    "norm_right_off_by_one": ("if (flux_face >= 0 && i >= flux_face) sr += rho;",
                              "if (flux_face >= 0 && i > flux_face) sr += rho;"),
    "field_profile_component": ("for (int d = 0; d < 3; ++d) At[d] = F[d] * g_fa[3 * cidx + d];",
                                "for (int d = 0; d < 3; ++d) At[d] = F[d] * g_fa[3 * cidx];"),
    "field_scalar_envelope": ("if (g_fw) vt = vt + F[3] * g_fw[cidx];", "if (g_fw) vt = vt + F[2] * g_fw[cidx];"),
    "field_step_row": ("return oracle_phase_field(psi, n, m, c, dt, V, layout, g_fenv + 4 * t);",
                       "return oracle_phase_field(psi, n, m, c, dt, V, layout, g_fenv + 4 * s);"),
    "fx_strang3d_shift": ("        fx_sweep_y(t, q, n, periodic, 2);\n        fx_sweep_x(q, t, n, periodic, 1);\n        fx_sweep_z(t, q, n, periodic, 2);",
                          "        fx_sweep_y(t, q, n, periodic, 1);\n        fx_sweep_x(q, t, n, periodic, 1);\n        fx_sweep_z(t, q, n, periodic, 2);"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / ("%s.c" % name)
    path.write_text(src.replace(old, new))
    so = tmp_path / ("lib%s.so" % name)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", str(path), "-o", str(so), "-lm"])
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    lib.oracle_sweep.argtypes = [P, oracle.I64_3, ctypes.c_int, ctypes.c_int]
    lib.oracle_step.argtypes = [P, oracle.I64_3, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P]
    lib.oracle_observables.argtypes = [P, oracle.I64_3, ctypes.c_int, ctypes.c_double, oracle.D3, ctypes.c_int64, P]
    lib.oracle_set_absorber.argtypes = [P]
    lib.oracle_set_absorber.restype = None
    lib.oracle_set_vector_potential.argtypes = [P, ctypes.c_int64, ctypes.c_int64]
    lib.oracle_set_vector_potential.restype = None
    lib.oracle_step_strang3d.argtypes = [P, oracle.I64_3, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P]
    lib.oracle_step_strang2d.argtypes = lib.oracle_step_strang3d.argtypes
    lib.oracle_set_shift.argtypes = [ctypes.c_int64]
    lib.oracle_set_shift.restype = None
    lib.oracle_set_field.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int64]
    lib.oracle_set_field.restype = None
    lib.oracle_step_fx.argtypes = [P, oracle.I64_3, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, P, ctypes.c_int, ctypes.c_int64]
    lib.oracle_step_fx.restype = ctypes.c_int
    lib.oracle_step_strang2d_fx.argtypes = [P, oracle.I64_3, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, P, ctypes.c_int, ctypes.c_int64]
    lib.oracle_step_strang2d_fx.restype = ctypes.c_int
    lib.oracle_step_strang3d_fx.argtypes = lib.oracle_step_strang2d_fx.argtypes
    lib.oracle_step_strang3d_fx.restype = ctypes.c_int
    return lib


def _pins_pass():
    """The quick pins of test_oracle_pins, run against whatever library oracle._lib holds."""
    ok = True
    for shape, axis, per in [((5, 1, 4), 0, False), ((5, 1, 4), 2, True), ((3, 4, 2), 1, False), ((4, 3, 2), 0, True)]:
        nx, ny, nz = shape
        psi = W.random_state(nz, ny, nx, seed=31 + axis)
        got = oracle.sweep(psi, axis, per)
        ok &= np.max(np.abs(got.reshape(-1) - A.sweep_matrix(shape, axis, per) @ psi.reshape(-1))) < 1e-15
    for ndim, shape in [(2, (6, 1, 5)), (3, (3, 4, 3))]:
        nx, ny, nz = shape
        psi = W.random_state(nz, ny, nx, seed=5)
        V = np.random.default_rng(3).uniform(-3e4, 3e4, nx * ny * nz)
        got, _ = oracle.step(psi, ndim, 1.0, C, DX, 1, V=V, periodic=False)
        step = A.sweep_matrix(shape, 2, False) @ (
            A.sweep_matrix(shape, 1, False) @ A.sweep_matrix(shape, 0, False) if ndim == 3 else A.sweep_matrix(shape, 0, False))
        want = A.phase_matrix(shape, 1.0, C, DX / C, V) @ step @ psi.reshape(-1)
        ok &= np.max(np.abs(got.reshape(-1) - want)) < 5e-15
    run = W.KleinRun(side=160, V0=2.5 * C * C, p0=0.7 * C, width=5 * DX, nsteps=20, face=80)
    psi0 = run.state()
    x_min, z_min, _, _, face = run.geometry()
    o0 = oracle.observables(psi0, 2, DX, (x_min, 0.0, z_min), face)
    out, F = oracle.step(psi0, 2, 1.0, C, DX, run.nsteps, V=run.potential(), flux_face=face)
    o1 = oracle.observables(out, 2, DX, (x_min, 0.0, z_min), face)
    ok &= abs((o1["norm_right"] - o0["norm_right"]) - F) < 1e-13
    # uniform vector potential: one-cell phase against the matrix exponential, Fourier evolution
    rng = np.random.default_rng(12)
    At = rng.uniform(-1.5, 1.5, (3, 3))
    psi = rng.standard_normal((1, 1, 1, 4)) + 1j * rng.standard_normal((1, 1, 1, 4))
    got, _ = oracle.step(psi, 2, 1.0, C, DX, 3, V=np.array([2e4]), periodic=True, A_tilde=At)
    want = psi.reshape(4)
    for a in At:
        want = A.phase_matrix_A_cell(1.0, C, DX / C, 2e4, a) @ want
    ok &= np.max(np.abs(got.reshape(4) - want)) < 1e-13
    psi = W.random_state(9, 1, 10, seed=93)
    got, _ = oracle.step(psi, 2, 1.0, C, DX, 4, periodic=True, A_tilde=At[[0, 1, 2, 0]])
    ok &= A.rel_l2(got, A.dft_exact_evolution_2d_A(psi, C * DX, At[[0, 1, 2, 0]])) < 1e-13
    # characteristic shift 3: explicit sweep matrix, Fourier evolution, flux identity
    psi = W.random_state(5, 1, 8, seed=94)
    got = oracle.sweep(psi, 0, False, shift=3)
    ok &= np.max(np.abs(got.reshape(-1) - A.sweep_matrix((8, 1, 5), 0, False, shift=3) @ psi.reshape(-1))) < 1e-15
    psi = W.random_state(12, 1, 14, seed=95)
    got, _ = oracle.step(psi, 2, 1.0, C, DX, 3, periodic=True, shift=3)
    ok &= A.rel_l2(got, A.dft_exact_evolution_2d(psi, 3, C * 3 * DX, shift=3)) < 1e-13
    run = W.KleinRun(side=200, V0=2.5 * C * C, p0=0.7 * C, width=6 * DX, nsteps=12, face=100)
    psi0 = run.state()
    x_min, z_min, _, _, face = run.geometry()
    o0 = oracle.observables(psi0, 2, DX, (x_min, 0.0, z_min), face)
    out, F = oracle.step(psi0, 2, 1.0, C, DX, run.nsteps, V=run.potential(), flux_face=face, shift=3)
    o1 = oracle.observables(out, 2, DX, (x_min, 0.0, z_min), face)
    ok &= abs((o1["norm_right"] - o0["norm_right"]) - F) < 1e-13
    # 3-D Strang step against its explicit matrix product
    shape = (5, 7, 6)  # 7 rows: a two-cell y shift does not wrap onto itself
    psi = W.random_state(6, 7, 5, seed=96)
    Vc = np.random.default_rng(97).uniform(-3e4, 3e4, 210)
    got, _ = oracle.step_strang3d(psi, 1.0, C, DX, 1, V=Vc, periodic=True)
    Ax, By, Cz = (A.sweep_matrix(shape, 0, True), A.sweep_matrix(shape, 1, True, shift=2),
                  A.sweep_matrix(shape, 2, True, shift=2))
    want = Ax @ By @ Ax @ Cz @ A.phase_matrix(shape, 1.0, C, 4 * DX / C, Vc) @ Cz @ Ax @ By @ Ax @ psi.reshape(-1)
    ok &= np.max(np.abs(got.reshape(-1) - want)) < 5e-15
    # fixed-point step: exact big-integer brute force, and exactness where FP64 is exact
    rng = np.random.default_rng(70)
    q = rng.integers(-(1 << 56), 1 << 56, size=(4, 1, 5, 4, 2), dtype=np.int64)
    Vq = rng.uniform(-3e4, 3e4, 5)
    dt = DX / C
    coef = lambda p: int(np.rint(np.ldexp(p * 0.25, 62)))
    P_up = [(coef(np.cos(C * C * dt + v * dt)), coef(-np.sin(C * C * dt + v * dt))) for v in Vq]
    P_dn = [(coef(np.cos(v * dt - C * C * dt)), coef(-np.sin(v * dt - C * C * dt))) for v in Vq]
    ok &= np.array_equal(oracle.step_fx(q, 1.0, C, DX, 1, V=Vq), _fx_step_bigint(q, P_up, P_dn, False))
    q = rng.integers(-1000, 1000, size=(7, 1, 9, 4, 2), dtype=np.int64) * 64
    want, _ = oracle.step(oracle.fx_decode(q, 40), 2, 0.0, C, DX, 3, periodic=True)
    ok &= np.array_equal(oracle.step_fx(q, 0.0, C, DX, 3, periodic=True), oracle.fx_encode(want, 40))
    q = rng.integers(-1000, 1000, size=(5, 4, 6, 4, 2), dtype=np.int64) * 512
    want, _ = oracle.step(oracle.fx_decode(q, 40), 3, 0.0, C, DX, 3, periodic=True)
    ok &= np.array_equal(oracle.step_fx(q, 0.0, C, DX, 3, periodic=True, ndim=3), oracle.fx_encode(want, 40))
    psi = W.random_state(6, 5, 7, seed=98)
    S = oracle.fx_shift(psi, 3)
    Vr = np.random.default_rng(99).uniform(-3e4, 3e4, 210)
    want, _ = oracle.step(psi, 3, 1.0, C, DX, 4, V=Vr, periodic=True)
    got = oracle.fx_decode(oracle.step_fx(oracle.fx_encode(psi, S), 1.0, C, DX, 4, V=Vr, periodic=True, ndim=3), S)
    ok &= A.rel_l2(got, want) < 1e-13
    # fixed-point second-order 2-D step: exact where FP64 is exact, and within 1e-13 of the FP64 Strang step
    q = rng.integers(-1000, 1000, size=(6, 1, 7, 4, 2), dtype=np.int64) * 4096
    want, _ = oracle.step_strang2d(oracle.fx_decode(q, 40), 0.0, C, DX, 3, periodic=True)
    ok &= np.array_equal(oracle.step_strang2d_fx(q, 0.0, C, DX, 3, periodic=True), oracle.fx_encode(want, 40))
    psi = W.random_state(9, 1, 11, seed=100)
    S = oracle.fx_shift(psi)
    Vr = np.random.default_rng(101).uniform(-3e4, 3e4, 11)
    want, _ = oracle.step_strang2d(psi, 1.0, C, DX, 5, V=Vr)
    ok &= A.rel_l2(oracle.fx_decode(oracle.step_strang2d_fx(oracle.fx_encode(psi, S), 1.0, C, DX, 5, V=Vr), S), want) < 1e-13
    # fixed-point second-order 3-D step: exact where FP64 is exact (7 rows: a two-cell shift does not wrap onto
    # itself), and within 1e-13 of the FP64 3-D Strang step
    q = rng.integers(-1000, 1000, size=(6, 7, 5, 4, 2), dtype=np.int64) * 65536
    want, _ = oracle.step_strang3d(oracle.fx_decode(q, 40), 0.0, C, DX, 2, periodic=True)
    ok &= np.array_equal(oracle.step_strang3d_fx(q, 0.0, C, DX, 2, periodic=True), oracle.fx_encode(want, 40))
    psi = W.random_state(6, 7, 5, seed=102)
    S = oracle.fx_shift(psi, 3, strang=True)
    Vr = np.random.default_rng(103).uniform(-3e4, 3e4, 210)
    want, _ = oracle.step_strang3d(psi, 1.0, C, DX, 3, V=Vr, periodic=True)
    got = oracle.fx_decode(oracle.step_strang3d_fx(oracle.fx_encode(psi, S), 1.0, C, DX, 3, V=Vr, periodic=True), S)
    ok &= A.rel_l2(got, want) < 1e-13
    q = rng.integers(-(1 << 40), 1 << 40, size=(6, 7, 5, 4, 2), dtype=np.int64)
    ok &= np.array_equal(oracle.step_strang3d_fx(q, 0.0, C, DX, 2, periodic=True), _fx_strang3d_free_periodic(q, 2))
    # a field varying from cell to cell: one step against the per-cell matrix exponentials (table row 1)
    shape = (5, 1, 4)
    psi = W.random_state(4, 1, 5, seed=104)
    rng = np.random.default_rng(105)
    Vf = rng.uniform(-3e4, 3e4, 20)
    a, w, F = rng.uniform(-1, 1, (20, 3)), rng.uniform(-2, 2, 20), rng.uniform(-1, 1, (3, 4))
    got, _ = oracle.step(psi, 2, 1.0, C, DX, 1, V=Vf, field=(a, w, F), step0=1)
    dtf = DX / C
    want = A.phase_matrix_field(shape, 1.0, C, dtf, Vf * dtf + F[1, 3] * w, F[1, :3][None, :] * a) @ \
        A.sweep_matrix(shape, 2, False) @ A.sweep_matrix(shape, 0, False) @ psi.reshape(-1)
    ok &= np.max(np.abs(got.reshape(-1) - want)) < 5e-15
    # observables of a one-cell 3-D state: norm, centroid = the cell's centre, norm right of the face
    psi = np.zeros((7, 6, 8, 4), np.complex128)
    psi[2, 3, 4] = [0.5 + 0.25j, -0.75j, 1.0, 0.5]
    for face, right in ((4, True), (5, False)):
        o = oracle.observables(psi, 3, 0.25, (-1.0, 0.5, 2.0), flux_face=face)
        ok &= o["norm"] == 2.125 * 0.25 ** 3 and o["norm_right"] == (o["norm"] if right else 0.0)
        ok &= max(abs(a - b) for a, b in zip(o["centroid"], (-1.0 + 4.5 * 0.25, 0.5 + 3.5 * 0.25, 2.0 + 2.5 * 0.25))) < 1e-15
    return bool(ok)


def test_unmutated_oracle_passes_the_quick_pins(oracle_mod):
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(oracle_mod, tmp_path, monkeypatch, name):
    old, new = MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    monkeypatch.setattr(oracle, "_lib", lib)
    assert not _pins_pass(), "mutant %s survived the pins" % name
