"""Characteristic shift K > 1 (Sec. 2.3: c dt = K dx, each sweep an exact K-cell translation of the
characteristics) beyond the 2-D first-order step: 3-D first-order steps, 2-D second-order steps (Sec. 2.4,
dt = 2 K dx / c) and 3-D second-order steps (dt = 4 K dx / c, x sweeps moving K cells, y and z 2 K), run as
single-sweep launches, against the oracle: FP64 bit for bit (state, both boundaries, x-only and per-cell
tables, graph replay), the face flux within 1e-12, FP32 within its rounding, and with a vector potential."""
import numpy as np
import pytest

import oracle
from paper_1107_4650_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C = W.C_AU
DX = W.DX_DEFAULT


@pytest.fixture(scope="module")
def D():
    from paper_1107_4650_gb300 import build as B
    B.build()
    oracle.build()
    import paper_1107_4650_gb300 as D
    D.load_library()
    return D


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def _bits_equal(a, b):
    return np.array_equal(a.view(np.float64), b.view(np.float64))


def _run(D, psi, ndim, nsteps, K, strang, V=None, periodic=False, fp32=False, flux_face=-1, graphs=True, x_min=None,
         A_tilde=None):
    nz, ny, nx, _ = psi.shape
    cfg = D.make_config((nx, ny, nz), ndim=ndim, precision=D.DIRAC_FP32 if fp32 else D.DIRAC_FP64,
                        boundary=D.DIRAC_BC_PERIODIC if periodic else D.DIRAC_BC_ZERO, flux_face=flux_face,
                        use_graphs=graphs, x_min=x_min, char_shift=K,
                        splitting=D.DIRAC_STRANG if strang else D.DIRAC_LIE)
    h = D.dirac_create_grid(cfg)
    try:
        if A_tilde is not None:
            D.dirac_set_vector_potential(h, A_tilde)
        if V is not None:
            D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY if V.size == nx else D.DIRAC_V_FULL)
        dt = np.complex64 if fp32 else np.complex128
        D.dirac_set_state(h, np.ascontiguousarray(psi.astype(dt)))
        D.dirac_step(h, nsteps)
        out = np.empty(psi.shape, dtype=dt)
        D.dirac_get_state(h, out)
        obs = D.dirac_observables(h)
        info = D.dirac_get_info(h)
    finally:
        D.dirac_destroy(h)
    return out, obs, info


def _oracle(psi, ndim, nsteps, K, strang, **kw):
    if strang:
        f = oracle.step_strang3d if ndim == 3 else oracle.step_strang2d
        return f(psi, 1.0, C, DX, nsteps, shift=K, **kw)
    return oracle.step(psi, ndim, 1.0, C, DX, nsteps, shift=K, **kw)


CASES = [(3, False), (2, True), (3, True)]  # (ndim, second order)


@pytest.mark.parametrize("ndim,strang", CASES)
@pytest.mark.parametrize("K", [2, 3, 4])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("full", [False, True])
def test_shift_sweeps_fp64_bit_exact(D, ndim, strang, K, periodic, full):
    shape = (37, 11, 23) if ndim == 3 else (53, 1, 41)
    nx, ny, nz = shape
    psi = W.random_state(nz, ny, nx, seed=100 * K + 10 * ndim + strang)
    rng = np.random.default_rng(K + 7)
    V = rng.uniform(-2e4, 6e4, nx * ny * nz if full else nx)
    want, _ = _oracle(psi, ndim, 5, K, strang, V=V, periodic=periodic)
    got, _, info = _run(D, psi, ndim, 5, K, strang, V=V, periodic=periodic)
    assert info["plan"] == (D.DIRAC_PLAN_3D_STRANG if (ndim == 3 and strang) else D.DIRAC_PLAN_SHIFT_SWEEPS)
    assert _bits_equal(got, want), rel_l2(got, want)


@pytest.mark.parametrize("ndim,strang", CASES)
@pytest.mark.parametrize("K", [2, 4])
def test_shift_sweeps_flux_and_graph_replay(D, ndim, strang, K):
    """A Klein packet crossing the face over 40 steps (graph replay past 32 steps, and direct launches): the
    state bit for bit, the K-cell face flux within 1e-12 of the oracle's, and the same flux either way."""
    if ndim == 2:
        run = W.KleinRun(side=192, V0=2.5 * C * C, p0=0.7 * C, width=8 * DX, nsteps=40, face=110)
        psi0, V = run.state(), run.potential()
        x_min, z_min, _, _, face = run.geometry()
        xm = (x_min, 0.0, z_min)
    else:
        n = 48
        psi0 = W.gaussian_packet(n, n, DX, -n * DX / 2, -n * DX / 2, -6 * DX, 0.0, 4 * DX, 0.6 * C, ny=20,
                                 y_min=-10 * DX)
        V = W.tanh_step(n, DX, -n * DX / 2, 0.0, 2.5 * C * C, 2 * DX)
        face, xm = n // 2, (-n * DX / 2, -10 * DX, -n * DX / 2)
    want, F = _oracle(psi0, ndim, 40, K, strang, V=V, flux_face=face)
    got, obs, _ = _run(D, psi0, ndim, 40, K, strang, V=V, flux_face=face, x_min=xm)
    direct, obs2, _ = _run(D, psi0, ndim, 40, K, strang, V=V, flux_face=face, x_min=xm, graphs=False)
    assert _bits_equal(got, want) and _bits_equal(direct, want)
    assert abs(F) > 1e-4
    assert abs(obs["flux_cum"] - F) <= 1e-12 * abs(F) and obs2["flux_cum"] == obs["flux_cum"]


@pytest.mark.parametrize("ndim,strang", CASES)
def test_shift_sweeps_fp32(D, ndim, strang):
    shape = (40, 16, 30) if ndim == 3 else (96, 1, 64)
    nx, ny, nz = shape
    psi = W.random_state(nz, ny, nx, seed=77)
    V = np.random.default_rng(78).uniform(-1e4, 1e4, nx)
    want, _ = _oracle(psi, ndim, 30, 3, strang, V=V, periodic=True)
    got, _, _ = _run(D, psi, ndim, 30, 3, strang, V=V, periodic=True, fp32=True)
    assert rel_l2(got.astype(np.complex128), want) < 2e-5


@pytest.mark.parametrize("ndim,strang", CASES)
def test_shift_sweeps_with_vector_potential(D, ndim, strang):
    """A uniform vector potential (the full phase matrix of Eq. sol_dis_4 over the step's dt) with K = 2."""
    shape = (21, 9, 14) if ndim == 3 else (33, 1, 27)
    nx, ny, nz = shape
    psi = W.random_state(nz, ny, nx, seed=81)
    V = np.random.default_rng(82).uniform(-2e4, 2e4, nx)
    At = np.random.default_rng(83).uniform(-1.2, 1.2, (6, 3))
    want, _ = _oracle(psi, ndim, 6, 2, strang, V=V, A_tilde=At)
    got, _, _ = _run(D, psi, ndim, 6, 2, strang, V=V, A_tilde=At)
    assert _bits_equal(got, want), rel_l2(got, want)


@pytest.mark.parametrize("ndim,strang", CASES)
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 2), (2, 5, 3), (5, 1, 4)])
@pytest.mark.parametrize("periodic", [False, True])
def test_shift_sweeps_degenerate_grids(D, ndim, strang, shape, periodic):
    """Grids smaller than the shift K = 4 (periodic: the characteristics wrap more than once; zero boundary:
    everything leaves), one-cell grids, and 2-D shapes: bit-exact with the oracle."""
    nx, ny, nz = shape
    if ndim == 2:
        ny = 1
    psi = W.random_state(nz, ny, nx, seed=nx * 7 + ny * 3 + nz)
    V = np.random.default_rng(nx + nz).uniform(-2e4, 2e4, nx)
    want, _ = _oracle(psi, ndim, 3, 4, strang, V=V, periodic=periodic)
    got, _, _ = _run(D, psi, ndim, 3, 4, strang, V=V, periodic=periodic)
    assert _bits_equal(got, want)


@pytest.mark.parametrize("ndim,strang", [(2, False)] + CASES)
@pytest.mark.parametrize("periodic,where", [(True, "K"), (True, "nx-K"), (False, "1"), (False, "nx-1")])
def test_shift_flux_face_near_the_edges(D, ndim, strang, periodic, where):
    """The face flux with K = 3 and the face at the edges allowed: periodic grids take faces in [K, nx-K] (the
    window of K cells each side inside the grid); zero-boundary grids any face, the cells outside being zero.
    The flux of a random state is a difference of terms of the order of its probability P = dx^d sum |psi|^2
    (periodic: about 1e-3 P after cancellation), so it is held to 1e-12 P per step."""
    K = 3
    shape = (19, 5, 11) if ndim == 3 else (23, 1, 17)
    nx, ny, nz = shape
    face = {"K": K, "nx-K": nx - K, "1": 1, "nx-1": nx - 1}[where]
    psi = W.random_state(nz, ny, nx, seed=7 * face + ndim)
    V = np.random.default_rng(face).uniform(-2e4, 2e4, nx)
    want, F = _oracle(psi, ndim, 4, K, strang, V=V, periodic=periodic, flux_face=face)
    got, obs, _ = _run(D, psi, ndim, 4, K, strang, V=V, periodic=periodic, flux_face=face)
    assert _bits_equal(got, want)
    P = float(np.sum(np.abs(psi) ** 2)) * DX ** ndim
    assert abs(F) > 1e-6 * P and abs(obs["flux_cum"] - F) <= 4e-12 * P
