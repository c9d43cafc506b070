"""DIRAC_FX64 (64-bit fixed-point storage, 2-D and 3-D first-order steps): the GPU's integer state against the
fixed-point oracle bit for bit, and the decoded state against the FP64 oracle within relative L2 1e-12 after
the Klein workload's 4000 steps (the tolerance the FP64 path is held to) and after 3-D Coulomb steps."""
import numpy as np
import pytest

import oracle
from paper_1107_4650_gb300 import workloads as W
from tests.dirac_algebra import rel_l2

pytestmark = pytest.mark.gpu

C = W.C_AU
DX = W.DX_DEFAULT


@pytest.fixture(scope="module")
def D():
    from paper_1107_4650_gb300 import build as B
    B.build()
    import paper_1107_4650_gb300 as D
    D.load_library()
    return D


def _grid(D, nx, nz, periodic=False, K=0, P=0, flux_face=-1, graphs=True, x_min=None):
    cfg = D.make_config((nx, 1, nz), precision=D.DIRAC_FX64, flux_face=flux_face, steps_per_launch=K,
                        points_per_lane=P, use_graphs=graphs, x_min=x_min,
                        boundary=D.DIRAC_BC_PERIODIC if periodic else D.DIRAC_BC_ZERO)
    return D.dirac_create_grid(cfg)


def _q_of(D, h, shape):
    q = np.empty(shape + (4, 2), dtype=np.int64)
    S = D.dirac_get_state_fx(h, q)
    return q, S


@pytest.mark.parametrize("shape", [(70, 45), (130, 33), (5, 7), (64, 64), (1, 9)])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("K,P", [(1, 1), (1, 2), (1, 4), (2, 2)])
@pytest.mark.parametrize("full", [False, True])
def test_fx_bit_exact_against_fixed_point_oracle(D, shape, periodic, K, P, full):
    nx, nz = shape
    psi = W.random_state(nz, 1, nx, seed=nx * nz + K)
    V = np.random.default_rng(nx + nz).uniform(-4e4, 4e4, nx * nz if full else nx)
    S = oracle.fx_shift(psi)
    q0 = oracle.fx_encode(psi, S)
    want = oracle.step_fx(q0, 1.0, C, DX, 5, V=V, periodic=periodic)
    h = _grid(D, nx, nz, periodic, K, P)
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_FULL if full else D.DIRAC_V_X_ONLY)
        D.dirac_set_state_fx(h, q0, S)
        D.dirac_step(h, 5)
        got, S1 = _q_of(D, h, (nz, 1, nx))
        info = D.dirac_get_info(h)
    finally:
        D.dirac_destroy(h)
    assert S1 == S and info["fx_shift"] == S
    assert info["steps_per_launch"] == K and info["points_per_lane"] == P
    assert np.array_equal(got, want)


def test_fx_set_state_encodes_with_the_norm_shift(D):
    """dirac_set_state picks S from the discrete norm and rounds to nearest even, as the oracle's encoder;
    dirac_get_state decodes exactly what the oracle's decoder gives."""
    psi = W.random_state(40, 1, 50, seed=3) * 7.5
    h = _grid(D, 50, 40)
    try:
        D.dirac_set_state(h, psi)
        q, S = _q_of(D, h, (40, 1, 50))
        back = np.empty_like(psi)
        D.dirac_get_state(h, back)
    finally:
        D.dirac_destroy(h)
    assert S == oracle.fx_shift(psi)
    assert np.array_equal(q, oracle.fx_encode(psi, S))
    assert np.array_equal(back.view(np.float64), oracle.fx_decode(q, S).view(np.float64))


def test_fx_klein_4000_steps_within_1e12_of_fp64_oracle(D):
    """The Klein step at 512^2 for the workload's 4000 steps (tanh step, packet width 25 dx, face flux): the
    decoded state within relative L2 1e-12 of the FP64 oracle, the flux and the norms within 1e-12 relative,
    and the integer state equal to the fixed-point oracle's."""
    base = W.klein_config_2d(side=512, nsteps=4000)
    run = W.KleinRun(side=512, V0=base.V0, p0=base.p0, width=25 * DX, nsteps=4000)
    psi0 = run.state()
    V = run.potential()
    x_min, z_min, _, _, face = run.geometry()
    want, F = oracle.step(psi0, 2, 1.0, C, DX, run.nsteps, V=V, flux_face=face)
    h = _grid(D, 512, 512, flux_face=face, x_min=(x_min, 0.0, z_min))
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY)
        D.dirac_set_state(h, psi0)
        q0, S = _q_of(D, h, (512, 1, 512))
        D.dirac_step(h, run.nsteps)
        got = np.empty_like(psi0)
        D.dirac_get_state(h, got)
        q1, _ = _q_of(D, h, (512, 1, 512))
        obs = D.dirac_observables(h)
    finally:
        D.dirac_destroy(h)
    err = rel_l2(got, want)
    print("FX64 vs FP64 oracle after 4000 steps: rel L2 %.3e" % err)
    assert err <= 1e-12
    assert abs(obs["flux_cum"] - F) <= 1e-12 * abs(F)
    o = oracle.observables(want, 2, DX, (x_min, 0.0, z_min), face)
    assert abs(obs["norm"] - o["norm"]) <= 1e-12 * o["norm"]
    assert abs(obs["norm_right"] - o["norm_right"]) <= 1e-12 * o["norm"]
    assert np.array_equal(q1, oracle.step_fx(q0, 1.0, C, DX, run.nsteps, V=V))


@pytest.mark.parametrize("graphs", [True, False])
def test_fx_absorber_flux_and_graphs(D, graphs):
    """Absorbing layers (factors in the phase coefficients) and the face flux over 70 steps (graph replay and
    the remainder): integer state bit-exact with the fixed-point oracle, flux within 1e-12 of the FP64 one."""
    run = W.KleinRun(side=192, V0=2.5 * C * C, p0=0.6 * C, width=10 * DX, nsteps=70, face=120, absorb=24, eta=0.1)
    psi0 = run.state()
    V = run.potential()
    mask = run.mask()
    x_min, z_min, _, _, face = run.geometry()
    _, F = oracle.step(psi0, 2, 1.0, C, DX, run.nsteps, V=V, flux_face=face, absorber=mask)
    h = _grid(D, 192, 192, flux_face=face, graphs=graphs, x_min=(x_min, 0.0, z_min))
    try:
        D.dirac_set_absorber(h, mask)
        D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY)
        D.dirac_set_state(h, psi0)
        q0, S = _q_of(D, h, (192, 1, 192))
        D.dirac_step(h, run.nsteps)
        q1, _ = _q_of(D, h, (192, 1, 192))
        obs = D.dirac_observables(h)
    finally:
        D.dirac_destroy(h)
    assert np.array_equal(q1, oracle.step_fx(q0, 1.0, C, DX, run.nsteps, V=V, absorber=mask))
    assert abs(obs["flux_cum"] - F) <= 1e-12 * abs(F)


def test_fx_autotune_restores_state(D):
    nx, nz = 300, 260
    psi = W.random_state(nz, 1, nx, seed=17)
    V = np.random.default_rng(18).uniform(-4e4, 4e4, nx)
    S = oracle.fx_shift(psi)
    q0 = oracle.fx_encode(psi, S)
    want = oracle.step_fx(q0, 1.0, C, DX, 9, V=V)
    h = _grid(D, nx, nz)
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY)
        D.dirac_set_state_fx(h, q0, S)
        D.dirac_autotune(h)
        D.dirac_step(h, 9)
        got, _ = _q_of(D, h, (nz, 1, nx))
    finally:
        D.dirac_destroy(h)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape", [(24, 20, 18), (7, 5, 6), (41, 9, 13), (33, 1, 4), (70, 30, 37)])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("P", [0, 1, 2, 4])
@pytest.mark.parametrize("full", [False, True])
def test_fx_3d_bit_exact_against_fixed_point_oracle(D, shape, periodic, P, full):
    """3-D on the int64 state, against oracle_step_fx bit for bit: the fused single pass (points_per_lane 0:
    30-cell strips, 14-row tiles, several z segments at 70 x 30 x 37) and the x-y pass + z/phase pass."""
    nx, ny, nz = shape
    psi = W.random_state(nz, ny, nx, seed=nx + ny * nz + P)
    V = np.random.default_rng(nz + P).uniform(-4e4, 4e4, nx * ny * nz if full else nx)
    S = oracle.fx_shift(psi, 3)
    q0 = oracle.fx_encode(psi, S)
    want = oracle.step_fx(q0, 1.0, C, DX, 4, V=V, periodic=periodic, ndim=3)
    cfg = D.make_config((nx, ny, nz), ndim=3, precision=D.DIRAC_FX64, points_per_lane=P,
                        boundary=D.DIRAC_BC_PERIODIC if periodic else D.DIRAC_BC_ZERO)
    h = D.dirac_create_grid(cfg)
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_FULL if full else D.DIRAC_V_X_ONLY)
        D.dirac_set_state_fx(h, q0, S)
        D.dirac_step(h, 4)
        got, _ = _q_of(D, h, (nz, ny, nx))
        info = D.dirac_get_info(h)
    finally:
        D.dirac_destroy(h)
    if P == 0:
        assert info["plan"] == D.DIRAC_PLAN_3D_FUSED
    else:
        assert info["plan"] == D.DIRAC_PLAN_3D_TWO_PASS and info["points_per_lane"] == P
    assert np.array_equal(got, want)


@pytest.mark.parametrize("tune", [True, False])
def test_fx_3d_coulomb_within_1e12_of_fp64_oracle(D, tune):
    """A moving packet in the soft-Coulomb potential (64^3, per-cell potential, face flux, 150 steps; autotuned,
    and the default fused pass): the decoded state within relative L2 1e-12 of the FP64 oracle, the flux
    within 1e-12 relative, the integer state equal to the fixed-point oracle's; dirac_set_state chooses the
    3-D shift."""
    n = 64
    psi = W.gaussian_packet(n, n, DX, -n * DX / 2, -n * DX / 2, -6 * DX, 0.0, 5 * DX, 0.4 * C, ny=n, y_min=-n * DX / 2)
    V = W.soft_coulomb_3d(n, DX, 10.0, 2 * DX).reshape(-1)
    want, F = oracle.step(psi, 3, 1.0, C, DX, 150, V=V, flux_face=n // 2)
    cfg = D.make_config((n, n, n), ndim=3, precision=D.DIRAC_FX64, flux_face=n // 2)
    h = D.dirac_create_grid(cfg)
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_FULL)
        D.dirac_set_state(h, psi)
        q0, S = _q_of(D, h, (n, n, n))
        if tune:
            D.dirac_autotune(h)
        else:
            assert D.dirac_get_info(h)["plan"] == D.DIRAC_PLAN_3D_FUSED
        D.dirac_step(h, 150)
        got = np.empty_like(psi)
        D.dirac_get_state(h, got)
        q1, _ = _q_of(D, h, (n, n, n))
        obs = D.dirac_observables(h)
    finally:
        D.dirac_destroy(h)
    assert S == oracle.fx_shift(psi, 3)
    err = rel_l2(got, want)
    print("FX64 3-D vs FP64 oracle after 150 steps: rel L2 %.3e" % err)
    assert err <= 1e-12
    assert F > 1e-3 and abs(obs["flux_cum"] - F) <= 1e-12 * abs(F)
    assert np.array_equal(q1, oracle.step_fx(q0, 1.0, C, DX, 150, V=V, ndim=3))


@pytest.mark.parametrize("shape", [(70, 45), (130, 33), (5, 7), (1, 9)])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("P", [1, 2])
def test_fx_strang2d_bit_exact_against_fixed_point_oracle(D, shape, periodic, P):
    """Second-order 2-D steps (x, z, phase, z, x as two pipelined levels) on the int64 state, bit for bit."""
    nx, nz = shape
    psi = W.random_state(nz, 1, nx, seed=nx * nz + P + 7)
    V = np.random.default_rng(nx + P).uniform(-4e4, 4e4, nx)
    S = oracle.fx_shift(psi)
    q0 = oracle.fx_encode(psi, S)
    want = oracle.step_strang2d_fx(q0, 1.0, C, DX, 5, V=V, periodic=periodic)
    cfg = D.make_config((nx, 1, nz), precision=D.DIRAC_FX64, splitting=D.DIRAC_STRANG, points_per_lane=P,
                        boundary=D.DIRAC_BC_PERIODIC if periodic else D.DIRAC_BC_ZERO)
    h = D.dirac_create_grid(cfg)
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY)
        D.dirac_set_state_fx(h, q0, S)
        D.dirac_step(h, 5)
        got, _ = _q_of(D, h, (nz, 1, nx))
        info = D.dirac_get_info(h)
    finally:
        D.dirac_destroy(h)
    assert info["plan"] == D.DIRAC_PLAN_STRANG_2D and info["points_per_lane"] == P
    assert np.array_equal(got, want)


def test_fx_strang2d_klein_within_1e12_of_fp64_oracle(D):
    """The second-order Klein step at 384^2 for 1500 steps with the face flux (graphs, autotuned): decoded state
    within relative L2 1e-12 of the FP64 Strang oracle, flux within 1e-12 relative, integer state equal to
    the fixed-point oracle's."""
    run = W.KleinRun(side=384, V0=2.5 * C * C, p0=0.6 * C, width=20 * DX, nsteps=1500, face=240)
    psi0 = run.state()
    V = run.potential()
    x_min, z_min, _, _, face = run.geometry()
    want, F = oracle.step_strang2d(psi0, 1.0, C, DX, run.nsteps, V=V, flux_face=face)
    cfg = D.make_config((384, 1, 384), precision=D.DIRAC_FX64, splitting=D.DIRAC_STRANG, flux_face=face,
                        x_min=(x_min, 0.0, z_min))
    h = D.dirac_create_grid(cfg)
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY)
        D.dirac_set_state(h, psi0)
        q0, S = _q_of(D, h, (384, 1, 384))
        D.dirac_autotune(h)
        D.dirac_step(h, run.nsteps)
        got = np.empty_like(psi0)
        D.dirac_get_state(h, got)
        q1, _ = _q_of(D, h, (384, 1, 384))
        obs = D.dirac_observables(h)
    finally:
        D.dirac_destroy(h)
    err = rel_l2(got, want)
    print("FX64 Strang vs FP64 oracle after 1500 steps: rel L2 %.3e" % err)
    assert err <= 1e-12
    assert F > 0.01 and abs(obs["flux_cum"] - F) <= 1e-12 * abs(F)
    assert np.array_equal(q1, oracle.step_strang2d_fx(q0, 1.0, C, DX, run.nsteps, V=V))


@pytest.mark.parametrize("shape", [(24, 20, 18), (7, 5, 6), (41, 9, 13), (60, 30, 40), (29, 13, 3)])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("pp,nsteps", [(1, 3), (2, 3), (2, 1), (2, 34), (4, 3), (4, 34)])
def test_fx_strang3d_bit_exact_against_fixed_point_oracle(D, shape, periodic, full, pp, nsteps):
    """3-D second-order steps on the int64 state, as eight single sweeps (points_per_lane 1), as single x and y
    sweeps with one z-phase-z pass (4) or as the fused x-y-x / z-phase-z / x-y-x-x-y-x passes (2; 34 steps: a
    captured 32-step run and a 2-step run), against oracle_step_strang3d_fx bit for bit."""
    nx, ny, nz = shape
    psi = W.random_state(nz, ny, nx, seed=nx * 3 + ny + nz)
    V = np.random.default_rng(ny + nz).uniform(-4e4, 4e4, nx * ny * nz if full else nx)
    S = oracle.fx_shift(psi, 3, strang=True)
    q0 = oracle.fx_encode(psi, S)
    want = oracle.step_strang3d_fx(q0, 1.0, C, DX, nsteps, V=V, periodic=periodic)
    cfg = D.make_config((nx, ny, nz), ndim=3, precision=D.DIRAC_FX64, splitting=D.DIRAC_STRANG, points_per_lane=pp,
                        boundary=D.DIRAC_BC_PERIODIC if periodic else D.DIRAC_BC_ZERO)
    h = D.dirac_create_grid(cfg)
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_FULL if full else D.DIRAC_V_X_ONLY)
        D.dirac_set_state_fx(h, q0, S)
        D.dirac_step(h, nsteps)
        got, _ = _q_of(D, h, (nz, ny, nx))
        info = D.dirac_get_info(h)
    finally:
        D.dirac_destroy(h)
    assert info["plan"] == {1: D.DIRAC_PLAN_3D_STRANG, 2: D.DIRAC_PLAN_3D_STRANG_FUSED,
                            4: D.DIRAC_PLAN_3D_STRANG_ZPASS}[pp]
    assert np.array_equal(got, want)


@pytest.mark.parametrize("pp", [1, 2])
def test_fx_strang3d_coulomb_within_1e12_of_fp64_oracle(D, pp):
    """3-D second-order steps in the soft-Coulomb potential (48^3, face flux, 40 steps, autotuned, graphs): the
    decoded state within relative L2 1e-12 of the FP64 oracle, flux within 1e-12 relative, integer state equal
    to the fixed-point oracle's; dirac_set_state picks the second-order shift."""
    n = 48
    psi = W.gaussian_packet(n, n, DX, -n * DX / 2, -n * DX / 2, -6 * DX, 0.0, 4 * DX, 0.4 * C, ny=n, y_min=-n * DX / 2)
    V = W.soft_coulomb_3d(n, DX, 10.0, 2 * DX).reshape(-1)
    want, F = oracle.step_strang3d(psi, 1.0, C, DX, 40, V=V, flux_face=n // 2)
    cfg = D.make_config((n, n, n), ndim=3, precision=D.DIRAC_FX64, splitting=D.DIRAC_STRANG, flux_face=n // 2,
                        points_per_lane=pp)
    h = D.dirac_create_grid(cfg)
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_FULL)
        D.dirac_set_state(h, psi)
        q0, S = _q_of(D, h, (n, n, n))
        D.dirac_autotune(h)
        D.dirac_step(h, 40)
        got = np.empty_like(psi)
        D.dirac_get_state(h, got)
        q1, _ = _q_of(D, h, (n, n, n))
        obs = D.dirac_observables(h)
    finally:
        D.dirac_destroy(h)
    assert S == oracle.fx_shift(psi, 3, strang=True)
    err = rel_l2(got, want)
    print("FX64 3-D Strang vs FP64 oracle after 40 steps: rel L2 %.3e" % err)
    assert err <= 1e-12
    assert F > 1e-3 and abs(obs["flux_cum"] - F) <= 1e-12 * abs(F)
    assert np.array_equal(q1, oracle.step_strang3d_fx(q0, 1.0, C, DX, 40, V=V))
