"""Full-length parity at the workloads' full sizes: the whole state, not sampled cells.

* The 2048^2 FP64 Klein grid (V0 = 2.5 m c^2, L = 4 dx, packet width 100 dx) after its full 4000 steps, in the
  benchmark's launch plan (autotuned, graph replay), against the CPU oracle run for the same 4000 steps: every
  word of the state bit for bit, and the face flux within 1e-12.  The 64-bit fixed-point path on the same
  workload is held to the scope's FP64 gate: relative L2 <= 1e-12 from the oracle's state.
* The 384^3 soft-Coulomb grid (Z = 10, per-cell FP64 table) after 100 first-order steps in the benchmark's
  plan, against the oracle (about 1 s of oracle time per step on 16 cores bounds the step count): FP64 bit for
  bit, fixed point within 1e-12, FP32 storage within 1e-4 (its error is reported, not gated, by the benchmark).

The oracle runs take a few minutes on the host's cores; each state is computed once per module.
"""
import numpy as np
import pytest

import oracle
from paper_1107_4650_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

C = W.C_AU
DX = W.DX_DEFAULT


@pytest.fixture(scope="module")
def D():
    from paper_1107_4650_gb300 import build as B
    B.build()
    import paper_1107_4650_gb300 as D
    D.load_library()
    return D


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module")
def klein2048():
    run = W.klein_config_2d(side=2048, nsteps=4000)
    psi0 = run.state()
    V = run.potential()
    face = run.geometry()[4]
    want, F = oracle.step(psi0, 2, 1.0, C, DX, run.nsteps, V=V, flux_face=face)
    return run, psi0, V, want, F


def _gpu_klein(D, run, psi0, V, precision):
    x_min, z_min, _, _, face = run.geometry()
    cfg = D.make_config((2048, 1, 2048), x_min=(x_min, 0.0, z_min), flux_face=face, precision=precision)
    h = D.dirac_create_grid(cfg)
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY)
        D.dirac_set_state(h, psi0)
        D.dirac_autotune(h)
        D.dirac_step(h, run.nsteps)
        got = np.empty_like(psi0)
        D.dirac_get_state(h, got)
        obs = D.dirac_observables(h)
        info = D.dirac_get_info(h)
    finally:
        D.dirac_destroy(h)
    return got, obs, info


def test_klein_2048_fp64_full_state_after_4000_steps_bit_exact(D, klein2048):
    run, psi0, V, want, F = klein2048
    got, obs, info = _gpu_klein(D, run, psi0, V, D.DIRAC_FP64)
    assert info["graphs"] == 1
    assert np.array_equal(got.view(np.float64), want.view(np.float64))
    assert abs(obs["flux_cum"] - F) <= 1e-12 * abs(F)
    assert F > 1e-3


def test_klein_2048_fx64_full_state_after_4000_steps_within_1e12(D, klein2048):
    run, psi0, V, want, F = klein2048
    got, obs, _ = _gpu_klein(D, run, psi0, V, D.DIRAC_FX64)
    assert rel_l2(got, want) <= 1e-12
    assert abs(obs["flux_cum"] - F) <= 1e-12 * abs(F)


@pytest.fixture(scope="module")
def coulomb384():
    n3, nsteps = 384, 100
    psi0 = W.gaussian_packet(n3, n3, DX, -n3 * DX / 2, -n3 * DX / 2, 32 * DX, 0.0, 16 * DX, 0.0, ny=n3,
                             y_min=-n3 * DX / 2)
    V = W.soft_coulomb_3d(n3, DX, 10.0, 2 * DX).reshape(-1)
    want, _ = oracle.step(psi0, 3, 1.0, C, DX, nsteps, V=V)
    return n3, nsteps, psi0, V, want


def _gpu_coulomb(D, n3, nsteps, psi0, V, precision):
    cfg = D.make_config((n3, n3, n3), ndim=3, precision=precision)
    h = D.dirac_create_grid(cfg)
    st = psi0.astype(np.complex64) if precision == D.DIRAC_FP32 else psi0
    try:
        D.dirac_set_potential(h, V, D.DIRAC_V_FULL)
        D.dirac_set_state(h, st)
        D.dirac_autotune(h)
        D.dirac_step(h, nsteps)
        got = np.empty_like(st)
        D.dirac_get_state(h, got)
    finally:
        D.dirac_destroy(h)
    return got


def test_coulomb_384_fp64_full_state_after_100_steps_bit_exact(D, coulomb384):
    n3, nsteps, psi0, V, want = coulomb384
    got = _gpu_coulomb(D, n3, nsteps, psi0, V, D.DIRAC_FP64)
    assert np.array_equal(got.view(np.float64), want.view(np.float64))


def test_coulomb_384_fx64_and_fp32_full_state_after_100_steps(D, coulomb384):
    n3, nsteps, psi0, V, want = coulomb384
    assert rel_l2(_gpu_coulomb(D, n3, nsteps, psi0, V, D.DIRAC_FX64), want) <= 1e-12
    got32 = _gpu_coulomb(D, n3, nsteps, psi0, V, D.DIRAC_FP32)
    assert rel_l2(got32.astype(np.complex128), want) <= 1e-4
