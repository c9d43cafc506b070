"""Batched Klein ensemble (one persistent kernel over many uneven runs) against the FP64 oracle.

Each run of a batch must evolve exactly as a single grid does: FP64 runs are compared bit for bit
with the oracle (same inputs, the step counts chosen odd so the single-step remainder launches run),
fluxes to 1e-12; FP32 runs within their rounding tolerance."""
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
    oracle.build()
    import paper_1107_4650_gb300 as D
    D.load_library()
    return D


def _runs():
    return [W.KleinRun(side=96, V0=2.5 * C * C, p0=0.6 * C, width=8 * DX, nsteps=37, face=60),
            W.KleinRun(side=64, V0=1.2 * C * C, p0=0.9 * C, width=6 * DX, nsteps=0, face=40),
            W.KleinRun(side=130, V0=3.0 * C * C, p0=0.3 * C, width=10 * DX, nsteps=52, face=90),
            W.KleinRun(side=72, V0=0.7 * C * C, p0=0.5 * C, width=5 * DX, nsteps=21, face=50),
            W.KleinRun(side=160, V0=2.0 * C * C, p0=0.8 * C, width=12 * DX, nsteps=44, face=100)]


def _run_batch(D, runs, fp32, K=2, P=0, seg=0, graphs=True, explicit=True):
    cfg = D.dirac_batch_default_config()
    cfg.precision = D.DIRAC_FP32 if fp32 else D.DIRAC_FP64
    cfg.steps_per_launch = K
    cfg.points_per_lane = P
    cfg.segment_rows = seg
    cfg.use_graphs = 1 if graphs else 0
    h = D.dirac_batch_create([r.as_batch_fields() for r in runs], cfg)
    dt = np.complex64 if fp32 else np.complex128
    try:
        if explicit:
            for i, r in enumerate(runs):
                D.dirac_batch_set_state(h, i, np.ascontiguousarray(r.state().astype(dt)))
                if r.absorb:
                    D.dirac_batch_set_absorber(h, i, r.mask())
                D.dirac_batch_set_potential(h, i, r.potential())
        D.dirac_batch_run(h)
        res = D.dirac_batch_results(h, len(runs))
        outs = []
        for i, r in enumerate(runs):
            o = np.empty((r.side, 1, r.side, 4), dtype=dt)
            D.dirac_batch_get_state(h, i, o)
            outs.append(o)
        info = D.dirac_batch_get_info(h)
    finally:
        D.dirac_batch_destroy(h)
    return outs, res, info


def _oracle(r):
    _, _, _, _, face = r.geometry()
    return oracle.step(r.state(), 2, 1.0, C, r.dx, r.nsteps, V=r.potential(), flux_face=face,
                       absorber=r.mask() if r.absorb else None)


def _absorbing_runs():
    return [W.KleinRun(side=140, V0=2.5 * C * C, p0=0.6 * C, width=8 * DX, nsteps=41, face=80, absorb=20, eta=0.1),
            W.KleinRun(side=96, V0=1.5 * C * C, p0=0.9 * C, width=5 * DX, nsteps=30, face=50, absorb=16, eta=0.2)]


def test_batch_absorbing_layers_bit_exact(D):
    runs = _absorbing_runs()
    outs, res, _ = _run_batch(D, runs, fp32=False)
    for r, got, F in zip(runs, outs, res["flux"]):
        want, Fw = _oracle(r)
        assert np.array_equal(got.view(np.float64), want.view(np.float64))
        assert abs(F - Fw) <= 1e-12 * max(abs(Fw), 1e-300)


def test_batch_device_packets_zero_in_the_layers(D):
    runs = _absorbing_runs()
    _, res, _ = _run_batch(D, runs, fp32=False, explicit=False)
    for r, T in zip(runs, res["T"]):
        want, Fw = _oracle(r)
        assert abs(T - Fw / oracle.observables(r.state(), 2, r.dx)["norm"]) < 1e-9


def test_ensemble_geometry_gives_smooth_transmission(D):
    """Neighbouring step heights at the widest packets give neighbouring transmissions (without the
    absorbing layers, waves reflected at the edges came back across the face and T jumped by 2x)."""
    qs = np.array([[V0, 0.943, 144.0] for V0 in np.linspace(2.70, 2.77, 6)])
    runs = [D.dirac_klein_run_from_reduced(q, DX, C, 1.0) for q in qs]
    cfg = D.dirac_batch_default_config()
    cfg.precision = D.DIRAC_FP32
    cfg.steps_per_launch = 2
    T, _ = D.dirac_batch_klein(runs, cfg)
    d = np.diff(T)
    assert np.all(d > 0) and np.max(np.abs(np.diff(d))) < 0.2 * np.max(np.abs(d)) + 1e-4, T


@pytest.mark.parametrize("K,P,seg", [(2, 2, 0), (1, 4, 32), (2, 2, 24)])
def test_batch_fp64_each_run_bit_exact(D, K, P, seg):
    runs = _runs()
    outs, res, info = _run_batch(D, runs, fp32=False, K=K, P=P, seg=seg)
    assert info["steps_per_launch"] == K
    for r, got, F, n0 in zip(runs, outs, res["flux"], res["norm0"]):
        want, Fw = _oracle(r)
        assert np.array_equal(got.view(np.float64), want.view(np.float64)), (r.side, r.nsteps)
        assert abs(F - Fw) <= 1e-12 * max(abs(Fw), 1e-300)
        assert abs(n0 - oracle.observables(r.state(), 2, r.dx)["norm"]) <= 1e-12


def test_batch_graph_and_direct_agree(D):
    runs = _runs()
    a, ra, _ = _run_batch(D, runs, fp32=False, graphs=True)
    b, rb, _ = _run_batch(D, runs, fp32=False, graphs=False)
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.float64), y.view(np.float64))
    assert np.array_equal(ra["flux"], rb["flux"])


@pytest.mark.parametrize("K,P", [(2, 2), (4, 2), (1, 4)])
def test_batch_fp32_against_oracle(D, K, P):
    runs = _runs()
    outs, res, _ = _run_batch(D, runs, fp32=True, K=K, P=P)
    for r, got, F in zip(runs, outs, res["flux"]):
        want, Fw = _oracle(r)
        if r.nsteps == 0:
            continue
        assert rel_l2(got.astype(np.complex128), want) < 1e-5
        assert abs(F - Fw) < 1e-5 * abs(Fw) + 1e-12


def test_batch_device_packets_match_host_packets(D):
    """The packets the library writes on the device give the transmitted fraction of the numpy packets."""
    runs = _runs()
    _, res_dev, _ = _run_batch(D, runs, fp32=False, explicit=False)
    for r, T in zip(runs, res_dev["T"]):
        if r.nsteps == 0:
            assert T == 0.0
            continue
        want, Fw = _oracle(r)
        n0 = oracle.observables(r.state(), 2, r.dx)["norm"]
        assert abs(T - Fw / n0) < 1e-9


def test_batch_autotune_then_run(D):
    runs = _runs()
    cfg = D.dirac_batch_default_config()
    cfg.precision = D.DIRAC_FP64
    h = D.dirac_batch_create([r.as_batch_fields() for r in runs], cfg)
    try:
        D.dirac_batch_autotune(h)
        D.dirac_batch_run(h)
        T = D.dirac_batch_results(h, len(runs))["T"]
        with pytest.raises(D.DiracError):
            D.dirac_batch_run(h)  # needs a reset first
        D.dirac_batch_reset(h)
        D.dirac_batch_run(h)
        T2 = D.dirac_batch_results(h, len(runs))["T"]
    finally:
        D.dirac_batch_destroy(h)
    assert np.allclose(T, T2, rtol=1e-12, atol=0)
    _, ref, _ = _run_batch(D, runs, fp32=False, explicit=False)
    assert np.allclose(T, ref["T"], rtol=1e-12, atol=1e-15)


def test_batch_one_call(D):
    runs = _runs()
    cfg = D.dirac_batch_default_config()
    cfg.precision = D.DIRAC_FP64
    cfg.steps_per_launch = 2
    T, R = D.dirac_batch_klein([r.as_batch_fields() for r in runs], cfg)
    assert np.allclose(T + R, 1.0)
    _, ref, _ = _run_batch(D, runs, fp32=False, explicit=False)
    assert np.allclose(T, ref["T"], rtol=1e-12, atol=1e-15)


def test_full_512_run_ensemble_sampled_outputs(D):
    """The benchmark's 512-run ensemble (sides, geometry, absorbing layers; FP64 storage, k = 2) with every
    run cut to 40 steps: for 6 runs, 3 sampled cells each recomputed by the oracle on their light-cone crops,
    bit for bit; every run's transmission finite."""
    import dataclasses
    full, _ = W.klein_ensemble(nruns=512)
    runs = [dataclasses.replace(r, nsteps=40) for r in full]
    cfg = D.dirac_batch_default_config()
    cfg.precision = D.DIRAC_FP64
    cfg.steps_per_launch = 2
    h = D.dirac_batch_create([r.as_batch_fields() for r in runs], cfg)
    picks = [0, 77, 150, 311, 480, 511]
    outs = {}
    try:
        for i in picks:  # the sampled runs take the host's packet, layers and potential (the rest their device ones)
            r = runs[i]
            D.dirac_batch_set_state(h, i, r.state())
            D.dirac_batch_set_absorber(h, i, r.mask())
            D.dirac_batch_set_potential(h, i, r.potential())
        D.dirac_batch_run(h)
        res = D.dirac_batch_results(h, len(runs))
        for i in picks:
            r = runs[i]
            o = np.empty((r.side, 1, r.side, 4), dtype=np.complex128)
            D.dirac_batch_get_state(h, i, o)
            outs[i] = o
    finally:
        D.dirac_batch_destroy(h)
    assert np.all(np.isfinite(res["T"]))
    for i in picks:
        r = runs[i]
        psi0 = r.state()
        V = r.potential()
        a = r.mask()
        _, _, _, _, face = r.geometry()
        for (z, x) in [(r.side // 2, face), (r.side // 2, face - 30), (r.side - 1, r.absorb - 1)]:
            sz = slice(max(0, z - 41), min(r.side, z + 42))
            sx = slice(max(0, x - 41), min(r.side, x + 42))
            want, _ = oracle.step(psi0[sz, :, sx], 2, 1.0, C, r.dx, 40, V=V[sx], absorber=a[sx])
            got = outs[i][z, 0, x]
            assert np.array_equal(got.view(np.float64), want[z - sz.start, 0, x - sx.start].view(np.float64)), (i, z, x)


def test_gap_transmission_bounded_below_by_the_initial_tail(D):
    """Runs whose packet energy lies in the gap |E - V0| < m c^2 of the step transmit nothing; their T, the net
    flux through the face over the initial norm, is then the part of the packet that started right of the step
    flowing back: T >= -erfc(4 / sqrt 2) / 2 = -3.2e-5 (the packet starts 4 widths left of the step), FP32 and FP64."""
    q = [(1.2, 0.2, 40.0), (1.5, 0.25, 60.0), (0.9, 0.3, 45.0), (1.8, 0.2, 80.0)]
    runs = [D.dirac_klein_run_from_reduced(x, DX, C, 1.0) for x in q]
    bound = -W.packet_mass_right_of_step()
    for prec in (D.DIRAC_FP32, D.DIRAC_FP64):
        cfg = D.dirac_batch_default_config()
        cfg.precision = prec
        cfg.steps_per_launch = 2
        T, _ = D.dirac_batch_klein(runs, cfg)
        assert np.all(T >= bound * 1.02), (prec, T)
        assert np.all(T < 1e-3), (prec, T)


def test_drawn_sides_ensemble_keeps_its_sides_and_matches_the_oracle(D):
    """The ensemble that keeps its drawn sides (the queue-balance workload): every allowed side occurs, and two of
    its runs (the smallest and a large one, steps cut to 31) evolve in the batch as the oracle's single grid."""
    runs, _ = W.klein_ensemble_drawn_sides(64, seed=W.SEED + 7)
    assert {r.side for r in runs} == set(W.ALLOWED_SIDES)
    small = min(runs, key=lambda r: r.side)
    big = max(runs, key=lambda r: r.side)
    pick = [W.KleinRun(side=r.side, V0=r.V0, p0=r.p0, width=r.width, nsteps=31, face=r.face, absorb=r.absorb,
                       eta=r.eta) for r in (small, big)]
    outs, res, _ = _run_batch(D, pick, fp32=False)
    for i, r in enumerate(pick):
        want, F = _oracle(r)
        assert np.array_equal(outs[i].view(np.float64), want.view(np.float64))
        assert abs(res["flux"][i] - F) <= 1e-12 * max(abs(F), 1e-30) + 1e-18
