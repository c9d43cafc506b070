"""Transmission surrogate: the GPU network's forward and backward against the CPU FP64 oracle, training,
and a small-box Klein surrogate trained on batched-solver output and checked against the FP64 solver."""
import time

import numpy as np
import pytest

from oracle import mlp as M
from paper_1107_4650_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C = W.C_AU
DX = W.DX_DEFAULT
LO = np.array([0.5, 0.2, 10.0])
HI = np.array([3.0, 1.0, 30.0])


@pytest.fixture(scope="module")
def D():
    from paper_1107_4650_gb300 import build as B
    B.build()
    import paper_1107_4650_gb300 as D
    D.load_library()
    return D


def _norm(q):
    return (2.0 * (q - LO) / (HI - LO) - 1.0).astype(np.float32).astype(np.float64)


def _blocks(v):
    out, o = {}, 0
    for name, shape in M.SHAPES:
        n = int(np.prod(shape))
        out[name] = v[o:o + n]
        o += n
    return out


@pytest.mark.parametrize("B", [64, 300])
def test_gradient_matches_oracle(D, B):
    rng = np.random.default_rng(B)
    h = D.dirac_surrogate_create(LO, HI, seed=7, max_batch=512)
    try:
        q = LO + (HI - LO) * rng.uniform(0, 1, (B, 3))
        t = rng.uniform(0, 1, B)
        loss, g = D.dirac_surrogate_gradient(h, q, t)
        p = D.dirac_surrogate_get_params(h).astype(np.float64)
        y = D.dirac_surrogate_predict(h, q)
    finally:
        D.dirac_surrogate_destroy(h)
    lo_, go = M.loss_and_grad(p, _norm(q), t, round_bf16=True)
    assert abs(loss - lo_) <= 1e-5 * lo_
    assert np.max(np.abs(y - M.predict(p, _norm(q)))) < 2e-4
    gb, ob = _blocks(g.astype(np.float64)), _blocks(go)
    for name in gb:
        err = np.linalg.norm(gb[name] - ob[name]) / max(np.linalg.norm(ob[name]), 1e-30)
        assert err < 2e-2, (name, err)
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-2


@pytest.mark.parametrize("n,max_batch", [(1, 512), (129, 512), (300, 128), (4096 + 257, 4096)])
def test_fused_inference_matches_training_forward_and_oracle(D, n, max_batch):
    """dirac_surrogate_predict runs the whole network in one launch per 128 queries (tcgen05 layers, TMA-staged
    packed weights), the training step through per-layer GEMM launches; both keep the same rounding points.
    Checked on a partial last tile, several tiles and calls split into max_batch chunks: (1) the training
    forward's loss, the sequential double sum of its per-sample FP32 squared errors, equals the one formed
    from the predictions, bit for bit; (2) against the CPU oracle's forward pass, the mean difference stays
    below 2e-5 and single queries differ by up to a few 1e-4 where a hidden activation lies at a BF16 rounding
    boundary and the tensor core's FP32 sum and the oracle's round it apart; (3) two calls give the same bits."""
    rng = np.random.default_rng(n)
    h = D.dirac_surrogate_create(LO, HI, seed=11, max_batch=max_batch)
    try:
        p = rng.normal(0.0, 0.08, D.dirac_surrogate_get_params(h).size)
        D.dirac_surrogate_set_params(h, p)
        q = LO + (HI - LO) * rng.uniform(0, 1, (n, 3))
        t = rng.uniform(0, 1, n)
        y1 = D.dirac_surrogate_predict(h, q)
        y2 = D.dirac_surrogate_predict(h, q)
        p32 = D.dirac_surrogate_get_params(h).astype(np.float64)
        if n <= max_batch:
            loss, _ = D.dirac_surrogate_gradient(h, q, t)
            dd = (y1.astype(np.float32) - t.astype(np.float32)).astype(np.float32)
            sq = (dd * dd).astype(np.float32)
            acc = 0.0
            for v in sq:
                acc += float(v)
            assert loss == acc / n
    finally:
        D.dirac_surrogate_destroy(h)
    want = M.predict(p32, _norm(q))
    d = np.abs(y1 - want)
    assert np.array_equal(y1, y2)
    assert d.max() < 1e-3 and d.mean() < 2e-5, (d.max(), d.mean())


def test_inference_follows_every_change_of_the_weights(D):
    """The inference kernel reads packed copies of W2-W4: after dirac_surrogate_set_params and after training,
    predictions equal those of a fresh handle holding the same parameters."""
    rng = np.random.default_rng(5)
    q = LO + (HI - LO) * rng.uniform(0, 1, (200, 3))
    t = rng.uniform(0.1, 0.9, 200)

    def fresh(params):
        h2 = D.dirac_surrogate_create(LO, HI, seed=1, max_batch=256)
        try:
            D.dirac_surrogate_set_params(h2, params)
            return D.dirac_surrogate_predict(h2, q)
        finally:
            D.dirac_surrogate_destroy(h2)

    h = D.dirac_surrogate_create(LO, HI, seed=3, max_batch=256)
    try:
        y0 = D.dirac_surrogate_predict(h, q)
        pb = rng.normal(0.0, 0.05, D.dirac_surrogate_get_params(h).size)
        D.dirac_surrogate_set_params(h, pb)
        y1 = D.dirac_surrogate_predict(h, q)
        D.dirac_surrogate_train(h, q, t, 2, 64, 1e-3)
        y2 = D.dirac_surrogate_predict(h, q)
        p2 = D.dirac_surrogate_get_params(h)
    finally:
        D.dirac_surrogate_destroy(h)
    assert not np.array_equal(y0, y1) and not np.array_equal(y1, y2)
    assert np.array_equal(y1, fresh(pb.astype(np.float32)))
    assert np.array_equal(y2, fresh(p2))


def test_stalled_weight_copy_is_reported_and_the_context_survives(D, monkeypatch):
    """DIRAC_INJECT_STALL makes the inference kernel's first weight wait run out (its barrier expects 16 bytes
    more than the copies deliver; the copies complete): the CTA gives up after its bounded wait, predict returns
    DIRAC_ERR_TIMEOUT, and the same process then predicts correctly with a network created without the hook."""
    import time
    rng = np.random.default_rng(9)
    q = LO + (HI - LO) * rng.uniform(0, 1, (100, 3))
    monkeypatch.setenv("DIRAC_INJECT_STALL", "1")
    h = D.dirac_surrogate_create(LO, HI, seed=2, max_batch=128)
    monkeypatch.delenv("DIRAC_INJECT_STALL")
    try:
        t0 = time.perf_counter()
        with pytest.raises(D.DiracError) as e:
            D.dirac_surrogate_predict(h, q)
        waited = time.perf_counter() - t0
        assert e.value.status == D.DIRAC_ERR_TIMEOUT
        assert 0.5 < waited < 20.0, waited
        p = D.dirac_surrogate_get_params(h)
    finally:
        D.dirac_surrogate_destroy(h)
    h2 = D.dirac_surrogate_create(LO, HI, seed=2, max_batch=128)
    try:
        D.dirac_surrogate_set_params(h2, p)
        y = D.dirac_surrogate_predict(h2, q)
    finally:
        D.dirac_surrogate_destroy(h2)
    want = M.predict(p.astype(np.float64), _norm(q))
    assert np.all(np.isfinite(y)) and np.max(np.abs(y - want)) < 1e-3


def test_training_fits_a_smooth_function(D):
    rng = np.random.default_rng(5)
    q = LO + (HI - LO) * rng.uniform(0, 1, (4096, 3))
    z = _norm(q)
    t = 1.0 / (1.0 + np.exp(-(1.5 * z[:, 0] - z[:, 1] + 0.5 * z[:, 0] * z[:, 2])))
    h = D.dirac_surrogate_create(LO, HI, seed=3, max_batch=512)
    try:
        loss0, _ = D.dirac_surrogate_gradient(h, q[:512], t[:512])
        loss = D.dirac_surrogate_train(h, q, t, epochs=60, batch=256, lr=2e-3)
        y = D.dirac_surrogate_predict(h, q[:512])
    finally:
        D.dirac_surrogate_destroy(h)
    assert loss < 1e-3 * loss0 + 2e-5
    assert np.max(np.abs(y - t[:512])) < 0.03


def _solver_cfg(D, fp32):
    cfg = D.dirac_batch_default_config()
    cfg.precision = D.DIRAC_FP32 if fp32 else D.DIRAC_FP64
    cfg.steps_per_launch = 2
    return cfg


def _solve(D, qs, fp32):
    runs = [D.dirac_klein_run_from_reduced(q, DX, C, 1.0) for q in qs]
    T, _ = D.dirac_batch_klein(runs, _solver_cfg(D, fp32))
    return T


def test_klein_surrogate_small_box(D):
    """Training from scratch inside the test (a smoke test of the training path, not the accuracy claim, which the
    shipped network's test above holds to |dT| <= 1e-3): 1024 batched FP32 solves train the network for 1500 epochs;
    48 held-out points are checked against the FP64 solver; queries outside the box fall back to the solver; the
    network answers >= 100x faster than per-run FP64 solves."""
    rng = np.random.default_rng(11)
    q_train = LO + (HI - LO) * rng.uniform(0, 1, (1024, 3))
    T_train = _solve(D, q_train, fp32=True)
    q_test = LO + (HI - LO) * rng.uniform(0, 1, (48, 3))
    t0 = time.perf_counter()
    T_fp64 = _solve(D, q_test, fp32=False)
    t_fp64 = (time.perf_counter() - t0) / len(q_test)
    h = D.dirac_surrogate_create(LO, HI, seed=1, max_batch=1024)
    try:
        D.dirac_surrogate_train(h, q_train, T_train, epochs=1500, batch=64, lr=1e-3)
        D.dirac_surrogate_predict(h, q_test)
        t0 = time.perf_counter()
        T_net = D.dirac_surrogate_predict(h, q_test)
        t_net = (time.perf_counter() - t0) / len(q_test)
        q_out = np.array([[0.4, 0.5, 20.0], [1.0, 1.2, 15.0]])
        T_out, used = D.dirac_surrogate_query(h, np.vstack([q_test[:3], q_out]), _solver_cfg(D, True))
    finally:
        D.dirac_surrogate_destroy(h)
    dT = np.abs(T_net - T_fp64)
    print("surrogate small box: mean |dT| %.2e, max %.2e; %.1f us/query vs FP64 solve %.1f ms/query"
          % (dT.mean(), dT.max(), t_net * 1e6, t_fp64 * 1e3))
    assert dT.mean() < 0.012 and dT.max() < 0.15
    assert list(used) == [False, False, False, True, True]
    assert np.allclose(T_out[3:], _solve(D, q_out, fp32=True), rtol=1e-12, atol=1e-15)
    assert t_fp64 / t_net > 100


def test_shipped_checkpoint_against_fp64_solver(D):
    """The shipped network (20000 FP32-labelled runs over V0/mc^2 in [0.5, 3], p0/mc in [0.2, 1], width/dx in
    [40, 150]) predicts the FP64 batched solver's transmission on 64 fresh points of the box to the scope's bar
    |dT| <= 1e-3: the mean within it and at most one point (the held-out 1000 had one, 1.1e-3) above it, that
    one below 2e-3."""
    import os
    path = os.path.join(os.path.dirname(D.__file__), "data", "surrogate_klein_box.npz")
    z = np.load(path)
    lo, hi = z["lo"], z["hi"]
    rng = np.random.default_rng(W.SEED + 5)
    q = lo + (hi - lo) * rng.uniform(0.0, 1.0, (64, 3))
    h = D.dirac_surrogate_create(lo, hi, seed=0, max_batch=64)
    try:
        D.dirac_surrogate_set_params(h, z["params"])
        T_net = D.dirac_surrogate_predict(h, q)
    finally:
        D.dirac_surrogate_destroy(h)
    cfg = D.dirac_batch_default_config()
    cfg.precision = D.DIRAC_FP64
    cfg.steps_per_launch = 2
    T64, _ = D.dirac_batch_klein([D.dirac_klein_run_from_reduced(x, DX, C, 1.0) for x in q], cfg)
    dT = np.abs(T_net - T64)
    print("shipped surrogate on 64 fresh points: mean |dT| %.2e, p99 %.2e, max %.2e"
          % (dT.mean(), np.percentile(dT, 99), dT.max()))
    assert dT.mean() <= 1e-3 and np.sum(dT > 1e-3) <= 1 and dT.max() < 2e-3, (dT.mean(), dT.max())


def test_checkpoint_save_load_resumes_training(D, tmp_path):
    """A checkpoint restores the box, parameters and Adam state: training on after a reload gives the same
    parameters as training on without it, and a foreign file is rejected."""
    rng = np.random.default_rng(21)
    q = LO + (HI - LO) * rng.uniform(0, 1, (512, 3))
    t = rng.uniform(0, 0.5, 512)
    path = str(tmp_path / "net.ckpt")
    h = D.dirac_surrogate_create(LO, HI, seed=3, max_batch=256)
    try:
        D.dirac_surrogate_train(h, q, t, 2, 128, 1e-3)
        D.dirac_surrogate_save(h, path)
        D.dirac_surrogate_train(h, q, t, 2, 128, 1e-3)
        want = D.dirac_surrogate_get_params(h)
    finally:
        D.dirac_surrogate_destroy(h)
    h2 = D.dirac_surrogate_create(np.zeros(3), np.ones(3), seed=99, max_batch=256)
    try:
        D.dirac_surrogate_load(h2, path)
        D.dirac_surrogate_train(h2, q, t, 2, 128, 1e-3)
        got = D.dirac_surrogate_get_params(h2)
        bad = tmp_path / "bad.ckpt"
        bad.write_bytes(b"not a checkpoint")
        with pytest.raises(D.DiracError) as e:
            D.dirac_surrogate_load(h2, str(bad))
        assert e.value.status == D.DIRAC_ERR_ARG
    finally:
        D.dirac_surrogate_destroy(h2)
    assert np.array_equal(got, want)
