"""Pins of the CPU network oracle: its FP64 gradient against central finite differences, and its BF16
rounding against torch's float -> bfloat16 conversion."""
import numpy as np
import pytest

from oracle import mlp as M


def _params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in M.SHAPES:
        fan_in = shape[1] if len(shape) == 2 else (M.HID if name.startswith("w") else 1)
        d[name] = rng.standard_normal(shape) * scale / np.sqrt(fan_in)
    return M.pack(d)


def test_fp64_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params()
    x = rng.uniform(-1, 1, (7, 3))
    t = rng.uniform(0, 1, 7)
    _, g = M.loss_and_grad(p, x, t, round_bf16=False)
    offs, o = {}, 0
    for name, shape in M.SHAPES:
        offs[name] = (o, int(np.prod(shape)))
        o += offs[name][1]
    idx = []
    for name, (o0, n) in offs.items():
        idx += list(o0 + rng.choice(n, size=min(n, 6), replace=False))
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_and_grad(pp, x, t, False)[0] - M.loss_and_grad(pm, x, t, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    a = np.concatenate([rng.standard_normal(5000).astype(np.float32) * 10 ** rng.uniform(-8, 8, 5000).astype(np.float32),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, -0.0], dtype=np.float32)])
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(a), want)


def test_rounded_gradient_is_close_to_exact():
    rng = np.random.default_rng(3)
    p = _params(seed=4)
    x = rng.uniform(-1, 1, (64, 3))
    t = rng.uniform(0, 1, 64)
    _, g0 = M.loss_and_grad(p, x, t, round_bf16=False)
    _, g1 = M.loss_and_grad(p, x, t, round_bf16=True)
    assert np.linalg.norm(g1 - g0) / np.linalg.norm(g0) < 0.05
