"""Caller-owned state buffers (dirac_config.ext_state): the grid steps in two torch-allocated device buffers
without copying the state in or out, and the result is the oracle's, bit for bit in FP64."""
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
    import paper_1107_4650_gb300 as D
    D.load_library()
    return D


def _klein(side=320, nsteps=200):
    run = W.KleinRun(side=side, V0=2.5 * C * C, p0=0.6 * C, width=12 * DX, nsteps=nsteps, face=side // 2)
    x_min, z_min, _, _, face = run.geometry()
    return run, run.state(), run.potential(), (x_min, 0.0, z_min), face


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fx64"])
def test_klein_steps_in_torch_owned_buffers(D, prec):
    torch = pytest.importorskip("torch")
    run, psi0, V, x_min, face = _klein()
    side = run.side
    want, F = oracle.step(psi0, 2, 1.0, C, DX, run.nsteps, V=V, flux_face=face)
    precision = {"fp64": D.DIRAC_FP64, "fp32": D.DIRAC_FP32, "fx64": D.DIRAC_FX64}[prec]
    if prec == "fp32":
        host = psi0.astype(np.complex64).view(np.float32)
    else:
        host = psi0.view(np.float64)
    bufs = [torch.from_numpy(np.ascontiguousarray(host)).cuda(), torch.full(host.shape, float("nan"),
                                                                            dtype=torch.float32 if prec == "fp32"
                                                                            else torch.float64, device="cuda")]
    if prec == "fx64":
        bufs = [b.view(torch.int64) for b in bufs]
    torch.cuda.synchronize()
    state_bytes = side * side * 8 * (4 if prec == "fp32" else 8)
    cfg = D.make_config((side, 1, side), x_min=x_min, flux_face=face, precision=precision, ext_state=bufs)
    h = D.dirac_create_grid(cfg)
    try:
        info = D.dirac_get_info(h)
        assert info["device_bytes"] < state_bytes  # the grid's own table and scratch only
        D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY)
        if prec == "fx64":
            # complex128 in through the idle caller buffer, encoded into the current one
            D.dirac_set_state(h, torch.from_numpy(psi0.view(np.float64)).cuda())
        else:
            D.dirac_set_state(h, bufs[0])  # the buffer already holds the state: no copy
        D.dirac_step(h, run.nsteps)
        obs = D.dirac_observables(h)
        info = D.dirac_get_info(h)
        assert D.dirac_state_ptr(h) == bufs[info["state_index"]].data_ptr()
        if prec == "fx64":
            got = np.empty_like(psi0)
            D.dirac_get_state(h, got)
        else:
            torch.cuda.synchronize()
            got = bufs[info["state_index"]].cpu().numpy().view(np.complex64 if prec == "fp32" else np.complex128)
            got = got.reshape(psi0.shape)
    finally:
        D.dirac_destroy(h)
    # the buffers outlive the grid and still hold the state
    torch.cuda.synchronize()
    assert torch.isfinite(bufs[0].double()).all() if prec != "fx64" else True
    if prec == "fp64":
        assert np.array_equal(got.view(np.float64), want.view(np.float64))
        assert abs(obs["flux_cum"] - F) <= 1e-12 * abs(F)
    elif prec == "fx64":
        assert np.linalg.norm((got - want).ravel()) <= 1e-12 * np.linalg.norm(want.ravel())
    else:
        err = np.linalg.norm((got.astype(np.complex128) - want).ravel()) / np.linalg.norm(want.ravel())
        assert err < 2e-5


def test_ext_state_in_3d_and_graph_replay(D):
    """3-D grid in caller buffers, enough steps for graph replay: the same bits as a grid with its own buffers."""
    torch = pytest.importorskip("torch")
    nx, ny, nz = 40, 24, 20
    psi0 = W.random_state(nz, ny, nx, seed=41)
    V = np.random.default_rng(42).uniform(-3e4, 3e4, nx * ny * nz)
    bufs = [torch.from_numpy(psi0.view(np.float64).copy()).cuda(), torch.zeros(psi0.size * 2, dtype=torch.float64,
                                                                               device="cuda")]
    torch.cuda.synchronize()
    out = []
    for ext in (bufs, None):
        cfg = D.make_config((nx, ny, nz), ndim=3, ext_state=ext)
        h = D.dirac_create_grid(cfg)
        try:
            D.dirac_set_potential(h, V, D.DIRAC_V_FULL)
            if ext is None:
                D.dirac_set_state(h, psi0)
            D.dirac_step(h, 70)
            got = np.empty_like(psi0)
            D.dirac_get_state(h, got)
            out.append(got)
        finally:
            D.dirac_destroy(h)
    assert np.array_equal(out[0].view(np.float64), out[1].view(np.float64))


def test_ext_state_rejects_host_and_misaligned_buffers(D):
    torch = pytest.importorskip("torch")
    side = 64
    good = torch.zeros(side * side * 8 + 2, dtype=torch.float64, device="cuda")
    other = torch.zeros(side * side * 8, dtype=torch.float64, device="cuda")
    host = np.zeros(side * side * 8, np.float64)
    for pair in ((host.ctypes.data, other.data_ptr()), (good.data_ptr() + 8, other.data_ptr()),
                 (good.data_ptr(), good.data_ptr() + 64)):
        cfg = D.make_config((side, 1, side))
        cfg.ext_state[0], cfg.ext_state[1] = pair
        with pytest.raises(D.DiracError) as e:
            D.dirac_create_grid(cfg)
        assert e.value.status == D.DIRAC_ERR_ARG


@pytest.mark.parametrize("shape,ndim", [((1, 1, 1), 2), ((1, 1, 1), 3), ((5, 1, 3), 2), ((3, 4, 2), 3)])
def test_ext_state_tiny_grids(D, shape, ndim):
    """Caller-owned buffers of one-cell and small grids: the same bits as the oracle after 9 steps."""
    torch = pytest.importorskip("torch")
    nx, ny, nz = shape
    psi = W.random_state(nz, ny, nx, seed=nx + 3 * ny + 7 * nz + ndim)
    want, _ = oracle.step(psi, ndim, 1.0, C, DX, 9)
    bufs = [torch.from_numpy(psi.view(np.float64).copy()).cuda(), torch.zeros(psi.size * 2, dtype=torch.float64,
                                                                              device="cuda")]
    torch.cuda.synchronize()
    h = D.dirac_create_grid(D.make_config((nx, ny, nz), ndim=ndim, ext_state=bufs))
    try:
        D.dirac_step(h, 9)
        got = np.empty_like(psi)
        D.dirac_get_state(h, got)
    finally:
        D.dirac_destroy(h)
    assert np.array_equal(got.view(np.float64), want.view(np.float64))
