"""The paper's 2-D Klein-paradox run (Sec. 5.2.2) at its full size on one GPU.

  python -m paper_1107_4650_gb300.paper_klein2d [--precision fp64|fp32|fx64] [--steps 12000]

Mesh 24576 x 8192 over x in [-15, 15], z in [-5, 5] a.u. (dx = 10/8192 a.u.), second-order splitting
(dt = 2 dx / c = 1.78e-5 a.u.), 12000 steps to t = 0.214 a.u., zero boundary; step V(x) = V0/2 (1 + tanh(x/L))
with L = 0.0025 a.u. and V0 = 2 m c^2 + 1e4 a.u. (the height that reproduces the printed analytic T);
initial state N [1, 0, 0, C] e^{i k0 x} exp(-((x - x0)^2 + z^2) / (4 width^2)) with k0 = 100 a.u., width 1 a.u.,
x0 = -6 a.u. (not printed: the packet starts clear of the step).  The paper reports T = 0.2407, R = 0.7593
(analytic 0.2621 / 0.7380) after about 22 h on 256 processors.

The packet is separable, so its two factors are built with numpy and their outer product is formed on the
device; the state never exists on the host.  Prints one JSON line: T as the cumulative flux through x = 0,
T and R as the norm right and left of x = 0 at the end, the wall time of the stepping and its rate.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def run(precision: str = "fp64", steps: int = 12000, x0: float = -6.0, stream=None, device: int = 0) -> dict:
    """Runs the experiment on cuda:device (the library already loaded) and returns the result dict."""
    import torch

    import paper_1107_4650_gb300 as D
    from paper_1107_4650_gb300 import workloads as W

    c, m = W.C_AU, W.M_E
    nx, nz = 24576, 8192
    dx = 30.0 / nx
    x_min, z_min = -15.0, -5.0
    face = nx // 2
    k0, width, L = 100.0, 1.0, 0.0025
    V0 = 2 * m * c * c + 1.0e4
    x = W.cell_centres(nx, dx, x_min)
    z = W.cell_centres(nz, dx, z_min)
    fx = np.exp(1j * k0 * x - (x - x0) ** 2 / (4 * width ** 2))
    fz = np.exp(-(z ** 2) / (4 * width ** 2))
    norm = np.sqrt((np.abs(fx) ** 2).sum() * (np.abs(fz) ** 2).sum() * dx * dx * (1 + W.spinor_C(k0, m, c) ** 2))
    fx = fx / norm
    fp32 = precision == "fp32"
    cdt = torch.complex64 if fp32 else torch.complex128
    dev = torch.device("cuda:%d" % device)
    psi = torch.zeros((nz, 1, nx, 4), dtype=cdt, device=dev)
    outer = torch.outer(torch.from_numpy(fz).to(dev), torch.from_numpy(fx).to(dev)).to(cdt)
    psi[:, 0, :, 0] = outer
    psi[:, 0, :, 3] = outer * W.spinor_C(k0, m, c)
    del outer
    stream = stream if stream is not None else torch.cuda.Stream(device=dev)
    cfg = D.make_config((nx, 1, nz), dx=dx, x_min=(x_min, 0.0, z_min), flux_face=face, splitting=D.DIRAC_STRANG,
                        precision={"fp32": D.DIRAC_FP32, "fx64": D.DIRAC_FX64}.get(precision, D.DIRAC_FP64),
                        stream=stream.cuda_stream, device=device)
    h = D.dirac_create_grid(cfg)
    try:
        D.dirac_set_potential(h, W.tanh_step(nx, dx, x_min, 0.0, V0, L), D.DIRAC_V_X_ONLY)
        torch.cuda.synchronize(dev)  # the packet is complete before the grid's stream copies it
        D.dirac_set_state(h, torch.view_as_real(psi).reshape(-1))
        stream.synchronize()         # and the copy is complete before the tensor is freed
        del psi
        o0 = D.dirac_observables(h)
        D.dirac_autotune(h)
        info = D.dirac_get_info(h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        D.dirac_step(h, steps)
        e1.record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
        ms = e0.elapsed_time(e1)
        o1 = D.dirac_observables(h)
    finally:
        D.dirac_destroy(h)
    n0 = o0["norm"]
    return {
        "run": "Sec. 5.2.2 2-D Klein paradox, %d x %d, %d second-order steps (t = %.4f a.u.), %s"
               % (nx, nz, steps, steps * 2 * dx / c, precision),
        "T_flux": o1["flux_cum"] / n0, "T_right": o1["norm_right"] / n0,
        "R_left": (o1["norm"] - o1["norm_right"]) / n0, "norm_end": o1["norm"] / n0,
        "paper": {"T": 0.2407, "R": 0.7593, "analytic_T": 0.2621, "wall_h": 22.0, "processes": 256},
        "gpu_ms": ms, "wall_s": wall, "point_steps_per_s": nx * nz * steps / (ms / 1e3),
        "speedup_vs_paper_wall": 22.0 * 3600.0 / wall,
        "steps_per_launch": info["steps_per_launch"], "points_per_lane": info["points_per_lane"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fx64"])
    ap.add_argument("--steps", type=int, default=12000)
    ap.add_argument("--x0", type=float, default=-6.0)
    args = ap.parse_args()

    import paper_1107_4650_gb300 as D
    from paper_1107_4650_gb300 import build as B

    B.build()
    D.load_library()
    print(json.dumps(run(args.precision, args.steps, args.x0)))


if __name__ == "__main__":
    main()
