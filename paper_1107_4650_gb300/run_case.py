"""Runs one Klein-step case through libdirac with a fixed launch plan and prints its timing.

  python -m paper_1107_4650_gb300.run_case --precision fp64 --side 2048 --nsteps 64 [--k 1 --p 4]

Used to profile one kernel configuration (no autotuning, no CPU work after the setup) and for quick
size sweeps.  The state is the 2-D Klein workload of the benchmark at the given side.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fx64"])
    ap.add_argument("--side", type=int, default=2048)
    ap.add_argument("--nsteps", type=int, default=64)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--k", type=int, default=0, help="steps per launch (0: library choice)")
    ap.add_argument("--p", type=int, default=0, help="points per lane (0: library choice)")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--ndim", type=int, default=2)
    ap.add_argument("--batch-runs", type=int, default=0, help="run this many ensemble runs as one batch instead")
    ap.add_argument("--seg", type=int, default=256, help="batch: rows per task")
    ap.add_argument("--shift", type=int, default=0, help="2-D: characteristic shift K (c dt = K dx)")
    ap.add_argument("--strang", action="store_true", help="second-order splitting (2-D or 3-D)")
    ap.add_argument("--autotune", action="store_true", help="let dirac_autotune choose the launch plan first")
    ap.add_argument("--field", action="store_true",
                    help="2-D: add a uniform two-cycle laser pulse (vector potential) over the run")
    ap.add_argument("--cellfield", action="store_true",
                    help="2-D/3-D: a field varying along x and in time (dirac_set_field) over the run")
    ap.add_argument("--mlp", type=int, default=0,
                    help="instead: train the transmission network this many epochs on seeded random targets")
    ap.add_argument("--queries", type=int, default=4096, help="--mlp: queries per timed prediction call")
    args = ap.parse_args()

    import torch

    import paper_1107_4650_gb300 as D
    from paper_1107_4650_gb300 import build as B
    from paper_1107_4650_gb300 import workloads as W

    B.build()
    D.load_library()
    prec = {"fp32": D.DIRAC_FP32, "fx64": D.DIRAC_FX64}.get(args.precision, D.DIRAC_FP64)
    stream = torch.cuda.Stream()
    if args.mlp > 0:
        lo, hi = np.array([0.5, 0.2, 40.0]), np.array([3.0, 1.0, 150.0])
        rng = np.random.default_rng(W.SEED + 6)
        X = lo + (hi - lo) * rng.uniform(0.0, 1.0, (4096, 3))
        T = rng.uniform(0.0, 0.3, 4096)
        hs = D.dirac_surrogate_create(lo, hi, seed=1, max_batch=4096, stream=stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loss = D.dirac_surrogate_train(hs, X, T, args.mlp, 256, 1e-3)
        e1.record(stream)
        stream.synchronize()
        Q = lo + (hi - lo) * rng.uniform(0.0, 1.0, (args.queries, 3))
        hq = D.dirac_surrogate_create(lo, hi, seed=1, max_batch=args.queries, stream=stream.cuda_stream)
        D.dirac_surrogate_set_params(hq, D.dirac_surrogate_get_params(hs))
        D.dirac_surrogate_predict(hq, Q)  # warm-up
        t_pred = []
        for _ in range(5):
            t0 = time.perf_counter()
            D.dirac_surrogate_predict(hq, Q)
            t_pred.append(time.perf_counter() - t0)
        D.dirac_surrogate_destroy(hq)
        D.dirac_surrogate_destroy(hs)
        ms = e0.elapsed_time(e1)
        print(json.dumps({"mlp_epochs": args.mlp, "train_ms": ms, "ms_per_iteration": ms / (args.mlp * 16),
                          "loss": loss, "queries": args.queries, "predict_s": min(t_pred),
                          "queries_per_s": args.queries / min(t_pred)}))
        return
    if args.batch_runs > 0:
        runs, _ = W.klein_ensemble(nruns=args.batch_runs)
        cfg = D.dirac_batch_default_config()
        cfg.precision = prec
        cfg.stream = stream.cuda_stream
        cfg.steps_per_launch = args.k or 2
        cfg.points_per_lane = args.p or 2
        cfg.segment_rows = args.seg
        cfg.use_graphs = 0 if args.no_graphs else 1
        hb = D.dirac_batch_create([r.as_batch_fields() for r in runs], cfg)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        D.dirac_batch_run(hb)
        e1.record(stream)
        stream.synchronize()
        info = D.dirac_batch_get_info(hb)
        T = D.dirac_batch_results(hb, len(runs))["T"]
        D.dirac_batch_destroy(hb)
        ms = e0.elapsed_time(e1)
        print(json.dumps({"batch_runs": len(runs), "ms": ms, "point_steps_per_s": info["point_steps"] / (ms / 1e3),
                          "k": info["steps_per_launch"], "p": info["points_per_lane"], "seg": info["segment_rows"],
                          "launches": info["launches"], "T_mean": float(np.mean(T))}))
        return
    if args.ndim == 2:
        run = W.klein_config_2d(side=args.side, nsteps=args.nsteps)
        x_min, z_min, _, _, face = run.geometry()
        psi = run.state()
        V = run.potential()
        shape = (args.side, 1, args.side)
        cfg = D.make_config(shape, x_min=(x_min, 0.0, z_min), flux_face=face, precision=prec,
                            stream=stream.cuda_stream, steps_per_launch=args.k, points_per_lane=args.p,
                            use_graphs=not args.no_graphs, char_shift=args.shift,
                            splitting=D.DIRAC_STRANG if args.strang else D.DIRAC_LIE)
        layout = D.DIRAC_V_X_ONLY
    else:
        n = args.side
        dx = W.DX_DEFAULT
        psi = W.gaussian_packet(n, n, dx, -n * dx / 2, -n * dx / 2, 32 * dx, 0.0, 16 * dx, 0.0, ny=n, y_min=-n * dx / 2)
        V = W.soft_coulomb_3d(n, dx, 10.0, 2 * dx).reshape(-1)
        shape = (n, n, n)
        cfg = D.make_config(shape, ndim=3, precision=prec, stream=stream.cuda_stream, points_per_lane=args.p,
                            steps_per_launch=args.k, use_graphs=not args.no_graphs,
                            splitting=D.DIRAC_STRANG if args.strang else D.DIRAC_LIE)
        layout = D.DIRAC_V_FULL
    h = D.dirac_create_grid(cfg)
    if args.cellfield:
        total = args.nsteps * args.repeat
        ncell = shape[0] * shape[1] * shape[2]
        xi = np.tile(np.arange(shape[0]), ncell // shape[0])
        a = np.stack([0.5 * np.sin(xi / 40.0), 0.2 * np.cos(xi / 25.0), 0.3 * np.cos(xi / 30.0)], axis=1)
        w = 1.5 * np.exp(-((xi - shape[0] / 2) / (shape[0] / 6)) ** 2)
        t = np.arange(total)
        F = np.stack([0.8 * np.sin(0.02 * t), 0.1 * np.cos(0.03 * t), 0.5 * np.cos(0.015 * t), 0.4 * np.sin(0.01 * t)],
                     axis=1)
        D.dirac_set_field(h, a, w, F)
    if args.field:
        total = args.nsteps * args.repeat
        dt = W.DX_DEFAULT / W.C_AU
        D.dirac_set_vector_potential(h, W.laser_A_tilde(total, dt, 2.0e4, 2 * np.pi / (total * dt / 2), 2.0))
    D.dirac_set_potential(h, V, layout)
    host = np.ascontiguousarray(psi.astype(np.complex64 if prec == D.DIRAC_FP32 else np.complex128))
    D.dirac_set_state(h, host)
    if args.autotune:
        D.dirac_autotune(h)
    times = []
    for it in range(args.repeat):
        if args.field or args.cellfield:
            D.dirac_set_counters(h, it * args.nsteps, 0.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        D.dirac_step(h, args.nsteps)
        e1.record(stream)
        stream.synchronize()
        times.append(e0.elapsed_time(e1))
    obs = D.dirac_observables(h)
    info = D.dirac_get_info(h)
    D.dirac_destroy(h)
    cells = shape[0] * shape[1] * shape[2]
    best = min(times)
    print(json.dumps({"precision": args.precision, "ndim": args.ndim, "side": args.side, "nsteps": args.nsteps,
                      "ms": best, "point_steps_per_s": cells * args.nsteps / (best / 1e3),
                      "k": info["steps_per_launch"], "p": info["points_per_lane"], "plan": info["plan"],
                      "warps": info["launch_warps"], "seg_rows": info["segment_rows"], "norm": obs["norm"],
                      "flux": obs["flux_cum"]}))


if __name__ == "__main__":
    t0 = time.time()
    main()
