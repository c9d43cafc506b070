"""Trains the Klein-transmission surrogate over the ensemble's parameter box and checks it against the FP64 solver.

  python -m paper_1107_4650_gb300.surrogate_train --train 20000 --heldout 1000 --epochs 6000 --out surrogate.npz

1. Draws `train` and `heldout` reduced parameter sets q = (V0/mc^2, p0/mc, width/dx) uniformly over the box
   [0.5, 3.0] x [0.2, 1.0] x [40, 150] (numpy PCG64, seeds 20111107+2 and +3).
2. Labels the training set with the batched FP32 solver (dirac_batch_klein, runs built by
   dirac_klein_run_from_reduced), in chunks.
3. Trains the network (dirac_surrogate_train) on the GPU.
4. Judges the held-out set with the batched FP64 solver and reports |dT|, plus the time per query of the
   network, of the batched FP32 solve and of the FP64 solve.
Writes the FP32 parameters, the box and the statistics to --out (npz).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

LO = np.array([0.5, 0.2, 40.0])
HI = np.array([3.0, 1.0, 150.0])


def draw(n, seed):
    rng = np.random.default_rng(seed)
    return LO + (HI - LO) * rng.uniform(0.0, 1.0, (n, 3))


def solve(D, W, qs, fp32, chunk=512):
    cfg = D.dirac_batch_default_config()
    cfg.precision = D.DIRAC_FP32 if fp32 else D.DIRAC_FP64
    cfg.steps_per_launch = 2
    cfg.points_per_lane = 2
    cfg.segment_rows = 256
    out = np.zeros(len(qs))
    for i in range(0, len(qs), chunk):
        runs = [D.dirac_klein_run_from_reduced(q, W.DX_DEFAULT, W.C_AU, 1.0) for q in qs[i:i + chunk]]
        out[i:i + chunk], _ = D.dirac_batch_klein(runs, cfg)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--heldout", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default="surrogate.npz")
    ap.add_argument("--data", default="", help="reuse the labelled sets saved in an earlier --out file")
    args = ap.parse_args()

    import paper_1107_4650_gb300 as D
    from paper_1107_4650_gb300 import build as B
    from paper_1107_4650_gb300 import workloads as W

    B.build()
    D.load_library()
    if args.data:
        z = np.load(args.data)
        q_tr, T_tr, q_te, T_te = z["q_train"], z["T_train"], z["q_heldout"], z["T_heldout_fp64"]
        old = json.loads(str(z["stats"]))
        t_label, t_check = old.get("label_s", 0.0), old.get("check_s", old.get("judge_s", 0.0))
        args.train, args.heldout = len(q_tr), len(q_te)
    else:
        q_tr = draw(args.train, W.SEED + 2)
        q_te = draw(args.heldout, W.SEED + 3)
        t0 = time.perf_counter()
        T_tr = solve(D, W, q_tr, fp32=True)
        t_label = time.perf_counter() - t0
        t0 = time.perf_counter()
        T_te = solve(D, W, q_te, fp32=False)
        t_check = time.perf_counter() - t0
    h = D.dirac_surrogate_create(LO, HI, seed=W.SEED, max_batch=4096)
    t0 = time.perf_counter()
    loss = D.dirac_surrogate_train(h, q_tr, T_tr, epochs=args.epochs, batch=args.batch, lr=args.lr)
    t_train = time.perf_counter() - t0
    D.dirac_surrogate_predict(h, q_te)
    t0 = time.perf_counter()
    T_net = D.dirac_surrogate_predict(h, q_te)
    t_net = time.perf_counter() - t0
    params = D.dirac_surrogate_get_params(h)
    D.dirac_surrogate_destroy(h)
    dT = np.abs(T_net - T_te)
    stats = {"train": args.train, "heldout": args.heldout, "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
             "final_train_mse": loss, "dT_mean": float(dT.mean()), "dT_p99": float(np.quantile(dT, 0.99)),
             "dT_max": float(dT.max()), "frac_dT_le_1e-3": float((dT <= 1e-3).mean()),
             "s_per_query_net": t_net / len(q_te), "s_per_query_fp32_batch": t_label / len(q_tr),
             "s_per_query_fp64_batch": t_check / len(q_te), "label_s": t_label, "check_s": t_check,
             "train_s": t_train, "T_train_mean": float(T_tr.mean()), "T_train_max": float(T_tr.max())}
    np.savez(args.out, params=params, lo=LO, hi=HI, stats=json.dumps(stats), q_train=q_tr, T_train=T_tr,
             q_heldout=q_te, T_heldout_fp64=T_te)
    print(json.dumps(stats))


if __name__ == "__main__":
    main()
