#!/usr/bin/env python
"""Benchmark of the split-operator Dirac stepper on one GB300.

Workload (one bench step): the 2-D Klein-step scattering run, FP64 state, 2048 x 2048 cells of
dx = 10/8192 a.u., tanh step V0 = 2.5 m c^2, L = 4 dx on the face at 5/8 of the x extent, Gaussian
[1,0,0,C] packet of width 100 dx with p0 drawn from U[0.2, 1.0] m c (numpy PCG64, seed 20111107),
4000 time steps with the transmitted flux accumulated every step.  The metric is 4-spinor
grid-point-steps per second (cells x time steps / s).

  value      device-resident inputs: each bench step re-seeds the state from a device copy and
             runs dirac_step(4000); timed with CUDA events on the grid's stream.
  e2e        the same through the C ABI with host buffers: pinned host state -> device, potential
             from host, 4000 steps, observables (norm, flux) read back to the host.
  roofline   the step kernel: algorithmic bytes per launch (128 B per FP64 point-step: the state
             read and written once) / its mean launch time; FP64 arithmetic (56 flops per 2-D
             point-step) against the FP64 rate.
  cpu_baseline  the FP64 CPU oracle on this host's cores, on a bounded sample of the same run.
  variants   further legs; "fx64" runs the same workload with 64-bit fixed-point storage (exact integer
             sweeps, the phase rounded once) and reports its relative L2 distance from the FP64 state.

With --gpus N > 1 (torchrun), every rank runs an independent replica of the single-grid legs (one grid per
GPU, not sharded) and its own share of a global ensemble draw in the batched leg; value = all ranks'
point-steps / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FP64_BYTES_PER_POINT_STEP = 128  # 2-D, x-only table: 64 B read + 64 B written
FP32_BYTES_PER_POINT_STEP = 64
FLOPS_PER_POINT_STEP_2D = 56    # 32 adds (two sweeps) + 4 complex products of 6 flops
FP64_INSTR_PER_POINT_STEP_2D = 48  # 32 DADD + 8 DMUL + 8 DFMA: what the FP64 pipe issues per 2-D point-step
FP64_INSTR_PER_POINT_STEP_2D_FIELD = 80  # with a vector potential: 32 DADD + 12 complex multiply-adds of 4 DFMA
# FP64 issue roof from GB300's unit counts and clock: 1.25 TFLOP/s FP64 with a DFMA counted as two flops is two
# FP64 instructions per SM per clock (DADD and DMUL issue at the DFMA rate): 2 x 152 SMs x 2.07 GHz.
FP64_INSTR_PER_SM_CLOCK = 2
SM_COUNT = 152
FP64_ISSUE_PEAK_NOMINAL = FP64_INSTR_PER_SM_CLOCK * SM_COUNT * 2.07e9 / 1e12  # 0.629 T FP64 instructions/s
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the step kernel on the 2048^2 workload, keyed
# by (steps per launch, points per lane) of the captured variant (profiles/step_kernel_fp64_klein2048.md,
# profiles/step_kernel_fp32_klein2048.md).  A variant without a capture reports null.
MEASURED_TRAFFIC_PER_LAUNCH = {"fp64": {(1, 2): 277.539584e6 + 216.977408e6, (1, 4): 287.031808e6 + 217.295616e6},
                               "fp32": {(2, 2): 152.147456e6 + 83.809024e6},
                               "fx64": {(1, 1): 277.640448e6 + 217.100288e6}}
# ncu sm__pipe_fp64_cycles_active of the same captures (fraction of active cycles)
MEASURED_FP64_PIPE = {(1, 2): 0.8311, (1, 4): 0.8297}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=2048)
    ap.add_argument("--nsteps", type=int, default=4000, help="time steps per bench step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-fx64", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-field", action="store_true")
    ap.add_argument("--no-2d-variants", action="store_true", help="skip the 2-D Strang and shift legs")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--paper-klein", action="store_true",
                    help="also run the paper's full 24576 x 8192 Klein experiment in FP32 (about 40 s)")
    ap.add_argument("--no-config3", action="store_true", help="skip the 384^3 x 1000-step soft-Coulomb sweep over Z")
    ap.add_argument("--config3-steps", type=int, default=1000)
    ap.add_argument("--config3-z", default="1,2,5,10,20")
    ap.add_argument("--side3d", type=int, default=384)
    ap.add_argument("--batch-runs", type=int, default=512)
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--check-points", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=0.0,
                    help="--impl reference: oracle seconds per step (0: about 60 s over all steps, 2 s at least)")
    ap.add_argument("--cpu-detail-seconds", type=float, default=3.0,
                    help="per sample of the CPU oracle detail (one thread; 3-D grid; ensemble); 0 = skip")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(run, seconds: float):
    """The FP64 CPU oracle, as it stands, on this host's cores: chunks of 25 steps of the same Klein run on a
    1024^2 crop until `seconds` of wall time; returns (point-steps/s, threads, description)."""
    ncores = os.cpu_count() or 1
    os.environ["OMP_NUM_THREADS"] = str(ncores)
    import oracle
    from paper_1107_4650_gb300 import workloads as W
    oracle.build()
    side = 1024
    crop = W.KleinRun(side=side, V0=run.V0, p0=run.p0, width=run.width / 2, nsteps=run.nsteps, dx=run.dx, L=run.L)
    psi = crop.state()
    V = crop.potential()
    _, _, _, _, face = crop.geometry()
    done = 0
    F = 0.0
    t0 = time.perf_counter()
    while True:
        psi, F = oracle.step(psi, 2, 1.0, W.C_AU, crop.dx, 25, V=V, flux_face=face, flux_cum=F)
        done += 25
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    rate = side * side * done / dt
    desc = ("FP64 CPU oracle, %d OpenMP threads, %dx%d crop of the Klein run (width 50 dx), %d time steps in %.1f s"
            % (ncores, side, side, done, dt))
    return rate, ncores, desc


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


_ONE_THREAD = r"""
import sys, time, json
sys.path.insert(0, %r)
import oracle
from paper_1107_4650_gb300 import workloads as W
side = 512
run = W.KleinRun(side=side, V0=%r, p0=%r, width=%r, nsteps=1, dx=%r, L=%r)
psi, V = run.state(), run.potential()
face = run.geometry()[4]
done, F, t0 = 0, 0.0, time.perf_counter()
while True:
    psi, F = oracle.step(psi, 2, 1.0, W.C_AU, run.dx, 5, V=V, flux_face=face, flux_cum=F)
    done += 5
    if time.perf_counter() - t0 >= %r:
        break
print(json.dumps({"rate": side * side * done / (time.perf_counter() - t0), "steps": done}))
"""


def cpu_detail(run, seconds: float) -> dict:
    """Oracle timings beside the headline CPU baseline, each a bounded sample of about `seconds`: the host's CPU
    model and core count; the 2-D Klein run on one thread (512^2 crop, a child process with OMP_NUM_THREADS=1);
    the 3-D soft-Coulomb grid (128^3 crop, first order, per-cell potential) and the ensemble (the first 16
    runs of the draw, absorbing layers on, 10 steps each, repeated) on all cores."""
    import oracle
    from paper_1107_4650_gb300 import workloads as W
    oracle.build()
    here = os.path.dirname(os.path.abspath(__file__))
    out = {"cpu_model": _cpu_model(), "nproc": os.cpu_count()}
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = _ONE_THREAD % (here, run.V0, run.p0, run.width / 4, run.dx, run.L, seconds)
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=120 + 10 * seconds)
        one = json.loads(r.stdout.strip().splitlines()[-1])
        out["klein2d_one_thread"] = {"value": one["rate"], "unit": "point-steps/s", "threads": 1,
                                     "sample": "512x512 crop of the Klein run (width 25 dx), %d steps" % one["steps"]}
    except (OSError, subprocess.SubprocessError, ValueError, IndexError, KeyError) as e:
        out["klein2d_one_thread"] = {"error": str(e)[:200]}
    n3, dx = 128, W.DX_DEFAULT
    psi3 = W.gaussian_packet(n3, n3, dx, -n3 * dx / 2, -n3 * dx / 2, 32 * dx, 0.0, 16 * dx, 0.0, ny=n3,
                             y_min=-n3 * dx / 2)
    V3 = W.soft_coulomb_3d(n3, dx, 10.0, 2 * dx).reshape(-1)
    done, t0 = 0, time.perf_counter()
    while True:
        psi3, _ = oracle.step(psi3, 3, 1.0, W.C_AU, dx, 2, V=V3)
        done += 2
        if time.perf_counter() - t0 >= seconds:
            break
    out["coulomb3d_all_cores"] = {"value": n3 ** 3 * done / (time.perf_counter() - t0), "unit": "point-steps/s",
                                  "threads": os.cpu_count(),
                                  "sample": "128^3 crop of the 3-D soft-Coulomb grid (Z = 10), %d first-order steps"
                                            % done}
    runs, _ = W.klein_ensemble(16, seed=W.SEED + 1)
    states = [(r, r.state(), r.potential(), r.geometry()[4], r.mask()) for r in runs]
    pts, passes, t0 = 0, 0, time.perf_counter()
    while True:
        for r, psi, V, face, mask in states:
            oracle.step(psi, 2, 1.0, W.C_AU, r.dx, 10, V=V, flux_face=face, absorber=mask)
            pts += r.side * r.side * 10
        passes += 1
        if time.perf_counter() - t0 >= seconds:
            break
    out["ensemble_all_cores"] = {"value": pts / (time.perf_counter() - t0), "unit": "point-steps/s",
                                 "threads": os.cpu_count(),
                                 "sample": "first 16 runs of the ensemble draw (sides %s), 10 steps each, %d passes"
                                           % (sorted({r.side for r in runs}), passes)}
    return out


def reference_arm(args, rank, world):
    if rank != 0:
        return
    from paper_1107_4650_gb300 import workloads as W
    run = W.klein_config_2d(side=args.side, nsteps=args.nsteps)
    per = args.ref_step_seconds if args.ref_step_seconds > 0 else max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(run, min(1.0, per))
    vals, secs = [], []
    cores, desc = None, ""
    for _ in range(args.steps):
        t0 = time.perf_counter()
        v, cores, desc = cpu_baseline(run, per)
        secs.append(time.perf_counter() - t0)
        vals.append(v)
    value = float(np.mean(vals))
    sampled_ms = float(np.mean(secs)) * 1e3
    full_ms = args.side * args.side * args.nsteps / value * 1e3
    line = {"impl": "reference", "metric": "4-spinor grid-point-steps/s", "value": value, "unit": "point-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sampled_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "2-D Klein step FP64 %dx%d, %d time steps (CPU oracle: each bench step is a "
                                   "bounded sample of about %.0f s on a 1024^2 crop of the run with the packet width "
                                   "halved to 50 dx so that it fits the crop; value is the sample's rate per "
                                   "point-step)" % (args.side, args.side, args.nsteps, per),
                       "sampled_seconds_per_step": sampled_ms / 1e3,
                       "extrapolated_ms_for_the_full_%d_steps_at_%d^2" % (args.nsteps, args.side): full_ms},
            "cpu_baseline": {"value": value, "unit": "point-steps/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "point-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch
    import paper_1107_4650_gb300 as D
    from paper_1107_4650_gb300 import build as B
    from paper_1107_4650_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if world > 1:
        dist.barrier()
    D.load_library()

    run = W.klein_config_2d(side=args.side, nsteps=args.nsteps)
    x_min, z_min, _, _, face = run.geometry()
    psi0 = run.state()
    V = run.potential()
    ncell = args.side * args.side
    stream = torch.cuda.Stream()

    def make_grid(precision):
        cfg = D.make_config((args.side, 1, args.side), x_min=(x_min, 0.0, z_min), flux_face=face,
                            stream=stream.cuda_stream, device=local, precision=precision)
        h = D.dirac_create_grid(cfg)
        D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY)
        return h

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed_device_run(h, dev_state, steps, warmup):
        """(total ms, ms inside dirac_step only, step-kernel launches in the timed region)."""
        for _ in range(warmup):
            D.dirac_set_state(h, dev_state)
            D.dirac_step(h, args.nsteps)
        stream.synchronize()
        barrier()
        torch.cuda.synchronize()
        l0 = D.dirac_get_info(h)["kernel_launches"]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        e_all0, e_all1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_all0.record(stream)
        for i in range(steps):
            D.dirac_set_state(h, dev_state)
            ev[i][0].record(stream)
            D.dirac_step(h, args.nsteps)
            ev[i][1].record(stream)
        e_all1.record(stream)
        stream.synchronize()
        barrier()
        torch.cuda.synchronize()
        total = e_all0.elapsed_time(e_all1)
        inner = sum(a.elapsed_time(b) for a, b in ev)
        launches = D.dirac_get_info(h)["kernel_launches"] - l0
        return total, inner, launches

    from paper_1107_4650_gb300 import distributed as PD

    def max_over_ranks(x):
        return PD.max_over_ranks(x, world, device="cuda")

    # ---------------------------------------------------------------- FP64, device-resident
    h = make_grid(D.DIRAC_FP64)
    dev_state = torch.from_numpy(psi0.view(np.float64)).to(f"cuda:{local}")
    torch.cuda.synchronize()
    D.dirac_set_state(h, dev_state)
    D.dirac_autotune(h)
    info = D.dirac_get_info(h)
    with ClockSampler(local) as clk:
        total_ms, inner_ms, launches = timed_device_run(h, dev_state, args.steps, args.warmup)
    clocks = clk.summary()
    obs = D.dirac_observables(h)
    n0 = float(np.sum(np.abs(psi0) ** 2) * run.dx ** 2)
    total_ms = max_over_ranks(total_ms)
    point_steps = ncell * args.nsteps * args.steps * world
    value = point_steps / (total_ms / 1e3)
    step_launches = args.steps * (args.nsteps // info["steps_per_launch"] + args.nsteps % info["steps_per_launch"])
    mean_launch_s = inner_ms / 1e3 / max(1, step_launches)
    k_launch = info["steps_per_launch"]
    alg_bytes = FP64_BYTES_PER_POINT_STEP * ncell * k_launch
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved_gbs = alg_bytes / mean_launch_s / 1e9
    fp64_tips = FP64_INSTR_PER_POINT_STEP_2D * ncell * k_launch / mean_launch_s / 1e12
    traffic = (MEASURED_TRAFFIC_PER_LAUNCH["fp64"].get((k_launch, info["points_per_lane"]))
               if args.side == 2048 else None)
    roofline = {"bound": "alu", "achieved": fp64_tips, "peak": FP64_ISSUE_PEAK_NOMINAL, "unit": "T FP64-instr/s",
                "frac": fp64_tips / FP64_ISSUE_PEAK_NOMINAL, "traffic": traffic,
                "peak_source": "derived from unit counts and clock: 2 FP64 instructions per SM per clock (GB300's "
                               "1.25 TFLOP/s FP64, a DFMA counted as two flops) x 152 SMs x 2.07 GHz; "
                               "MEASURED_PEAKS.json has no FP64 figure",
                "ncu_fp64_pipe_active": MEASURED_FP64_PIPE.get((k_launch, info["points_per_lane"])),
                "achieved_tflops": FLOPS_PER_POINT_STEP_2D * ncell * k_launch / mean_launch_s / 1e12,
                "kernel": "dirac::sweep_kernel<double,%d,%d,0>" % (k_launch, info["points_per_lane"]),
                "mean_launch_ms": mean_launch_s * 1e3,
                "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
                        "peak_source": hbm_src, "algorithmic_bytes_per_launch": alg_bytes,
                        "basis": "128 B per FP64 point-step (state read and written once, x-only table)"}}

    # ---------------------------------------------------------------- e2e through host buffers
    e2e = None
    if not args.no_e2e:
        host_state = torch.from_numpy(psi0.view(np.float64)).pin_memory()
        def e2e_step():
            D.dirac_set_state(h, host_state)
            D.dirac_set_potential(h, V, D.DIRAC_V_X_ONLY)
            D.dirac_step(h, args.nsteps)
            return D.dirac_observables(h)
        e2e_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r = e2e_step()
        stream.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": point_steps / e2e_s, "unit": "point-steps/s",
               "h2d_bytes_per_step": int(psi0.nbytes + V.nbytes), "d2h_bytes_per_step": 6 * 8,
               "result": {"T": r["flux_cum"] / n0, "norm": r["norm"]}}
    # the FP64 state after one bench step (bit-exact with the oracle) and its flux: the reference of the
    # fixed-point leg below
    fp64_final = torch.empty_like(dev_state)
    D.dirac_set_state(h, dev_state)
    D.dirac_step(h, args.nsteps)
    D.dirac_get_state(h, fp64_final)
    stream.synchronize()
    obs_final = D.dirac_observables(h)
    fp64_flux, fp64_norm = obs_final["flux_cum"], obs_final["norm"]
    D.dirac_destroy(h)
    variants = {}

    # ---------------------------------------------------------------- 64-bit fixed-point storage (DIRAC_FX64)
    if not args.no_fx64:
        hx = make_grid(D.DIRAC_FX64)
        D.dirac_set_state(hx, dev_state)
        D.dirac_autotune(hx)
        ix = D.dirac_get_info(hx)
        tx, _, _ = timed_device_run(hx, dev_state, args.steps, args.warmup)
        tx = max_over_ranks(tx)
        vx = point_steps / (tx / 1e3)
        fx_final = torch.empty_like(dev_state)
        D.dirac_get_state(hx, fx_final)
        stream.synchronize()
        obs_fx = D.dirac_observables(hx)
        fx_flux = obs_fx["flux_cum"]
        D.dirac_destroy(hx)
        rel = float(torch.linalg.vector_norm(fx_final - fp64_final) / torch.linalg.vector_norm(fp64_final))
        del fx_final
        variants["fx64"] = {
            "value": vx, "unit": "point-steps/s", "ms_per_step": tx / args.steps,
            "steps_per_launch": ix["steps_per_launch"], "points_per_lane": ix["points_per_lane"],
            "fx_shift": ix["fx_shift"], "bytes_per_point_step": FP64_BYTES_PER_POINT_STEP,
            "traffic_per_launch": (MEASURED_TRAFFIC_PER_LAUNCH["fx64"].get((ix["steps_per_launch"], ix["points_per_lane"]))
                                   if args.side == 2048 else None),
            "hbm_frac": FP64_BYTES_PER_POINT_STEP * vx / world / 1e9 / hbm_peak,
            "rel_l2_vs_fp64_after_%d_steps" % args.nsteps: rel,
            "flux_rel_diff_vs_fp64": abs(fx_flux - fp64_flux) / abs(fp64_flux) if fp64_flux else None,
            "norm_drift_vs_fp64": obs_fx["norm"] - fp64_norm, "dT_vs_fp64": (fx_flux - fp64_flux) / n0,
            "speedup_vs_fp64": vx / value,
            "workload": "the headline 2-D Klein run, 64-bit fixed-point storage (exact integer sweeps, phase "
                        "rounded once after a 128-bit product)"}

    # ---------------------------------------------------------------- FP32 storage variant
    if not args.no_fp32:
        h32 = make_grid(D.DIRAC_FP32)
        dev32 = torch.from_numpy(psi0.astype(np.complex64).view(np.float32)).to(f"cuda:{local}")
        torch.cuda.synchronize()
        D.dirac_set_state(h32, dev32)
        D.dirac_autotune(h32)
        i32 = D.dirac_get_info(h32)
        t32, in32, _ = timed_device_run(h32, dev32, args.steps, 1)
        o32 = D.dirac_observables(h32)
        # the state after the timed run is the FP32 state after the full nsteps from psi0: its distance from the
        # FP64 state (bit-exact with the oracle) is the error FP32 storage adds
        fin32 = torch.empty_like(dev32)
        D.dirac_get_state(h32, fin32)
        stream.synchronize()
        fin32 = torch.view_as_real(torch.view_as_complex(fin32.view(-1, 2)).to(torch.complex128)).view(-1)
        rel32 = float(torch.linalg.vector_norm(fin32 - fp64_final.view(-1)) / torch.linalg.vector_norm(fp64_final))
        del fin32
        t32 = max_over_ranks(t32)
        k32 = i32["steps_per_launch"]
        launches32 = args.steps * (args.nsteps // k32 + args.nsteps % k32)
        mean32 = in32 / 1e3 / max(1, launches32)
        v32 = point_steps / (t32 / 1e3)
        eff = FP32_BYTES_PER_POINT_STEP * v32 / world / 1e9
        variants["fp32"] = {"value": v32, "unit": "point-steps/s", "ms_per_step": t32 / args.steps,
                            "steps_per_launch": k32, "points_per_lane": i32["points_per_lane"],
                            "effective_hbm_frac": eff / hbm_peak,
                            "step_kernel_algorithmic_gbs": FP32_BYTES_PER_POINT_STEP * ncell * k32 / mean32 / 1e9,
                            "traffic_per_launch": (MEASURED_TRAFFIC_PER_LAUNCH["fp32"].get((k32, i32["points_per_lane"]))
                                                   if args.side == 2048 else None),
                            "T": o32["flux_cum"] / n0, "T_fp64": fp64_flux / n0,
                            "error_vs_fp64_after_%d_steps" % args.nsteps: {
                                "rel_l2_psi": rel32, "norm_drift": o32["norm"] - fp64_norm,
                                "norm_fp32": o32["norm"], "norm_fp64": fp64_norm,
                                "dT": (o32["flux_cum"] - fp64_flux) / n0}}
        D.dirac_destroy(h32)
        # the same FP32 step at one step per launch (k = 1, P = 2): it moves the full 64 B per point-step, so
        # its HBM fraction is on its own traffic (the k = 2 plan above moves half of that and runs faster)
        c1 = D.make_config((args.side, 1, args.side), x_min=(x_min, 0.0, z_min), flux_face=face,
                           stream=stream.cuda_stream, device=local, precision=D.DIRAC_FP32, steps_per_launch=1,
                           points_per_lane=2)
        h1 = D.dirac_create_grid(c1)
        D.dirac_set_potential(h1, V, D.DIRAC_V_X_ONLY)
        D.dirac_set_state(h1, dev32)
        n1 = 400
        D.dirac_step(h1, 64)  # warm-up
        e10, e11 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e10.record(stream)
        D.dirac_step(h1, n1)
        e11.record(stream)
        stream.synchronize()
        t1 = max_over_ranks(e10.elapsed_time(e11))
        D.dirac_destroy(h1)
        v1 = ncell * n1 * world / (t1 / 1e3)
        variants["fp32_k1"] = {
            "value": v1, "unit": "point-steps/s", "steps": n1, "ms_per_step": t1 / n1, "steps_per_launch": 1,
            "points_per_lane": 2, "bytes_per_point_step": FP32_BYTES_PER_POINT_STEP,
            "hbm_frac": FP32_BYTES_PER_POINT_STEP * v1 / world / 1e9 / hbm_peak,
            "workload": "the 2048^2 Klein grid, FP32 storage, one step per launch (the state read and written "
                        "once per step: 64 B per point-step)"}
    del fp64_final

    # ---------------------------------------------------------------- FP64 with a laser field
    if not args.no_field:
        nf = 400
        hf = make_grid(D.DIRAC_FP64)
        dtf = run.dx / W.C_AU
        D.dirac_set_vector_potential(hf, W.laser_A_tilde(nf * 3, dtf, 2.0e4, 2 * np.pi / (nf * dtf / 2), 2.0,
                                                         pol=(0.8, 0.0, 0.6)))
        D.dirac_set_state(hf, dev_state)
        D.dirac_autotune(hf)
        inf_ = D.dirac_get_info(hf)
        D.dirac_step(hf, nf)  # warm-up (table rows 0..nf-1)
        ef0, ef1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        ef0.record(stream)
        D.dirac_step(hf, nf)
        ef1.record(stream)
        stream.synchronize()
        tf = max_over_ranks(ef0.elapsed_time(ef1))
        D.dirac_destroy(hf)
        vf = ncell * nf * world / (tf / 1e3)
        variants["fp64_laser_field"] = {
            "value": vf, "unit": "point-steps/s", "steps": nf, "steps_per_launch": inf_["steps_per_launch"],
            "points_per_lane": inf_["points_per_lane"],
            "workload": "the 2048^2 Klein FP64 grid in a uniform two-cycle laser pulse (vector potential, full "
                        "phase matrix of Eq. sol_dis_4), %d timed steps" % nf,
            "fp64_instr_per_point_step": FP64_INSTR_PER_POINT_STEP_2D_FIELD,
            "frac_of_fp64_issue_roof": FP64_INSTR_PER_POINT_STEP_2D_FIELD * vf / world / 1e12 / FP64_ISSUE_PEAK_NOMINAL}

    # ---------------------------------------------------------------- 2-D second order and characteristic shifts
    if not args.no_2d_variants:
        legs2 = [("fp64_strang2d", dict(splitting=D.DIRAC_STRANG), 2), ("fp64_shift2", dict(char_shift=2), 2),
                 ("fp64_shift4", dict(char_shift=4), 4)]
        if not args.no_fx64:
            legs2.append(("fx64_strang2d", dict(splitting=D.DIRAC_STRANG, precision=D.DIRAC_FX64), 2))
        for vname, kw, per_step in legs2:
            cfgv = D.make_config((args.side, 1, args.side), x_min=(x_min, 0.0, z_min), flux_face=face,
                                 stream=stream.cuda_stream, device=local, **kw)
            hv = D.dirac_create_grid(cfgv)
            D.dirac_set_potential(hv, V, D.DIRAC_V_X_ONLY)
            D.dirac_set_state(hv, dev_state)
            D.dirac_autotune(hv)
            nv = 400
            D.dirac_step(hv, 64)  # warm-up
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            ev0.record(stream)
            D.dirac_step(hv, nv)
            ev1.record(stream)
            stream.synchronize()
            tv = max_over_ranks(ev0.elapsed_time(ev1))
            iv = D.dirac_get_info(hv)
            D.dirac_destroy(hv)
            vv = ncell * nv * world / (tv / 1e3)
            instr = 80 if vname == "fp64_strang2d" else FP64_INSTR_PER_POINT_STEP_2D  # Strang: 4 sweeps + phase
            if vname.startswith("fx64"):
                variants[vname] = {
                    "value": vv, "unit": "point-steps/s", "steps": nv, "ms_per_step": tv / nv,
                    "physical_time_per_step_dx_over_c": per_step,
                    "first_order_equivalent_point_steps_per_s": vv * per_step,
                    "steps_per_launch": iv["steps_per_launch"], "points_per_lane": iv["points_per_lane"],
                    "workload": "the 2048^2 Klein grid, second-order steps of 2 dx/c, 64-bit fixed-point storage",
                    "hbm_frac": FP64_BYTES_PER_POINT_STEP * vv / world / 1e9 / hbm_peak,
                    "speedup_vs_fp64": (vv / variants["fp64_strang2d"]["value"]) if "fp64_strang2d" in variants else None}
                continue
            variants[vname] = {
                "value": vv, "unit": "point-steps/s", "steps": nv, "ms_per_step": tv / nv,
                "physical_time_per_step_dx_over_c": per_step, "first_order_equivalent_point_steps_per_s": vv * per_step,
                "steps_per_launch": iv["steps_per_launch"], "points_per_lane": iv["points_per_lane"],
                "workload": "the 2048^2 Klein FP64 grid, %s" % ("second-order (Strang) steps of 2 dx/c"
                                                             if vname == "fp64_strang2d" else
                                                             "first-order steps with c dt = %d dx" % per_step),
                "fp64_instr_per_point_step": instr,
                "frac_of_fp64_issue_roof": instr * vv / world / 1e12 / FP64_ISSUE_PEAK_NOMINAL}

    # ---------------------------------------------------------------- 3-D soft-Coulomb grid (first and second order)
    if not args.no_3d:
        n3 = args.side3d
        dx3 = W.DX_DEFAULT
        psi3 = W.gaussian_packet(n3, n3, dx3, -n3 * dx3 / 2, -n3 * dx3 / 2, 32 * dx3, 0.0, 16 * dx3, 0.0, ny=n3,
                                 y_min=-n3 * dx3 / 2)
        V3 = W.soft_coulomb_3d(n3, dx3, 10.0, 2 * dx3).reshape(-1)
        ref3 = {}  # the FP64 states after each leg (warm-up + timed steps): the fixed-point references
        precs3 = [(D.DIRAC_FP64, "fp64"), (D.DIRAC_FP32, "fp32")] + ([] if args.no_fx64 else [(D.DIRAC_FX64, "fx64")])
        for prec, pname in precs3:
            wide = prec != D.DIRAC_FP32  # complex128 in (FP64 and fixed point)
            dev3 = torch.from_numpy(psi3.astype(np.complex128 if wide else np.complex64)
                                    .view(np.float64 if wide else np.float32)).to(f"cuda:{local}")
            for split, sname, per_step in ((D.DIRAC_LIE, "first_order", 1), (D.DIRAC_STRANG, "strang", 4)):
                cfg3 = D.make_config((n3, n3, n3), ndim=3, precision=prec, splitting=split, stream=stream.cuda_stream,
                                     device=local)
                h3 = D.dirac_create_grid(cfg3)
                D.dirac_set_potential(h3, V3, D.DIRAC_V_FULL)
                D.dirac_set_state(h3, dev3)
                D.dirac_autotune(h3)  # fused single pass or x-y + z/phase passes, whichever is faster here
                i3 = D.dirac_get_info(h3)
                n_steps3 = 12 if split == D.DIRAC_LIE else 32
                D.dirac_step(h3, n_steps3)  # warm-up
                e30, e31 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                stream.synchronize()
                e30.record(stream)
                D.dirac_step(h3, n_steps3)
                e31.record(stream)
                stream.synchronize()
                t3 = max_over_ranks(e30.elapsed_time(e31))
                o3 = D.dirac_observables(h3)
                rel3 = None
                if prec != D.DIRAC_FP32:
                    fin = torch.empty_like(dev3)
                    D.dirac_get_state(h3, fin)
                    stream.synchronize()  # the copy runs on the grid's stream; torch reads on its own
                    if prec == D.DIRAC_FP64:
                        ref3[split] = fin
                    elif split in ref3:
                        ref = ref3.pop(split)
                        rel3 = float(torch.linalg.vector_norm(fin - ref) / torch.linalg.vector_norm(ref))
                        del fin, ref
                D.dirac_destroy(h3)
                v3 = n3 ** 3 * n_steps3 * world / (t3 / 1e3)
                instr = 64 if split == D.DIRAC_LIE else 144
                entry = {"value": v3, "unit": "point-steps/s", "steps": n_steps3, "ms_per_step": t3 / n_steps3,
                         "physical_time_per_step_dx_over_c": per_step,
                         "first_order_equivalent_point_steps_per_s": v3 * per_step,
                         "workload": "%d^3 soft-Coulomb grid (Z = 10, per-cell table), %s splitting" % (n3, sname),
                         "steps_per_launch": i3["steps_per_launch"],
                         "plan": {D.DIRAC_PLAN_3D_FUSED: "fused pass, %d step(s) per launch" % i3["steps_per_launch"],
                                  D.DIRAC_PLAN_3D_TWO_PASS: "x-y pass + z/phase pass, P=%d" % i3["points_per_lane"],
                                  D.DIRAC_PLAN_3D_STRANG: "eight single-sweep launches",
                                  D.DIRAC_PLAN_3D_STRANG_ZPASS: "x, y, x single sweeps, one z-phase-z pass, x, y, x "
                                                                "single sweeps",
                                  D.DIRAC_PLAN_3D_STRANG_FUSED: "fused passes: x-y-x, then per step z-phase-z and "
                                                                "x-y-x-x-y-x (the last x-y-x)"}
                                 .get(i3["plan"], str(i3["plan"])),
                         "norm_end": o3["norm"]}
                if prec == D.DIRAC_FP64:
                    entry["fp64_instr_per_point_step"] = instr
                    entry["frac_of_fp64_issue_roof"] = instr * v3 / world / 1e12 / FP64_ISSUE_PEAK_NOMINAL
                elif prec == D.DIRAC_FX64:
                    # algorithmic: the state read and written once plus the per-cell int64 table (32 B); first
                    # order moves that in the fused pass and 2 x 128 + 32 B in its two passes, second order
                    # 8 x 128 + 32 B in its eight single sweeps or about 288 B in its fused passes
                    if split == D.DIRAC_LIE:
                        moved = 160 if i3["plan"] == D.DIRAC_PLAN_3D_FUSED else 288
                    elif i3["plan"] == D.DIRAC_PLAN_3D_STRANG_FUSED:
                        # per step a z-phase-z pass (128 B + the 32 B table) and an x-y pass (128 B), one more x-y
                        # pass per run
                        moved = 160 + 128 * (n_steps3 + 1) / n_steps3
                    else:
                        moved = 8 * 128 + 32
                    entry["bytes_per_point_step"] = 160
                    entry["hbm_frac"] = 160 * v3 / world / 1e9 / hbm_peak
                    entry["pass_bytes_per_point_step"] = moved
                    entry["hbm_frac_of_pass_bytes"] = moved * v3 / world / 1e9 / hbm_peak
                    entry["rel_l2_vs_fp64_after_%d_steps" % (2 * n_steps3)] = rel3
                    ref_name = "fp64_3d_%s" % sname
                    entry["speedup_vs_fp64"] = (v3 / variants[ref_name]["value"]) if ref_name in variants else None
                    entry["workload"] += ", 64-bit fixed-point storage"
                else:
                    # second order: the unfused basis is eight single sweeps (8 x 64 B + the 16 B table); a run
                    # of m fused steps moves m z-phase-z passes (80 B) and m + 1 x-y passes (64 B)
                    bytes3 = 80 if split == D.DIRAC_LIE else 8 * 64 + 16
                    entry["bytes_per_point_step"] = bytes3
                    entry["effective_hbm_frac"] = bytes3 * v3 / world / 1e9 / hbm_peak
                    if i3["plan"] == D.DIRAC_PLAN_3D_STRANG_FUSED:
                        moved = 80 + 64 * (n_steps3 + 1) / n_steps3
                        entry["pass_bytes_per_point_step"] = moved
                        entry["hbm_frac_of_pass_bytes"] = moved * v3 / world / 1e9 / hbm_peak
                variants["%s_3d_%s" % (pname, sname)] = entry
            del dev3
        del ref3

    # ---------------------------------------------------------------- config 3: 384^3 soft Coulomb, 1000 steps, Z sweep
    if not args.no_config3 and not args.no_3d:
        n3 = args.side3d
        dx3 = W.DX_DEFAULT
        zs = [float(z) for z in args.config3_z.split(",") if z.strip()]
        nst = args.config3_steps
        psi3 = W.gaussian_packet(n3, n3, dx3, -n3 * dx3 / 2, -n3 * dx3 / 2, 32 * dx3, 0.0, 16 * dx3, 0.0, ny=n3,
                                 y_min=-n3 * dx3 / 2)
        norm0 = float(np.sum(np.abs(psi3) ** 2) * dx3 ** 3)
        per_z = {("%g" % z): {} for z in zs}
        fp64_states = {}
        timing = {}
        precs = [(D.DIRAC_FP64, "fp64"), (D.DIRAC_FP32, "fp32")] + ([] if args.no_fx64 else [(D.DIRAC_FX64, "fx64")])
        for prec, pname in precs:
            wide = prec != D.DIRAC_FP32
            dev3 = torch.from_numpy(psi3.astype(np.complex128 if wide else np.complex64)
                                    .view(np.float64 if wide else np.float32)).to(f"cuda:{local}")
            h3 = D.dirac_create_grid(D.make_config((n3, n3, n3), ndim=3, precision=prec, stream=stream.cuda_stream,
                                                   device=local))
            ms_total, plan3 = 0.0, None
            for zi, Z in enumerate(zs):
                D.dirac_set_potential(h3, W.soft_coulomb_3d(n3, dx3, Z, 2 * dx3).reshape(-1), D.DIRAC_V_FULL)
                D.dirac_set_state(h3, dev3)
                if zi == 0:
                    D.dirac_autotune(h3)
                    plan3 = D.dirac_get_info(h3)
                ec0, ec1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                stream.synchronize()
                ec0.record(stream)
                D.dirac_step(h3, nst)
                ec1.record(stream)
                stream.synchronize()
                ms_total += ec0.elapsed_time(ec1)
                o3 = D.dirac_observables(h3)
                fin = torch.empty_like(dev3)
                D.dirac_get_state(h3, fin)
                stream.synchronize()
                if not wide:
                    fin = torch.view_as_real(torch.view_as_complex(fin.view(-1, 2)).to(torch.complex128)).view(-1)
                fin = fin.view(-1)
                key = "%g" % Z
                rec = {"norm_end": o3["norm"], "centroid": o3["centroid"]}
                if prec == D.DIRAC_FP64:
                    fp64_states[key] = (fin, o3["norm"])
                    rec["norm_change_from_start"] = o3["norm"] - norm0
                else:
                    ref, ref_norm = fp64_states[key]
                    rec["rel_l2_psi_vs_fp64"] = float(torch.linalg.vector_norm(fin - ref) / torch.linalg.vector_norm(ref))
                    rec["norm_drift_vs_fp64"] = o3["norm"] - ref_norm
                    del fin
                per_z[key][pname] = rec
            D.dirac_destroy(h3)
            del dev3
            timing[pname] = {"value": n3 ** 3 * nst * len(zs) * world / (max_over_ranks(ms_total) / 1e3),
                             "unit": "point-steps/s", "plan": plan3["plan"],
                             "steps_per_launch": plan3["steps_per_launch"], "points_per_lane": plan3["points_per_lane"]}
        del fp64_states
        variants["config3_coulomb%d_%d_steps" % (n3, nst)] = {
            "workload": "%d^3 grid, V = -Z / sqrt(r^2 + (2 dx)^2) centred, spin-up Gaussian width 16 dx at rest "
                        "offset +32 dx in x, zero boundary, %d first-order steps per Z; FP32 storage and 64-bit fixed "
                        "point compared with the FP64 state (bit-exact with the oracle) after the same steps"
                        % (n3, nst),
            "norm_start": norm0, "per_Z": per_z, "rates": timing}

    # ---------------------------------------------------------------- the paper's own 2-D Klein run, FP32
    if args.paper_klein:
        from paper_1107_4650_gb300 import paper_klein2d as PK
        pk = PK.run("fp32", stream=stream, device=local)
        variants["paper_klein2d_fp32"] = {
            "value": pk["point_steps_per_s"] * world, "unit": "point-steps/s", "workload": pk["run"],
            "T_flux": pk["T_flux"], "R_left": pk["R_left"], "paper_T_R": [0.2407, 0.7593],
            "gpu_s": pk["gpu_ms"] / 1e3, "paper_wall_s": 22.0 * 3600.0, "paper_processes": 256}

    # ---------------------------------------------------------------- batched ensemble (FP32)
    if not args.no_batch:
        # independent runs: each rank takes batch_runs of one global draw of batch_runs * world (weak scaling)
        runs, _, deviations = PD.ensemble_shard(args.batch_runs, rank, world)
        bcfg = D.dirac_batch_default_config()
        bcfg.precision = D.DIRAC_FP32
        bcfg.stream = stream.cuda_stream
        bcfg.device = local
        hb = D.dirac_batch_create([r.as_batch_fields() for r in runs], bcfg)
        D.dirac_batch_autotune(hb)
        D.dirac_batch_run(hb)           # warm-up: graph capture and one full pass
        stream.synchronize()
        D.dirac_batch_reset(hb)
        stream.synchronize()
        barrier()
        eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        eb0.record(stream)
        D.dirac_batch_run(hb)
        eb1.record(stream)
        stream.synchronize()
        tb = max_over_ranks(eb0.elapsed_time(eb1))
        bres = D.dirac_batch_results(hb, len(runs))
        binfo = D.dirac_batch_get_info(hb)
        D.dirac_batch_destroy(hb)
        bps = binfo["point_steps"] * world / (tb / 1e3)
        variants["batched_fp32"] = {
            "value": bps, "unit": "point-steps/s", "ms_per_pass": tb, "runs": len(runs),
            "point_steps_per_pass": binfo["point_steps"], "steps_per_launch": binfo["steps_per_launch"],
            "points_per_lane": binfo["points_per_lane"], "segment_rows": binfo["segment_rows"],
            "launches_per_pass": binfo["launches"], "effective_hbm_frac": FP32_BYTES_PER_POINT_STEP * bps / world / 1e9 / hbm_peak,
            "workload": "%d independent 2-D Klein runs, sides %s, 2000-6000 steps, one persistent kernel per "
                        "block of steps, graph-replayed; %d drawn sides raised to hold the packet"
                        % (len(runs), sorted(set(r.side for r in runs)), len(deviations)),
            "T_mean": float(np.mean(bres["T"])), "T_min": float(np.min(bres["T"])), "T_max": float(np.max(bres["T"])),
            "T_lower_bound": -W.packet_mass_right_of_step(),
            "T_lower_bound_note": "T is the net flux through the face over the initial norm; the part of the packet "
                                  "already right of the step (erfc(4/sqrt 2)/2 = 3.2e-5 for a packet 4 widths "
                                  "left of it) can flow back, so T >= -3.2e-5 in the gap where nothing transmits"}

        # the same persistent kernel on an ensemble that keeps its drawn sides 256..1024 (packets narrowed to fit):
        # how the task queue balances grids of uneven size and step count
        runs_u, log_u = W.klein_ensemble_drawn_sides(args.batch_runs, seed=W.SEED + 7 + rank)
        hu = D.dirac_batch_create([r.as_batch_fields() for r in runs_u], bcfg)
        D.dirac_batch_autotune(hu)
        D.dirac_batch_run(hu)
        stream.synchronize()
        D.dirac_batch_reset(hu)
        stream.synchronize()
        barrier()
        eu0, eu1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        eu0.record(stream)
        D.dirac_batch_run(hu)
        eu1.record(stream)
        stream.synchronize()
        tu = max_over_ranks(eu0.elapsed_time(eu1))
        uinfo = D.dirac_batch_get_info(hu)
        D.dirac_batch_destroy(hu)
        ups = uinfo["point_steps"] * world / (tu / 1e3)
        sides_u = [r.side for r in runs_u]
        variants["batched_fp32_drawn_sides"] = {
            "value": ups, "unit": "point-steps/s", "ms_per_pass": tu, "runs": len(runs_u),
            "point_steps_per_pass": uinfo["point_steps"], "steps_per_launch": uinfo["steps_per_launch"],
            "points_per_lane": uinfo["points_per_lane"], "segment_rows": uinfo["segment_rows"],
            "effective_hbm_frac": FP32_BYTES_PER_POINT_STEP * ups / world / 1e9 / hbm_peak,
            "runs_per_side": {str(sd): sides_u.count(sd) for sd in sorted(set(sides_u))},
            "relative_to_raised_sides_ensemble": ups / bps,
            "workload": "%d independent 2-D Klein runs keeping their drawn sides 256..1024 (widths capped to fit: %d "
                        "of them), 16-column layers, 2000-6000 steps: the queue's balance over uneven grids"
                        % (len(runs_u), len(log_u))}

    # ---------------------------------------------------------------- transmission surrogate
    ckpt = os.path.join(ROOT, "paper_1107_4650_gb300", "data", "surrogate_klein_box.npz")
    if not args.no_surrogate and os.path.exists(ckpt):
        z = np.load(ckpt)
        lo, hi = z["lo"], z["hi"]
        hs = D.dirac_surrogate_create(lo, hi, seed=0, max_batch=4096, stream=stream.cuda_stream, device=local)
        D.dirac_surrogate_set_params(hs, z["params"])
        rng = np.random.default_rng(W.SEED + 4)
        qq = lo + (hi - lo) * rng.uniform(0, 1, (4096, 3))
        D.dirac_surrogate_predict(hs, qq)
        t0 = time.perf_counter()
        for _ in range(5):
            D.dirac_surrogate_predict(hs, qq)
        t_net = (time.perf_counter() - t0) / (5 * len(qq))
        qj = qq[:args.check_points]
        T_net = D.dirac_surrogate_predict(hs, qj)
        D.dirac_surrogate_destroy(hs)
        # the same network on 65,536 queries per call (one fused launch of 512 CTAs per call)
        big = 65536
        hb_ = D.dirac_surrogate_create(lo, hi, seed=0, max_batch=big, stream=stream.cuda_stream, device=local)
        D.dirac_surrogate_set_params(hb_, z["params"])
        qb = lo + (hi - lo) * rng.uniform(0, 1, (big, 3))
        D.dirac_surrogate_predict(hb_, qb)
        t0 = time.perf_counter()
        for _ in range(5):
            D.dirac_surrogate_predict(hb_, qb)
        t_big = (time.perf_counter() - t0) / (5 * big)
        D.dirac_surrogate_destroy(hb_)

        def solve(qs, prec):
            cfg_b = D.dirac_batch_default_config()
            cfg_b.precision = prec
            cfg_b.stream = stream.cuda_stream
            cfg_b.device = local
            cfg_b.steps_per_launch = 2
            cfg_b.points_per_lane = 2
            cfg_b.segment_rows = 256
            runs = [D.dirac_klein_run_from_reduced(q, W.DX_DEFAULT, W.C_AU, 1.0) for q in qs]
            t = time.perf_counter()
            T, _ = D.dirac_batch_klein(runs, cfg_b)
            return T, (time.perf_counter() - t) / len(qs)

        T64, t64 = solve(qj, D.DIRAC_FP64)
        dT = np.abs(T_net - T64)
        bq = variants.get("batched_fp32", {})
        t32 = bq["ms_per_pass"] / 1e3 / bq["runs"] if bq else None
        variants["surrogate"] = {
            "queries_per_s_network": 1.0 / t_net, "queries_per_s_network_65536_per_call": 1.0 / t_big,
            "queries_per_call": len(qq), "queries_per_s_fp64_solver": 1.0 / t64,
            "queries_per_s_batched_fp32_solver": (1.0 / t32) if t32 else None,
            "gain_network_over_fp64_solve": t64 / t_net,
            "gain_batched_fp32_over_fp64_solve": (t64 / t32) if t32 else None,
            "checked_points": len(qj), "dT_mean": float(dT.mean()), "dT_p99": float(np.percentile(dT, 99)),
            "dT_max": float(dT.max()),
            "checkpoint": "paper_1107_4650_gb300/data/surrogate_klein_box.npz",
            "box": "V0/mc^2 [%g, %g], p0/mc [%g, %g], width/dx [%g, %g]" % (lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]),
            "training": json.loads(str(z["stats"])) if "stats" in z else None}

    # ---------------------------------------------------------------- CPU baseline (rank 0)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, desc = cpu_baseline(run, args.cpu_seconds)
        cpu = {"value": rate, "unit": "point-steps/s", "cores": cores, "kind": "oracle", "sample": desc}
        if args.cpu_detail_seconds > 0:
            cpu["detail"] = cpu_detail(run, args.cpu_detail_seconds)

    if rank == 0:
        line = {"metric": "4-spinor grid-point-steps/s", "value": value, "unit": "point-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": "2-D Klein step, FP64, %dx%d cells, %d time steps per bench step, V0=2.5 mc^2, "
                                       "L=4 dx, width 100 dx, p0=%.4f mc, flux face %d"
                                       % (args.side, args.side, args.nsteps, run.p0 / W.C_AU, face),
                           "point_steps_per_bench_step": ncell * args.nsteps,
                           "l2": "inputs larger than L2: two 268 MB state buffers ping-pong",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "steps_per_launch": k_launch, "points_per_lane": info["points_per_lane"]},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks, "variants": variants,
                "physics": {"T_flux": obs["flux_cum"] / n0, "norm_end": obs["norm"], "norm_start": n0}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
