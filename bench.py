#!/usr/bin/env python
"""Throughput benchmark of the A-DOT time step on one GB300 (or N replicas).

Workload: the smooth periodic problem on [0, 1] m (h = 1 + 0.1 sin 2 pi x,
u = 0.3 + 0.05 cos 2 pi x, z = 0.1 sin 2 pi x; Grass A_g = 0.005, p = 0.4,
CFL 0.8) at N = 1e7 cells, float32 arithmetic with a float-float state. One
step = one time step over all cells (edge fluctuations, update, CFL maximum),
replayed from a CUDA graph. Metric: cell-updates/s = N * steps / seconds.

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle on
the host cores instead (one step = one oracle time step on a bounded sample of
the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s at N=1e7 (A-DOT FP32 vs surrogate) at L1 err vs FP64 oracle"
UNIT = "cell-updates/s"
# Per-launch counts of the fused step kernel from ncu captures at N = 4e6 (one
# launch = one time step), per kernel shape (kind, threads, register cap); None
# where the kernel changed after its capture or no capture exists.
#  flops: executed FP32 flops per updated cell (2 FFMA + FADD + FMUL thread
#         instructions) of the -DADOT_SCALAR_NODES build (ncu's per-opcode
#         counters skip the paired float32x2 instructions of the default build,
#         which does the same arithmetic); the edges evaluated twice (1 per warp
#         range, 0.09 %) removed;
#  instr: executed thread instructions per cell-update (smsp__inst_executed x 32 / cells);
#  xu:    XU-pipe thread instructions per cell-update (sm__inst_executed_pipe_xu x 32 / cells);
#  dram:  dram__bytes_read.sum + dram__bytes_write.sum per cell-update.
KERNEL_COUNTS = {
    # static ranges over 4/8 of the chunks (assigned across blocks, the split formed on the
    # host) plus the 63-cell work pool: at 4e6 cells and 3648 warps (cap 80), 4,035,698 edges
    # evaluated for 4,000,001 (35,697 evaluated twice, removed); arccos(x)/3 by the library's
    # polynomial form; float64 redo deferred to k_fixup (which the smooth workload never
    # calls); CFL Newton steps skipped below the lane's running maximum. The flop count is the
    # all-scalar build's (the same arithmetic at either register cap).
    ("warp", 256, 80): {"flops": (2 * 443.619368e6 + 333.91313e6 + 547.090924e6) / 4e6
                        * (1 - 35697 / 4e6),
                        "instr": 67.00175e6 * 32 / 4e6, "xu": 3.369332e6 * 32 / 4e6,
                        "dram": (96.802816e6 + 51.708416e6) / 4e6},
    ("warp", 256, 64): {"flops": (2 * 443.619368e6 + 333.91313e6 + 547.090924e6) / 4e6
                        * (1 - 35697 / 4e6),
                        "instr": 67.596198e6 * 32 / 4e6, "xu": 3.388325e6 * 32 / 4e6,
                        "dram": (97.00864e6 + 51.615488e6) / 4e6},
    ("order2", 256, 64): {"flops": None, "instr": None, "xu": None, "dram": None},
}
# The block kernel's all-scalar count (1 edge in 256 evaluated twice, removed).
FLOPS_BLOCK = 498.6
# The algorithmic flop count per cell-update of the planning estimate: three
# Gauss-Legendre nodes of ~130 FP32-pipe instructions each plus ~20 for the
# update and CFL epilogue, ~410 instructions, about 700-800 flops counting an
# FMA as 2; the midpoint is the roofline's primary basis, the executed count
# the second.
FLOPS_PER_CELL_UPDATE_PLAN = 750.0
BYTES_PER_CELL_UPDATE = 48.0  # float-float state: 3 x 8 B read + 3 x 8 B written


def counts(kind: str, block: int, cap: int) -> dict:
    c = KERNEL_COUNTS.get((kind, block, cap), {})
    if kind == "block":
        c = {"flops": FLOPS_BLOCK}
    return c


def issue_roofline(ipc, n: int, per_launch_s: float):
    """The binding term of the FP32 step kernel: instruction issue. Achieved
    thread instructions per second (ncu count per cell-update x cells / live
    launch time) against 152 SMs x 4 schedulers x 32 lanes x 2070 MHz."""
    if not ipc:
        return None
    peak = 152 * 4 * 32 * 2070e6 / 1e12
    achieved = ipc * n / per_launch_s / 1e12
    return {"instr_per_cell_update": ipc, "achieved": achieved, "peak": peak,
            "unit": "T thread-instructions/s", "frac": achieved / peak,
            "peak_source": "152 SM x 4 schedulers x 32 lanes x 2070 MHz (derived)"}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2400)
    ap.add_argument("--warmup", type=int, default=96)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=float, default=1e7, help="cells of the benchmark workload")
    ap.add_argument("--block", type=int, default=0, help="threads per block (0 = autotuned)")
    ap.add_argument("--reg-cap", type=int, default=0, help="64, -1 = none, 0 = autotuned")
    ap.add_argument("--step-kernel", type=int, default=0,
                    help="1 = block kernel, 2 = persistent warp tiles, 0 = autotuned")
    ap.add_argument("--sweep", action="store_true", help="also time every kernel variant")
    ap.add_argument("--cpu-steps", type=int, default=3,
                    help="oracle steps on the full workload for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ensemble-t-end", type=float, default=0.1,
                    help="t_end of the 4096-channel ensemble measurement, a tenth of the "
                         "workload's 1 s (0 = skip)")
    ap.add_argument("--ensemble-channels", type=int, default=4096,
                    help="channels of the ensemble measurement (the first of the seeded 4096)")
    ap.add_argument("--ensemble-form", type=int, default=0,
                    help="step_kernel of the ensemble's main measurement: 0 = chosen per state, "
                         "3 = persistent channel loops, 1/2/4 = per-step launches")
    ap.add_argument("--ensemble-per-step", type=int, default=1,
                    help="also time the per-step form of the ensemble (0 = skip)")
    ap.add_argument("--sur-steps", type=int, default=20000,
                    help="training steps of the |A|_Psi surrogate at batch 65536 (0 = skip the leg)")
    ap.add_argument("--sur-samples", type=int, default=50_000_000,
                    help="edge samples harvested from the smooth, bump and ensemble workloads")
    ap.add_argument("--l1-sweep-kmax", type=int, default=6,
                    help="t_end sweep of the smooth problem at N = 1e3 * 2^k, k <= this (-1 = skip)")
    ap.add_argument("--l1-sweep-oracle-max", type=int, default=4000,
                    help="largest N of the t_end sweep that the CPU oracle also runs")
    ap.add_argument("--config3-steps", type=int, default=480,
                    help="FP32 steps of the 1e6-cell bump workload per transport law (0 = skip)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the pipe-throughput probes")
    ap.add_argument("--friction-steps", type=int, default=960,
                    help="timed steps of the workload with the Strickler friction source (0 = skip)")
    ap.add_argument("--order2-steps", type=int, default=480,
                    help="timed steps of the second-order (MUSCL-Hancock) variant (0 = skip)")
    ap.add_argument("--price-steps", type=int, default=960,
                    help="timed steps of the PRICE-C jump function on the workload (0 = skip)")
    ap.add_argument("--accuracy-steps", type=int, default=96,
                    help="steps of the FP32-vs-FP64 increment check (0 = skip)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1, 0
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return dist, rank, ws, local


def max_over_ranks(value: float, dist, device=None) -> float:
    """Largest value over all ranks (the slowest rank's time); the value itself
    when not distributed. Uses the process group's backend (NCCL on GPUs, gloo
    on CPUs)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist, device=None) -> float:
    """Sum of a per-rank value (work done by every rank); the value itself when
    not distributed."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def min_over_ranks(value: float, dist, device=None) -> float:
    """Smallest per-rank value (e.g. whether every rank's check held)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item())


def oracle_throughput(n: int, steps: int, threads: int | None = None):
    """The FP64 oracle (as it stands) on the smooth periodic workload with n
    cells for `steps` time steps on the host cores. Returns (cell-updates/s,
    seconds, threads)."""
    import oracle as O
    from paper_1912_04791_gb300 import workloads as W
    O.build()
    if threads:
        O.set_num_threads(threads)
    P = W.smooth_periodic(n)
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi), P.bc_left, P.bc_right)
    t0 = time.perf_counter()
    O.run(cfg, P.h, P.q, P.z, max_steps=steps)
    dt = time.perf_counter() - t0
    return n * steps / dt, dt, O.num_threads()


def surrogate_leg(args, adot, W, P, n, stream, dev, local, time_steps, ref64, sweep=None):
    """Harvest edges (float64 labels) from the smooth periodic workload (over its
    convergence sweep's sizes and times to t_end, and at N = 1e6), the
    Gaussian bump and the ensemble, train the MLP at batch 65536, then run the benchmark
    workload with |A|_Psi from the network (analytic fallback near Fr = 1).
    sweep(net), when given, runs while the trained network is alive; its result
    is returned under "_sweep"."""
    import torch
    n_h = int(args.sur_samples)
    X = torch.empty((n_h, 7), dtype=torch.float32, device=dev)
    T = torch.empty((n_h, 9), dtype=torch.float32, device=dev)
    k = 0
    seed = 1000

    def harvest(solver, m, steps_between, parts):
        nonlocal k, seed
        for _ in range(parts):
            take = min(m // parts, n_h - k)
            if take <= 0:
                return
            adot.adot_harvest(solver.ctx, take, seed, X[k:k + take], T[k:k + take])
            k += take
            seed += 1
            solver.step(steps_between)

    t0 = time.perf_counter()
    # the smooth problem over its convergence sweep (N = 1e3 ... 6.4e4), 16 snapshots
    # each spread over [0, t_end): states of every size and time the sweep visits
    sizes = [1000 * 2 ** j for j in range(7)]
    for m in sizes:
        Pm = W.smooth_periodic(m)
        with adot.Solver(adot.config_for(Pm, adot.FP32, device=local), stream=stream) as sm:
            sm.set_state(Pm.h, Pm.q, Pm.z)
            per_snap = int(0.25 * n_h) // (len(sizes) * 16)
            for j in range(16):
                take = min(per_snap, n_h - k)
                adot.adot_harvest(sm.ctx, take, seed, X[k:k + take], T[k:k + take])
                k += take
                seed += 1
                sm.run_to(Pm.t_end * (j + 1) / 16)
    # and at N = 1e6 (early times)
    P2 = W.smooth_periodic(1_000_000)
    with adot.Solver(adot.config_for(P2, adot.FP32, device=local), stream=stream) as s2:
        s2.set_state(P2.h, P2.q, P2.z)
        harvest(s2, int(0.2 * n_h), 3000, 4)
    P3 = W.gaussian_bump(100_000, Ag=0.001)
    with adot.Solver(adot.config_for(P3, adot.FP32, device=local), stream=stream) as s3:
        s3.set_state(P3.h, P3.q, P3.z)
        harvest(s3, int(0.2 * n_h), 3000, 4)
    E = W.riemann_ensemble(64, seed=77, n_min=1000, n_max=100000)
    per_c = (n_h - k) // len(E.n_cells) + 1
    for c in range(len(E.n_cells)):
        h, q, z = E.channel(c)
        cfg = adot.make_config(int(E.n_cells[c]), 0.0, float(E.length[c]), E.cfl, float(E.Ag[c]), E.xi,
                               precision=adot.FP32, device=local)
        with adot.Solver(cfg, stream=stream) as sc:
            sc.set_state(h.copy(), q.copy(), z.copy())
            sc.step(int(E.n_cells[c]) // 20)
            harvest(sc, per_c, 0, 1)
    harvest_s = time.perf_counter() - t0
    with adot.Mlp(65536, stream=stream) as net:
        net.set_params(W.mlp_init())
        net.set_data(X[:k], T[:k])
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hist = net.train(args.sur_steps, 65536, lr=1e-3, seed=4242)
        b.record(stream)
        torch.cuda.synchronize(dev)
        train_ms = a.elapsed_time(b)
        # the same training step on the mma.sync kernels, for comparison (300 steps)
        with adot.Mlp(65536, stream=stream) as net0:
            net0.set_train_engine(1)
            net0.set_params(W.mlp_init())
            net0.set_data(X[:k], T[:k])
            net0.train(20, 65536, lr=1e-3, seed=4243)
            torch.cuda.synchronize(dev)
            a.record(stream)
            net0.train(300, 65536, lr=1e-3, seed=4243)
            b.record(stream)
            torch.cuda.synchronize(dev)
            train_ms_mma = a.elapsed_time(b) / 300
        del X, T
        out = {"samples": k, "harvest_s": harvest_s, "train_steps": args.sur_steps, "batch": 65536,
               "train_engine": "tcgen05",
               "train_ms_per_step": train_ms / max(args.sur_steps, 1),
               "train_flops_per_step": 3 * 2 * 65536 * 51200,
               "loss_first": float(hist[:10].mean()), "loss_last": float(hist[-10:].mean())}
        out["train_tflops"] = out["train_flops_per_step"] / (out["train_ms_per_step"] * 1e-3) / 1e12
        out["train_ms_per_step_mma_sync"] = train_ms_mma
        out["train_tflops_mma_sync"] = out["train_flops_per_step"] / (train_ms_mma * 1e-3) / 1e12
        with adot.Solver(adot.config_for(P, adot.FP32, device=local), stream=stream) as ss:
            ss.set_state(P.h, P.q, P.z)
            adot.adot_set_surrogate(ss.ctx, net, 0.8, 1.2)
            K = ref64[0] if ref64 else 96
            ms_k = time_steps(ss, K)
            got = ss.get_state()
            edges, fb = adot.adot_surrogate_stats(ss.ctx)
            ss.set_state(P.h, P.q, P.z)
            adot.adot_step(ss.ctx, 6)
            ms_t = time_steps(ss, 480)
            # the inference kernel alone (adot_surrogate_eval, no copy-out), per engine:
            # CUDA events on the context's stream around each call, mean of 10 after 2
            infer = {}
            for eng, name in ((0, "tcgen05"), (2, "tcgen05_two_groups"), (1, "mma.sync")):
                net.set_engine(eng)
                ts = []
                for i in range(12):
                    a.record(stream)
                    adot.adot_surrogate_eval(ss.ctx, n + 1, False)
                    b.record(stream)
                    torch.cuda.synchronize(dev)
                    if i >= 2:
                        ts.append(a.elapsed_time(b))
                ms_i = float(np.mean(ts))
                infer[name] = {"ms_per_launch": ms_i, "edges": n + 1,
                               "tflops": (n + 1) * 2 * 51200 / (ms_i * 1e-3) / 1e12}
            # the same steps with the mma.sync inference engine
            net.set_engine(1)
            ss.set_state(P.h, P.q, P.z)
            adot.adot_step(ss.ctx, 6)
            ms_m = time_steps(ss, 480)
            net.set_engine(0)
        peak = measured_peaks().get("bf16_tflops")
        tc = infer["tcgen05"]["tflops"]
        out.update({"cell_updates_per_s": n * 480 / (ms_t * 1e-3), "engine": "tcgen05",
                    "cell_updates_per_s_mma_sync": n * 480 / (ms_m * 1e-3),
                    "infer_flops_per_edge": 2 * 51200, "inference_kernel": infer,
                    "roofline": {"bound": "tensor",
                                 "kernel": "k_mlp_tcp<edges> (tcgen05, bf16, TMEM, warp-specialised)",
                                 "achieved": tc, "peak": peak, "unit": "TFLOP/s",
                                 "frac": tc / peak if peak else None,
                                 "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst; kernel timed alone)"},
                    "fallback_fraction": fb / max(edges, 1)})
        if ref64:
            for name, a_, b_, a0 in zip("hqz", got, ref64[1], (P.h, P.q, P.z)):
                out[f"l1_rel_increment_{name}"] = float(np.abs((a_ - a0) - (b_ - a0)).sum()
                                                        / np.abs(b_ - a0).sum())
                out[f"l1_rel_state_{name}"] = float(np.abs(a_ - b_).sum() / np.abs(b_).sum())
        if sweep is not None:
            out["_sweep"] = sweep(net)
        return out


KS_BENCH = 30.0  # Strickler coefficient of the friction line (s_f ~ 1e-4 on this flow)
FRICTION_FLOPS_PER_CELL = 10.0  # q|q|, 1/h, h^(-1/3), four products, dt scaling, one add


def friction_leg(args, adot, W, P, n, stream, dev, local, time_steps, plain_value, peaks=None):
    """The benchmark workload with the friction source compiled in (the EXT step
    kernels), then the Soni case end to end through the public API."""
    import torch

    K = args.friction_steps
    cfg = adot.config_for(P, adot.FP32, block_threads=args.block, reg_cap=args.reg_cap,
                          step_kernel=args.step_kernel, device=local, ks=KS_BENCH)
    with adot.Solver(cfg, stream=stream) as sf:
        sf.set_state(P.h, P.q, P.z)
        fb, fc, fk = adot.adot_autotune(sf.ctx, 8)
        adot.adot_step(sf.ctx, 48)
        ms = time_steps(sf, K)
    per_launch_s = ms * 1e-3 / K
    kind = "warp" if fk == 2 else "block"
    f_peak = peaks["ffma_tflops"] if peaks else 152 * 128 * 2 * (2070e6) / 1e12
    base = counts(kind, fb, max(fc, 0)).get("flops") or FLOPS_PER_CELL_UPDATE_PLAN
    achieved = (base + FRICTION_FLOPS_PER_CELL) * n / per_launch_s / 1e12
    out = {"workload": f"smooth_periodic N={n} with Strickler friction K_s={KS_BENCH} (FP32)",
           "steps": K, "ms_per_step": ms / K, "cell_updates_per_s": n * K / (ms * 1e-3),
           "vs_frictionless": (n * K / (ms * 1e-3)) / plain_value,
           "kernel": f"{'k_step_warp' if fk == 2 else 'k_step'}<float,GRASS,{fb},{max(fc, 0)},EXT>",
           "roofline": {"bound": "alu", "achieved": achieved, "peak": f_peak, "unit": "TFLOP/s",
                        "frac": achieved / f_peak,
                        "flops_per_cell_update": base + FRICTION_FLOPS_PER_CELL,
                        "flops_basis": "executed count of the frictionless kernel of the same shape "
                                       "(the plan estimate where none) + the source's 10",
                        "hbm_achieved_gbs": BYTES_PER_CELL_UPDATE * n / per_launch_s / 1e9}}
    S = W.soni_aggradation()
    soni = {"case": "Soni aggradation as printed: 100 cells, 2400 s, q_s = 1.45e-3 u^5, K_s = 49.4, "
                    "feed 5 Q_S0 upstream, h0 downstream",
            "paper_cpu_s": {"A-DOT": 1.50, "DOT": 14.97, "PRICE-C": 1.48,
                            "note": "the paper's own CPU times, hardware unstated: context"}}
    for prec_name, prec in (("fp32", adot.FP32), ("fp64", adot.FP64)):
        cfg = adot.config_for(S, prec, law=adot.LAW_POWER, beta=S.extra["beta"], ks=S.extra["ks"],
                              device=local)
        with adot.Solver(cfg, stream=stream) as ss:
            ss.set_state(S.h, S.q, S.z)
            ss.run_to(10.0)  # graph capture and autotuning outside the timed call
            ss.set_state(S.h, S.q, S.z)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ss.run_to(S.t_end)
            h, q, z = ss.get_state()
            wall = time.perf_counter() - t0
            t, steps, _ = ss.query()
        soni[prec_name] = {"wall_s": wall, "steps": int(steps), "t_end": t,
                           "dz_at_feed_m": float(z[0] - S.z[0]), "_z": z,
                           "note": "run_to(2400 s) plus get_state, host wall clock"}
    zs = {k: soni[k].pop("_z") for k in ("fp32", "fp64")}
    soni["fp32_vs_fp64_max_rel_dz"] = float(np.abs(zs["fp32"] - zs["fp64"]).max()
                                            / np.abs(zs["fp64"] - S.z).max())
    out["soni"] = soni
    return out


def order2_leg(args, adot, P, n, stream, local, time_steps, plain_value, acc_steps=96):
    """The benchmark workload with the second-order variant (order = 2), FP32,
    autotuned among its warp-tile variants; its FP32 increment over acc_steps
    steps against the GPU FP64 second-order path."""
    K = args.order2_steps
    cfg = adot.config_for(P, adot.FP32, block_threads=args.block, reg_cap=args.reg_cap,
                          step_kernel=args.step_kernel, device=local, order=2)
    with adot.Solver(cfg, stream=stream) as s2:
        s2.set_state(P.h, P.q, P.z)
        b2, c2, k2 = adot.adot_autotune(s2.ctx, 8)
        adot.adot_step(s2.ctx, 48)
        ms = time_steps(s2, K)
        s2.set_state(P.h, P.q, P.z)
        s2.step(acc_steps)
        got = s2.get_state()
    with adot.Solver(adot.config_for(P, adot.FP64, device=local, order=2), stream=stream) as s64:
        s64.set_state(P.h, P.q, P.z)
        s64.step(acc_steps)
        ref = s64.get_state()
    per_launch_s = ms * 1e-3 / K
    out = {"workload": f"smooth_periodic N={n}, second-order MUSCL-Hancock (FP32)",
           "steps": K, "ms_per_step": ms / K, "cell_updates_per_s": n * K / (ms * 1e-3),
           "vs_first_order": (n * K / (ms * 1e-3)) / plain_value,
           "kernel": f"k_step2_warp<float,GRASS,{b2},{max(c2, 0)}>",
           "hbm_achieved_gbs": BYTES_PER_CELL_UPDATE * n / per_launch_s / 1e9,
           "accuracy": {"steps": acc_steps, "reference": "GPU FP64 second-order path"}}
    ipc = counts("order2", b2, max(c2, 0)).get("instr")
    if ipc:
        out["issue_slots"] = issue_roofline(ipc, n, per_launch_s)
    for name, a, b, a0 in zip("hqz", got, ref, (P.h, P.q, P.z)):
        out["accuracy"][f"l1_rel_increment_{name}"] = float(np.abs((a - a0) - (b - a0)).sum()
                                                            / np.abs(b - a0).sum())
    return out


def price_leg(args, adot, P, n, stream, local, time_steps, plain_value, acc_steps=96):
    """The benchmark workload advanced with the PRICE-C jump function (Sec. 3.2,
    epsilon = 1e-4 as in the paper's Tests 1-2), FP32 float-float state,
    autotuned among its launch shapes; HBM roofline of the step kernel and the
    FP32 increment over acc_steps steps against the GPU FP64 PRICE-C path."""
    K = args.price_steps
    kw = dict(scheme=adot.SCHEME_PRICE_C, price_eps=1e-4, device=local)
    with adot.Solver(adot.config_for(P, adot.FP32, **kw), stream=stream) as sp:
        sp.set_state(P.h, P.q, P.z)
        bp, cp, kp = adot.adot_autotune(sp.ctx, 8)
        adot.adot_step(sp.ctx, 48)
        ms = time_steps(sp, K)
        sp.set_state(P.h, P.q, P.z)
        sp.step(acc_steps)
        got = sp.get_state()
    with adot.Solver(adot.config_for(P, adot.FP64, **kw), stream=stream) as s64:
        s64.set_state(P.h, P.q, P.z)
        s64.step(acc_steps)
        ref = s64.get_state()
    per_launch_s = ms * 1e-3 / K
    hbm = BYTES_PER_CELL_UPDATE * n / per_launch_s / 1e9
    peak = measured_peaks().get("hbm_gbs")
    out = {"workload": f"smooth_periodic N={n}, PRICE-C jump function, eps = 1e-4 (FP32)",
           "steps": K, "ms_per_step": ms / K, "cell_updates_per_s": n * K / (ms * 1e-3),
           "vs_adot": (n * K / (ms * 1e-3)) / plain_value,
           "kernel": f"k_step_warp<float,GRASS,{bp},{max(cp, 0)},0,1> (PRICE-C edge)",
           "roofline": {"bound": "hbm", "achieved": hbm, "peak": peak, "unit": "GB/s",
                        "frac": hbm / peak if peak else None,
                        "bytes_per_cell_update": BYTES_PER_CELL_UPDATE,
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)"},
           "accuracy": {"steps": acc_steps, "reference": "GPU FP64 PRICE-C path"}}
    for name, a, b, a0 in zip("hqz", got, ref, (P.h, P.q, P.z)):
        out["accuracy"][f"l1_rel_increment_{name}"] = float(np.abs((a - a0) - (b - a0)).sum()
                                                            / np.abs(b - a0).sum())
    return out


def measure_pipes(adot, local):
    """Measured throughput of the pipes the step kernels use (library probes,
    CUDA events): FP32 FFMA and paired FFMA2 (TFLOP/s), MUFU rsqrt, sine, float32
    tanh and paired bf16 tanh (T ops/s), FP64 DFMA (TFLOP/s)."""
    out = {}
    for kind, name in ((adot.PIPE_FFMA, "ffma_tflops"), (adot.PIPE_FFMA2, "ffma2_tflops"),
                       (adot.PIPE_RSQ, "mufu_rsq_tops"), (adot.PIPE_SIN, "mufu_sin_tops"),
                       (adot.PIPE_TANH, "mufu_tanh_tops"),
                       (adot.PIPE_TANH_BF16X2, "mufu_tanh_bf16x2_tops"),
                       (adot.PIPE_DFMA, "dfma_tflops")):
        rate, sec = adot.adot_measure_pipe(kind, local)
        out[name] = rate / 1e12
    out["how"] = ("adot_measure_pipe: 8 blocks x 256 threads per SM, 8 independent chains per "
                  "thread, one timed launch after a warm-up, CUDA events")
    return out


def config3_leg(args, adot, W, stream, local, time_steps):
    """Trans-critical flow over the Gaussian bump at N = 1e6 (inflow q = 0.6,
    outflow h = 0.33): a fixed-bed spin-up on the GPU (FP64, 1e4 cells, to
    t = 6 s) prolonged to 1e6 cells, then K steps in FP32 with the fixed bed
    (coalescing roots at Fr = 1, float64 redo), Grass A_g = 0.001 and MPM:
    cell-updates/s, the share of quadrature nodes redone in float64, and the
    FP32 increment against the GPU FP64 path over the same steps."""
    K = args.config3_steps
    P0 = W.gaussian_bump(10_000, Ag=0.0)
    with adot.Solver(adot.config_for(P0, adot.FP64, device=local), stream=stream) as s0:
        s0.set_state(P0.h, P0.q, P0.z)
        s0.run_to(6.0)
        h0, q0, _ = s0.get_state()
    mpm = dict(law=adot.LAW_MPM, s_rel=2.65, d50=1e-3, manning_n=0.02)
    out = {"workload": "Gaussian bump N=1e6, fixed-bed spin-up (1e4 cells, FP64, 6 s) prolonged, "
                       "then FP32 steps", "steps": K}
    for name, Ag, kw in (("fixed_bed", 0.0, {}), ("grass", 0.001, {}), ("mpm", 0.001, mpm)):
        P = W.gaussian_bump_prolonged(h0, q0, 1_000_000, Ag=Ag)
        with adot.Solver(adot.config_for(P, adot.FP32, device=local, **kw), stream=stream) as sf:
            sf.set_state(P.h, P.q, P.z)
            nodes, redo = adot.adot_precision_stats(sf.ctx)
            b, c, k = adot.adot_autotune(sf.ctx, 8)
            sf.set_state(P.h, P.q, P.z)
            sf.step(K)
            got = sf.get_state()
            sf.set_state(P.h, P.q, P.z)
            ms = time_steps(sf, K)
        with adot.Solver(adot.config_for(P, adot.FP64, device=local, **kw), stream=stream) as s64:
            s64.set_state(P.h, P.q, P.z)
            s64.step(K)
            ref = s64.get_state()
        r = {"cell_updates_per_s": P.n * K / (ms * 1e-3), "ms_per_step": ms / K,
             "kernel": f"{'k_step_warp' if k == 2 else 'k_step'}<float,{'MPM' if kw else 'GRASS'},{b},{max(c, 0)}>",
             "fp64_redo_nodes": redo, "nodes": nodes, "fp64_redo_fraction": redo / nodes}
        for v, a, bb, a0 in zip("hqz", got, ref, (P.h, P.q, P.z)):
            if name == "fixed_bed" and v == "z":  # the bed stays: its motion is rounding only
                r["max_abs_bed_motion_fp32"] = float(np.abs(a - a0).max())
                r["max_abs_bed_motion_fp64"] = float(np.abs(bb - a0).max())
                continue
            r[f"l1_rel_increment_{v}"] = float(np.abs((a - a0) - (bb - a0)).sum()
                                               / np.abs(bb - a0).sum())
        out[name] = r
    return out


def soni_oracle_time(W):
    """The Soni case (100 cells, 2400 s) run by the FP64 oracle on one host core."""
    import oracle as O

    S = W.soni_aggradation()
    law = O.power(S.Ag, S.extra["beta"], xi=S.xi, g=S.g)
    cfg = O.make_cfg(S.n, S.x_min, S.x_max, S.cfl, law, S.bc_left, S.bc_right, S.bcl, S.bcr,
                     ks=S.extra["ks"])
    thr = O.num_threads()
    O.set_num_threads(1)
    t0 = time.perf_counter()
    _, _, z, _, steps, _ = O.run(cfg, S.h, S.q, S.z, t_end=S.t_end)
    wall = time.perf_counter() - t0
    O.set_num_threads(thr)
    return {"wall_s": wall, "steps": int(steps), "cores": 1, "dz_at_feed_m": float(z[0] - S.z[0])}


def l1_sweep(adot, W, stream, local, k_max=8, n_oracle_max=32000, net=None):
    """Full-t_end errors on the smooth periodic problem: FP32 (and, with a
    trained network, the surrogate form) vs the GPU FP64 path (itself
    parity-tested against the oracle) for N = 1e3 * 2^k, k <= k_max, and GPU
    FP64 / FP32 vs the CPU oracle for N <= n_oracle_max."""
    import oracle as O
    rows = []
    for k in range(k_max + 1):
        n = 1000 * 2 ** k
        P = W.smooth_periodic(n)
        res = {"n": n}
        states = {}
        forms = [("fp64", adot.FP64), ("fp32", adot.FP32)] + ([("surrogate", adot.FP32)] if net else [])
        for name, prec in forms:
            with adot.Solver(adot.config_for(P, prec, device=local), stream=stream) as s:
                s.set_state(P.h, P.q, P.z)
                if name == "surrogate":
                    adot.adot_set_surrogate(s.ctx, net, 0.8, 1.2)
                t0 = time.perf_counter()
                s.run_to(P.t_end)
                res[f"{name}_seconds"] = time.perf_counter() - t0
                _, steps, _ = s.query()
                res[f"{name}_steps"] = steps
                states[name] = s.get_state()
                if name == "surrogate":
                    edges, fb = adot.adot_surrogate_stats(s.ctx)
                    res["surrogate_fallback_fraction"] = fb / max(edges, 1)
        for v, a, b in zip("hqz", states["fp32"], states["fp64"]):
            res[f"l1_fp32_vs_fp64_{v}"] = float(np.abs(a - b).sum() / np.abs(b).sum())
        if net:
            for v, a, b in zip("hqz", states["surrogate"], states["fp64"]):
                res[f"l1_surrogate_vs_fp64_{v}"] = float(np.abs(a - b).sum() / np.abs(b).sum())
        if n <= n_oracle_max:
            cfg = O.make_cfg(n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi), P.bc_left, P.bc_right)
            t0 = time.perf_counter()
            ho, qo, zo, _, so, _ = O.run(cfg, P.h, P.q, P.z, t_end=P.t_end)
            res["oracle_seconds"] = time.perf_counter() - t0
            res["oracle_steps"] = so
            for name in ("fp64", "fp32"):
                res[f"l1_{name}_vs_oracle"] = max(float(np.abs(a - b).sum() / np.abs(b).sum())
                                                  for a, b in zip(states[name], (ho, qo, zo)))
        rows.append(res)
    return rows


def run_reference(args, rank, ws):
    """Reference arm: the FP64 CPU oracle, each step one oracle time step on a
    sample of the workload sized so that warmup + steps end within ~3 min."""
    if rank != 0:
        return
    import oracle as O
    from paper_1912_04791_gb300 import workloads as W
    O.build()
    n_full = int(args.cells)
    # calibrate the per-cell cost on a small grid
    rate, _, thr = oracle_throughput(100_000, 2)
    budget = 150.0  # seconds for warmup + timed steps
    n_s = int(min(n_full, max(1000, budget * rate / max(1, args.steps + args.warmup))))
    P = W.smooth_periodic(n_s)
    cfg = O.make_cfg(P.n, P.x_min, P.x_max, P.cfl, O.grass(P.Ag, xi=P.xi), P.bc_left, P.bc_right)
    h, q, z, *_ = O.run(cfg, P.h, P.q, P.z, max_steps=args.warmup)
    t0 = time.perf_counter()
    O.run(cfg, h, q, z, max_steps=args.steps)
    sec = time.perf_counter() - t0
    value = n_s * args.steps / sec
    sample = f"{n_s} cells of the N={n_full} smooth periodic workload (same initial data), one oracle time step per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"smooth_periodic N={n_full} (oracle sample)", "n_cells": n_s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    dist, rank, ws, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws)
        if dist:
            dist.destroy_process_group()
        return

    import torch

    from paper_1912_04791_gb300 import adot
    from paper_1912_04791_gb300 import build as B
    from paper_1912_04791_gb300 import workloads as W

    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = int(args.cells)
    P = W.smooth_periodic(n)
    stream = torch.cuda.Stream(device=dev)
    cfg = adot.config_for(P, adot.FP32, block_threads=args.block, reg_cap=args.reg_cap,
                          step_kernel=args.step_kernel, device=local)
    solver = adot.Solver(cfg, stream=stream)
    solver.set_state(P.h, P.q, P.z)
    block, reg_cap, kern = adot.adot_autotune(solver.ctx, 8)

    def time_steps(s, k):
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        adot.adot_enqueue_steps(s.ctx, k)
        b.record(stream)
        torch.cuda.synchronize(dev)
        adot.adot_query(s.ctx)
        return a.elapsed_time(b)

    variants = None
    if args.sweep and rank == 0:
        variants = {}
        for vb, vc, vk in [(128, 64, 1), (128, -1, 1), (256, 64, 1), (256, -1, 1), (512, 64, 1),
                           (512, -1, 1), (256, 64, 2), (128, 64, 2), (128, 72, 2), (256, 80, 2)]:
            with adot.Solver(adot.config_for(P, adot.FP32, block_threads=vb, reg_cap=vc,
                                             step_kernel=vk, device=local), stream=stream) as sv:
                sv.set_state(P.h, P.q, P.z)
                adot.adot_step(sv.ctx, 48)
                ms_v = time_steps(sv, 480)
            name = f"{'warp' if vk == 2 else 'block'}{vb}x{'cap%d' % vc if vc > 0 else 'nocap'}"
            variants[name] = n * 480 / (ms_v * 1e-3)

    # warm-up
    adot.adot_step(solver.ctx, args.warmup)

    # timed region: K graph-replayed steps, CUDA events on the launching stream
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    adot.adot_enqueue_steps(solver.ctx, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    t_sim, steps_done, dt_last = adot.adot_query(solver.ctx)  # raises on a device error
    ms = max_over_ranks(ms, dist, dev)
    value = ws * n * args.steps / (ms * 1e-3)
    per_launch_s = ms * 1e-3 / args.steps

    # end to end through the public API with pinned host buffers:
    # set_state (H2D) + K steps + get_state (D2H)
    e2e = None
    if not args.no_e2e:
        hin = [torch.from_numpy(a).pin_memory() for a in (P.h, P.q, P.z)]
        hout = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(3)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        adot.adot_set_state(solver.ctx, *hin)
        adot.adot_enqueue_steps(solver.ctx, args.steps)
        adot.adot_get_state(solver.ctx, *hout)
        sec = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": ws * n * args.steps / sec, "unit": UNIT,
               "h2d_bytes_per_step": 3 * 8 * n / args.steps,
               "d2h_bytes_per_step": 3 * 8 * n / args.steps,
               "note": f"per call: set_state of 3x{n} float64 from pinned host, {args.steps} steps, get_state to pinned host"}

    # accuracy: FP32 increment vs the GPU FP64 path over the same steps
    accuracy = None
    ref64 = None
    if args.accuracy_steps > 0 and rank == 0:
        K = args.accuracy_steps
        with adot.Solver(adot.config_for(P, adot.FP64, device=local), stream=stream) as s64:
            s64.set_state(P.h, P.q, P.z)
            ms64 = time_steps(s64, K)
            ref = s64.get_state()
            ref64 = (K, ref)
        solver.set_state(P.h, P.q, P.z)
        solver.step(K)
        got = solver.get_state()
        accuracy = {"steps": K, "reference": "GPU FP64 path (parity-tested against the oracle)",
                    "fp64_cell_updates_per_s": n * K / (ms64 * 1e-3)}
        for name, a, b, a0 in zip("hqz", got, ref, (P.h, P.q, P.z)):
            accuracy[f"l1_rel_increment_{name}"] = float(np.abs((a - a0) - (b - a0)).sum()
                                                         / np.abs(b - a0).sum())
            accuracy[f"l1_rel_state_{name}"] = float(np.abs(a - b).sum() / np.abs(b).sum())

    # measured peaks of the FP32, MUFU and FP64 pipes (the ALU rooflines' denominators)
    peaks = None
    if rank == 0 and not args.no_peaks:
        peaks = measure_pipes(adot, local)

    # batched ensemble: 4096 movable-bed Riemann channels, N_c log-uniform in [1e3, 1e5];
    # with N ranks each runs its shard of the channels (no data moves between ranks):
    # the time is the slowest rank's, the cell-updates the sum over ranks
    ensemble = None
    if args.ensemble_t_end > 0:
        E = W.riemann_ensemble(4096)
        if args.ensemble_channels < 4096:
            E = W.Ensemble(E.n_cells[:args.ensemble_channels].copy(), E.length[:args.ensemble_channels].copy(),
                           E.Ag[:args.ensemble_channels].copy(), *(v[:E.offsets[args.ensemble_channels]].copy()
                                                                   for v in (E.h, E.q, E.z)))
        total_cells = int(E.n_cells.sum())
        n_channels = len(E.n_cells)
        if ws > 1:
            E = W.shard_ensemble(E, rank, ws)
        forms = [args.ensemble_form] + ([4] if args.ensemble_per_step and args.ensemble_form != 4 else [])
        runs = {}
        for form_k in forms:
            with adot.Ensemble.from_workload(E, adot.FP32, device=local, stream=stream,
                                             step_kernel=form_k) as ens:
                ens.set_state(E.h, E.q, E.z)
                blk, n_tiles, grid, ens_kernel = ens.info()
                plan = ens.plan(0)
                torch.cuda.synchronize(dev)
                if dist is not None:
                    dist.barrier()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                launches = ens.run_to(args.ensemble_t_end)
                b.record(stream)
                torch.cuda.synchronize(dev)
                t_c, steps_c, cu = ens.query()
                ms_e = a.elapsed_time(b)
            all_at = bool((t_c == args.ensemble_t_end).all())
            sec = max_over_ranks(ms_e * 1e-3, dist, device=dev)
            cu_all = sum_over_ranks(float(cu), dist, device=dev)
            all_at = min_over_ranks(1.0 if all_at else 0.0, dist, device=dev) == 1.0
            name = {1: "per-step block tiles", 2: "per-step warp tiles",
                    3: "persistent channel loops"}[ens_kernel]
            runs[form_k] = {"form": name, "cell_updates": int(cu_all), "seconds": sec,
                          "cell_updates_per_s": cu_all / sec, "launches": int(launches),
                          "max_steps": int(max_over_ranks(float(steps_c.max()), dist, device=dev)),
                          "min_steps": int(min_over_ranks(float(steps_c.min()), dist, device=dev)),
                          "threads_per_block": blk,
                          ("channels" if ens_kernel == 3 else "tiles"): n_tiles, "grid": plan["grid"],
                          "cluster_team": plan["cluster"], "channels_on_teams": plan["teamed"],
                          "estimated_imbalance": plan["imbalance"], "all_at_t_end": all_at}
        ensemble = {"workload": f"{n_channels} movable-bed Riemann channels, N_c log-uniform [1e3,1e5], FP32",
                    "total_cells": total_cells, "t_end": args.ensemble_t_end,
                    "ranks": ws, "sharding": "channels split over the ranks by list scheduling of "
                                             "N_c^2/length_c, no collective" if ws > 1 else None,
                    **runs[args.ensemble_form]}
        if 4 in runs and args.ensemble_form != 4:
            ensemble["other_form"] = runs[4]

    # Strickler friction source (Sec. 2) on the benchmark workload, and the Soni
    # aggradation case (Sec. 5.1: friction, sediment feed, q_s = alpha u^5) as printed
    friction = None
    if args.friction_steps > 0 and rank == 0:
        friction = friction_leg(args, adot, W, P, n, stream, dev, local, time_steps, value, peaks)

    # second-order MUSCL-Hancock variant on the benchmark workload
    order2 = None
    if args.order2_steps > 0 and rank == 0:
        order2 = order2_leg(args, adot, P, n, stream, local, time_steps, value)

    # PRICE-C jump function (the paper's centred comparison scheme) on the same workload
    price = None
    if args.price_steps > 0 and rank == 0:
        price = price_leg(args, adot, P, n, stream, local, time_steps, value)

    # trans-critical bump at N = 1e6: fixed bed, Grass and MPM
    config3 = None
    if args.config3_steps > 0 and rank == 0:
        config3 = config3_leg(args, adot, W, stream, local, time_steps)

    # t_end errors of the smooth problem over a bounded size sweep (with the
    # trained surrogate when its leg runs)
    sweep_fn = None
    if args.l1_sweep_kmax >= 0 and rank == 0:
        def sweep_fn(net):
            return l1_sweep(adot, W, stream, local, args.l1_sweep_kmax, args.l1_sweep_oracle_max, net)

    # learned |A|_Psi surrogate: harvest, train, then drive the benchmark workload
    surrogate = None
    if args.sur_steps > 0 and rank == 0:
        surrogate = surrogate_leg(args, adot, W, P, n, stream, dev, local, time_steps, ref64, sweep_fn)
    sweep = surrogate.pop("_sweep", None) if surrogate else None
    if sweep is None and sweep_fn is not None:
        sweep = sweep_fn(None)


    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, sec, thr = oracle_throughput(n, args.cpu_steps)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"{args.cpu_steps} oracle time steps of the full N={n} workload ({sec:.1f} s)"}
        if friction is not None:
            cpu["soni"] = soni_oracle_time(W)

    solver.close()
    if rank == 0:
        f_derived = 152 * 128 * 2 * (2070e6) / 1e12  # FP32 FMA peak at the maximum SM clock, TFLOP/s
        f_peak = peaks["ffma_tflops"] if peaks else f_derived
        kind = "warp" if kern == 2 else "block"
        kc = counts(kind, block, max(reg_cap, 0))
        achieved = FLOPS_PER_CELL_UPDATE_PLAN * n / per_launch_s / 1e12
        achieved_exec = kc["flops"] * n / per_launch_s / 1e12 if kc.get("flops") else None
        xu = None
        if peaks and kc.get("xu"):
            xr = kc["xu"] * n / per_launch_s / 1e12
            xu = {"ops_per_cell_update": kc["xu"], "achieved": xr,
                  "peak": peaks["mufu_rsq_tops"], "unit": "T ops/s", "frac": xr / peaks["mufu_rsq_tops"],
                  "note": "XU-pipe thread instructions (ncu sm__inst_executed_pipe_xu x 32 / cells) "
                          "over the measured MUFU rsqrt rate"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"smooth_periodic N={n} (A-DOT FP32, float-float state)",
                       "n_cells": n, "domain": "[0,1] m periodic", "Ag": P.Ag, "xi": P.xi,
                       "cfl": P.cfl, "block_threads": block, "reg_cap": reg_cap,
                       "step_kernel": "warp tiles" if kern == 2 else "block",
                       "steps_per_graph": 48,
                       "l2": "inputs larger than L2 (2 x 240 MB state buffers, no flush)",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": f_peak, "unit": "TFLOP/s",
                         "frac": achieved / f_peak,
                         "flops_per_cell_update": FLOPS_PER_CELL_UPDATE_PLAN,
                         "flops_basis": "planning estimate: 3 nodes x ~130 FP32-pipe instructions + "
                                        "~20, 700-800 flops with FMA = 2 (midpoint)",
                         "achieved_executed": achieved_exec,
                         "frac_executed": achieved_exec / f_peak if achieved_exec else None,
                         "flops_per_cell_update_executed": kc.get("flops"),
                         "executed_basis": "ncu FFMA x 2 + FADD + FMUL thread instructions of the "
                                           "-DADOT_SCALAR_NODES build per updated cell",
                         "traffic": kc["dram"] * n if kc.get("dram") else None,
                         "traffic_note": "ncu dram read+write of one launch at N=4e6, scaled to N",
                         "kernel": f"{'k_step_warp' if kern == 2 else 'k_step'}<float,GRASS,{block},{max(reg_cap, 0)}>",
                         "peak_source": ("measured: adot_measure_pipe FFMA (peaks.ffma_tflops)" if peaks
                                         else "152 SM x 128 FP32 lanes x 2 x 2070 MHz (derived)"),
                         "peak_derived": f_derived, "xu": xu,
                         "hbm_achieved_gbs": BYTES_PER_CELL_UPDATE * n / per_launch_s / 1e9,
                         "hbm_peak_gbs": measured_peaks().get("hbm_gbs", 6800.0),
                         "issue_slots": issue_roofline(kc.get("instr"), n, per_launch_s)},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps * (2 if kern == 2 else 1), "clocks": clocks,
            "accuracy": accuracy, "sim_time_after_timed_steps": t_sim, "variants": variants,
            "ensemble": ensemble, "surrogate": surrogate, "friction": friction, "order2": order2,
            "price_c": price, "config3": config3, "peaks": peaks,
            "l1_t_end_sweep": sweep,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
