#!/usr/bin/env python3
"""Benchmark: RandNet-Parareal time-to-solution on GB300.

One *step* is one full solve (Alg. 1: k = 0 coarse sweep, then iterations
of the parallel fine step, dataset append + features, exact leftmost slice,
sequential RandNet predictor-corrector sweep and the Eq. 5 stopping rule)
of the 2D diffusion-reaction workload: 128 x 128 x 2 periodic grid
(d = 32768), N = 64 slices on [0, 5], F = RK4 2000 steps/slice, G = forward
Euler 8 steps/slice, M = 100 ReLU features, m = 4 neighbours, lambda = 1e-7,
tol = 1e-6, initial state i.i.d. N(0,1) (seeded, synthetic).  The timed
form is the mixed-precision fused path (FP32 stencils on a compensated state,
random features from BF16 operands with FP32 accumulation on the tensor
cores, FP64 ridge, correction and norm); the plain FP64 GPU form is timed
beside it.

value = fine cell-updates per second over the whole job (sum over ranks of
the fine RK4 unknown-steps the solves performed / max over ranks of the
timed wall time).  ms_per_step = time-to-solution of one solve.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank solves its own seeded replica (weak scaling, no
collective on the data path); only the barrier and the max-reduction of the
timings cross ranks.  ``--impl reference`` times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOAD = "diffreact2d"  # the benchmark workload; --workload measures the others
METRIC = ("Parareal time-to-solution @tol 1e-6 vs plain FP64; cell-updates/s, %HBM; "
          "p50/p99")
UNIT = "cell-updates/s"

# Algorithmic FP32 flops per fine cell-update (one unknown, one RK4 step),
# counted from the right-hand side formulas with every multiply and add
# separate, plus 13 per unknown for the four stage combinations:
#   diffusion-reaction 2D: per grid point and stage 16 (u) + 12 (v)
#   Brusselator 2D: 16 (u) + 13 (v); 3D: 21 (u) + 18 (v)
#   Burgers 1D: 9 per point and stage
#   shallow water: 39 per Rusanov face (4 divisions, 2 square roots, the
#   two physical fluxes, speeds, the maximum, 3 x 5 for the face flux) x 4
#   faces + 15 for the flux differences = 171 per grid point and stage
FLOPS_PER_CELL_UPDATE = {"diffreact2d": (4 * (16 + 12) + 2 * 13) / 2.0,
                         "bruss2d": (4 * (16 + 13) + 2 * 13) / 2.0,
                         "bruss3d": (4 * (21 + 18) + 2 * 13) / 2.0,
                         "burgers1d": 4 * 9 + 13.0,
                         "swe_box": (4 * 171 + 3 * 13) / 3.0}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one fine launch
# over all 64 slices of the diffusion-reaction workload, per tiling (cluster,
# threads, PX, RS), from the ncu captures summarised in
# profiles/k_stencil_mixed_diffreact2d_128x128_N64.md; valid only for the
# captured kernels, scaled by the slices a launch runs (the kernel reads each
# start state once; its results stay in L2).
STENCIL_TRAFFIC = {"workload": "diffreact2d", "slices": 64,
                   "bytes": {(8, 256, 2, 4): 16828416, (16, 128, 2, 4): 17310976}}


def traffic_per_launch(tf: dict, slices: float):
    t = STENCIL_TRAFFIC
    key = (tf["cluster"], tf["threads"], tf["px"], tf["rs"])
    if WORKLOAD != t["workload"] or key not in t["bytes"]:
        return None
    return t["bytes"][key] * slices / t["slices"]


def peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path))
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0,
            "fallback": True}


def fp32_alu_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    # 128 FP32 lanes per SM, an FMA counted as 2 flops
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"rnp_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def describe(cfg: dict) -> str:
    grid = "x".join(str(v) for v in (cfg["nx"], cfg["ny"], cfg["nz"]) if v > 1)
    bc = "walls" if cfg.get("bc", "periodic") == "neumann" else "periodic"
    fs = cfg.get("fscheme", "rk4").upper()
    return (f"{cfg['pde']} {grid}x{W.ncomp(cfg)} {bc}, N={cfg['N']}, "
            f"F={fs}x{cfg['nF']}, G=Eulerx{cfg['nG']}, M={cfg['M']}, m={cfg['m']}, "
            f"tol={cfg['tol']}, batch={cfg.get('batch', 1)}, max_iters={cfg['max_iters']}")


def replica_seed(rank: int) -> int:
    """Seed of the replica a rank solves (weak scaling: one solve per rank)."""
    return W.CONFIGS[WORKLOAD]["seed"] + 1000 * rank


def aggregate(t_local: float, work_local: float, dist=None, device=None):
    """Whole-job (time, work): the max over ranks of the timed seconds and the
    sum over ranks of the work; no other cross-rank traffic."""
    if dist is None:
        return t_local, work_local
    import torch
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    ww = torch.tensor([work_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(ww, op=dist.ReduceOp.SUM)
    return tt.item(), ww.item()


def cpu_baseline(seconds_hint: float = 20.0) -> dict:
    """The FP64 oracle on the host cores: a bounded sample of the same
    workload (same grid, slices and coarse solver; nF cut to 1000 of 2000
    fine steps per slice: about 12 s on 16 cores), reported in fine
    cell-updates per second."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    full = W.config(WORKLOAD)
    cfg = W.config(WORKLOAD, nF=min(1000, full["nF"]))
    p = oracle.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    t0 = time.perf_counter()
    rc, U, st, _ = oracle.solve(p, u0)
    dt = time.perf_counter() - t0
    grid = "x".join(str(v) for v in (cfg["nx"], cfg["ny"], cfg["nz"]) if v > 1)
    return {"value": st.fine_cell_updates / dt, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": (f"{WORKLOAD} {grid}x{W.ncomp(cfg)}, N={cfg['N']}, nF={cfg['nF']} of "
                       f"{full['nF']} RK4 steps per slice, full solve K={st.K} in {dt:.2f} s, "
                       f"FP64, slice-parallel over {cores} threads")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    full = W.config(WORKLOAD)
    cfg = W.config(WORKLOAD, nF=min(1000, full["nF"]))   # the cpu_baseline sample
    samples = []
    base = None
    for i in range(args.warmup + args.steps):
        b = cpu_baseline()
        if i >= args.warmup:
            samples.append(b["value"])
        base = b
    value = statistics.median(samples) if samples else base["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{describe(cfg)} (CPU sample: nF={cfg['nF']} of {full['nF']})",
                   "grid": "x".join(str(v) for v in (cfg["nx"], cfg["ny"], cfg["nz"]) if v > 1)
                   + f"x{W.ncomp(cfg)}", "N": cfg["N"], "nF": cfg["nF"], "nG": cfg["nG"]},
        "cpu_baseline": {"kind": "oracle", "cores": base["cores"], "sample": base["sample"],
                         "value": value, "unit": UNIT},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    import paper_2411_06225_gb300 as rnp
    global WORKLOAD
    WORKLOAD = args.workload
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rnp.lib()
    cfg = W.config(WORKLOAD, seed=replica_seed(rank))
    if args.max_iters:
        cfg["max_iters"] = args.max_iters
    d = W.dim(cfg)
    N = cfg["N"]
    u0_h = torch.as_tensor(W.initial_condition(cfg)).pin_memory()
    u0 = u0_h.to(dev)
    stream = torch.cuda.current_stream(dev)
    if args.tile:
        # a fixed stencil tiling (cluster, threads), e.g. to profile one
        # configuration: the autotuner's pick can differ under a profiler
        c_, t_ = (int(x) for x in args.tile.split(","))
        prob = rnp.problem(cfg, precision=args.precision, exec="fused", autotune=0,
                           cluster=c_, threads=t_)
    else:
        prob = rnp.problem(cfg, precision=args.precision, exec="fused", autotune=1)
    solver = rnp.Solver(prob, stream=stream)
    tiling = {"fine": solver.stencil_config("fine"), "coarse": solver.stencil_config("coarse")}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    for _ in range(args.warmup):
        solver.solve(u0)
    if args.profile:
        # the fine step and the batched feature map of the timed form, one each
        U0 = solver.coarse_sweep(0, u0)
        starts = U0[:, :N].contiguous()
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_push("rnp_fine")
        solver.fine_batch(starts)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
        torch.cuda.nvtx.range_push("rnp_features")
        solver.features(starts[0])
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
        solver.reset()
        torch.cuda.nvtx.range_push("rnp_solve")
        solver.solve(u0)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
        solver.close()
        print(json.dumps({"profile": "done", "precision": args.precision, "tiling": tiling}))
        return 0

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = local
    clocks = ClockSampler(gpu_id)
    tts, fine_ms, cells, launches, stats = [], [], 0, 0, None
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    clocks.start()
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)                       # L2 flush between timed steps (untimed)
        ev0.record(stream)
        U, st = solver.solve(u0)
        ev1.record(stream)
        ev1.synchronize()
        tts.append(ev0.elapsed_time(ev1))
        fine_ms.append(st["t_fine_ms"] / max(st["K"], 1))
        cells += st["fine_cell_updates"]
        launches += st["kernel_launches"]
        stats = st
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    t_sum = sum(tts) / 1e3
    # max over ranks of the timed device time, sum of the work
    t_max, cells_all = aggregate(t_sum, float(cells), dist, dev)
    value = cells_all / t_max

    # e2e: host buffers in, result back to host, through the same C ABI
    U_h = torch.empty((cfg.get("batch", 1), N + 1, d), dtype=torch.float64).pin_memory()
    e2e_t = []
    for _ in range(max(2, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        u0_d = u0_h.to(dev, non_blocking=True)
        Ud, st_e = solver.solve(u0_d)
        U_h.copy_(Ud, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = st_e["fine_cell_updates"] * ws / max(e2e_t) if ws > 1 else \
        st_e["fine_cell_updates"] / statistics.median(e2e_t)

    extra = {}
    if rank == 0 and not args.skip_fp64:
        # plain FP64 GPU RandNet-Parareal (per-stage kernels, FP64 features)
        for label, prec, ex in (("fp64_plain", "fp64", "plain"), ("fp64_fused", "fp64", "fused"),
                                ("mixed_bf16", "mixed_bf16", "fused")):
            with rnp.Solver(rnp.problem(cfg, precision=prec, exec=ex, autotune=int(ex == "fused")),
                            stream=stream) as s2:
                if label == "mixed_bf16":
                    s2.solve(u0)                   # warm-up (graph capture)
                torch.cuda.synchronize(dev)
                ev0.record(stream)
                U2, st2 = s2.solve(u0)
                ev1.record(stream)
                ev1.synchronize()
                extra[f"tts_{label}_ms"] = ev0.elapsed_time(ev1)
                extra[f"K_{label}"] = st2["K"]
                if label == "fp64_fused":
                    Uf = U2.clone()
                    extra["mixed_vs_fp64_max_abs"] = float((U - U2).abs().max().item())
                if label == "mixed_bf16":
                    extra["mixed_bf16_vs_fp64_rel"] = float(((U2 - Uf).abs().max() /
                                                              Uf.abs().max()).item())
                    extra["mixed_vs_fp64_rel"] = float(((U - U2).abs().max() /
                                                        U2.abs().max()).item())
        # classic Parareal (the correction of Eq. 4), same workload and mixed
        # precision: the in-repo counterpart of the paper's speed-up over
        # Parareal
        try:
            with rnp.Solver(rnp.problem(cfg, precision=args.precision, exec="fused",
                                        autotune=1, corr="parareal"), stream=stream) as s2:
                s2.solve(u0, check=False)          # warm-up (graph capture)
                torch.cuda.synchronize(dev)
                ev0.record(stream)
                U2, st2 = s2.solve(u0, check=False)
                ev1.record(stream)
                ev1.synchronize()
                extra["tts_parareal_ms"] = ev0.elapsed_time(ev1)
                extra["K_parareal"] = st2["K"]
                extra["parareal_converged"] = bool(st2["converged"])
        except rnp.RnpError as e:                  # classic Parareal can diverge
            extra["parareal_error"] = str(e)[:120]

    if rank == 0:
        pk = peaks()
        sm_mhz = clk.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
        flops_cu = FLOPS_PER_CELL_UPDATE[WORKLOAD]
        cells_per_launch = stats["fine_cell_updates"] / max(stats["K"], 1)
        achieved = cells_per_launch * flops_cu / (statistics.mean(fine_ms) / 1e3) / 1e12
        peak_alu = fp32_alu_peak_tflops(pk.get("sm_max_mhz", 2070.0))
        tf = tiling["fine"]
        kname = (f"k_stencil_mixed<{WORKLOAD}, PX={tf['px']}, RS={tf['rs']}> "
                 f"cluster {tf['cluster']} x {tf['threads']} threads") if tf["px"] else \
            f"k_stencil_fused<{WORKLOAD}, double> cluster {tf['cluster']}"
        # slices per fine launch = cell-updates per launch / (nF steps x d unknowns)
        traffic = traffic_per_launch(tf, cells_per_launch / (cfg["nF"] * W.dim(cfg)))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(tts), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16+f64" if args.precision == "mixed_bf16" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": describe(cfg),
                       "precision": args.precision, "exec": "fused", "autotune": True,
                       "replica_per_rank": True, "l2": "flushed between timed steps "
                       "(256 MB write)", "parallelism": f"replicas x{ws}"},
            "time_to_solution_ms": {"p50": statistics.median(tts), "min": min(tts),
                                    "max": max(tts)},
            "K": stats["K"], "fine_ms_per_iteration": statistics.mean(fine_ms),
            "stencil_tiling": tiling,
            "sweep_ms": stats["t_sweep_ms"], "fit_ms": stats["t_fit_ms"],
            "roofline": {"kernel": kname, "bound": "alu",
                         "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
                         "frac": achieved / peak_alu, "traffic": traffic,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock "
                                        f"{pk.get('sm_max_mhz', 2070.0)} MHz (MEASURED_PEAKS)",
                         # the same kernel against HBM: its measured DRAM bytes
                         # per launch over the launch time, of the measured copy
                         # bandwidth (the state lives in shared memory, so this
                         # stays far below 1)
                         "hbm": None if traffic is None else {
                             "achieved_gbs": traffic / (statistics.mean(fine_ms) / 1e3) / 1e9,
                             "peak_gbs": pk["hbm_gbs"],
                             "frac": traffic / (statistics.mean(fine_ms) / 1e3) / 1e9
                             / pk["hbm_gbs"]}},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(u0_h.numel() * 8),
                    "d2h_bytes_per_step": int(U_h.numel() * 8),
                    "ms_per_step": statistics.median(e2e_t) * 1e3},
            "gpu_launches": launches,
            "clocks": clk,
            "wall_s": t_wall,
        }
        line.update(extra)
        if not args.skip_cpu:
            try:
                line["cpu_baseline"] = cpu_baseline()
            except Exception as e:  # report, do not fail the GPU line
                line["cpu_baseline"] = {"error": repr(e)}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    solver.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_bf16", "fp64"])
    ap.add_argument("--profile", action="store_true",
                    help="one solve, then one fine step, one batched feature map and one "
                         "more solve inside NVTX ranges 'rnp_fine', 'rnp_features' and "
                         "'rnp_solve' (for ncu --nvtx)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["diffreact2d", "burgers1d", "bruss2d", "bruss3d", "swe_box"])
    ap.add_argument("--max-iters", type=int, default=0)
    ap.add_argument("--tile", default="",
                    help="fixed stencil tiling 'cluster,threads' instead of the autotuner's")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
