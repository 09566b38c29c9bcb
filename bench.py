#!/usr/bin/env python3
"""Benchmark: RandNet-Parareal time-to-solution on GB300.

One *step* is one full solve (Alg. 1: k = 0 coarse sweep, then iterations
of the parallel fine step, dataset append + features, exact leftmost slice,
sequential RandNet predictor-corrector sweep and the Eq. 5 stopping rule).

The headline workload is the largest single-GPU configuration: the 3D
Brusselator (App. E shape), 40^3 grid x 2 species (d = 128000), periodic,
side 16, a = 1, b = 3, D = 0.02 / 0.01, N = 256 slices on [0, 5],
F = RK4 1000 steps/slice, G = forward Euler 4 steps/slice, a batch of 8
seeded initial conditions (steady state plus U(0, 0.1) noise) solved
together, M = 100 ReLU features, m = 4 neighbours, lambda = 1e-7,
tol = 1e-6; the dataset arena is sized for 16 iterations.  The timed form is
the mixed-precision fused path: FP32 stencils on a compensated (two-word)
state, random features from BF16 operands with FP32 accumulation (the
batched dataset rows of each iteration on the tcgen05 tensor cores, the
sweep's single queries on CUDA cores), FP32 neighbour distances, FP64 ridge
solve, correction and norm.  The 2D diffusion-reaction workload (128^2 x 2,
N = 64, F = RK4 x 2000, G = Euler x 8) is measured after it and reported
under "workloads", in its own timed form (FP32 features on CUDA cores: BF16
features cost it one more iteration), with the plain FP64 GPU form, the
fused FP64 form, BF16 features and classic Parareal beside it; so are the
2D Brusselator (256^2 x 2, N = 128), the paper's shallow-water dam break
(100 x 50 x 3 with walls, N = 235, beside its plain FP64 form) and the 1D
Burgers workload (d = 128, N = 16, all FP64 as specified).  Under
"serving": Poisson streams of shallow-water solves served with continuous
batching at 0.3, 0.7 and 0.9 x the measured closed-loop throughput (p50 /
p99 latency, solves/s).

value = fine cell-updates per second over the whole job (sum over ranks of
the fine RK4 unknown-steps the solves performed / max over ranks of the
timed device time).  ms_per_step = time-to-solution of one solve.  e2e:
the same metric through the same C ABI call given HOST buffers (pinned
u0 in, pinned U out): the library copies the initial states in and the
states out, each member's converged states while later iterations run.

roofline: the fine stencil kernel, with the algorithmic work per cell-step
the workload's roof is stated in (the 3D and 2D Brusselator and the dam
break: bytes of an FP32 state streamed through HBM, against the measured
copy bandwidth; diffusion-reaction: FP32 flops, against the FP32 ALU peak),
over the kernel's launch time from CUDA events on the launching stream.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload bruss3d|diffreact2d|bruss2d|swe_box|burgers1d]

Under torchrun every rank solves its own seeded replica (weak scaling, no
collective on the data path); only the barrier and the max-reduction of the
timings cross ranks.  ``--impl reference`` times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload (its line carries the
same ``config``; the sample is described in ``cpu_baseline.sample``).
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

WORKLOAD = "bruss3d"  # the headline workload; --workload measures the others
# Workloads measured after the headline (reported under "workloads"), with
# the other forms timed beside each: every form on the 2D diffusion-reaction
# workload; the plain FP64 form on the paper's dam break; none where a full
# FP64 solve takes minutes (2D Brusselator) or the timed form is FP64.
SECONDARY = {
    "diffreact2d": (("fp64_plain", "fp64", "plain"), ("fp64_fused", "fp64", "fused"),
                    ("mixed_bf16", "mixed_bf16", "fused")),
    "bruss2d": (),
    "swe_box": (("fp64_plain", "fp64", "plain"),),
    "burgers1d": (),
}
METRIC = ("Parareal time-to-solution @tol 1e-6 vs plain FP64; cell-updates/s, %HBM; "
          "p50/p99")
UNIT = "cell-updates/s"

# Timed form per workload: BF16 random features where they leave the
# iteration count unchanged and save time (3D Brusselator: K = 3 either way),
# FP32 features elsewhere (diffusion-reaction: K = 5 with BF16, 4 without);
# the 1D Burgers workload is specified all-FP64 (its coarse step is unstable
# in FP32 rounding).
TIMED_PRECISION = {"bruss3d": "mixed_bf16", "burgers1d": "fp64"}

# Workload settings of the benchmark beyond the canonical configurations:
# the 3D Brusselator's dataset arena is sized for 16 iterations (8 members x
# 3976 stored rows of 128000 unknowns: 49 GB) instead of N = 256.
BENCH_OVERRIDES = {"bruss3d": dict(max_iters=16)}

# The algorithmic work per fine cell-step (one unknown, one RK4 step) that
# each workload's roofline is stated in, and the roof it is compared with:
#   bytes: the FP32 state read and written once per step, 8 B per unknown,
#          against the measured HBM copy bandwidth;
#   flops: FP32 flops per cell-step, against the FP32 ALU peak.
#   fp64flops: FP64 flops per cell-step (the all-FP64 Burgers workload),
#          against the nominal FP64 rate (no measured FP64 peak is given).
ROOF_UNIT = {"bruss3d": ("bytes", 8.0), "bruss2d": ("bytes", 8.0),
             "swe_box": ("bytes", 8.0), "diffreact2d": ("flops", 40.0),
             "burgers1d": ("fp64flops", 60.0)}
FP64_NOMINAL_TFLOPS = 1.25

# Every FP32 multiply and add of the fine step counted separately, per
# cell-update, from the right-hand side formulas, plus 13 per unknown for
# the four stage combinations:
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

# DRAM bytes per slice of one fine launch (dram__bytes_read.sum +
# dram__bytes_write.sum of an ncu capture of the kernel divided by the
# slices it ran), per workload and tiling (cluster, threads, PX, RS).  The
# kernel reads each start state once and writes each result once, so the
# traffic grows in proportion to the slices; a tiling with no capture
# reports null.
STENCIL_TRAFFIC_PER_SLICE = {
    # 64 slices of 128^2 x 2: 16,840,192 B read, 0 B written
    ("diffreact2d", (8, 256, 2, 4)): 16840192 / 64,
    # the same launch at the 16-CTA clusters of 128 threads: 16,838,144 B
    # read, 0 B written
    ("diffreact2d", (16, 128, 2, 4)): 16838144 / 64,
    # 16 slices of 40^3 x 2 (one member): 16,448,512 B read, 0 B written
    # (the FP64 results stayed in L2 within the capture)
    ("bruss3d", (10, 800, 2, 4)): 16448512 / 16,
}


def traffic_per_launch(workload: str, tf: dict, slices: float):
    key = (workload, (tf["cluster"], tf["threads"], tf["px"], tf["rs"]))
    b = STENCIL_TRAFFIC_PER_SLICE.get(key)
    return None if b is None else b * slices


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


def bench_config(name: str, **kw) -> dict:
    """The benchmark's configuration of a workload."""
    over = dict(BENCH_OVERRIDES.get(name, {}))
    over.update(kw)
    return W.config(name, **over)


def describe(cfg: dict) -> str:
    grid = "x".join(str(v) for v in (cfg["nx"], cfg["ny"], cfg["nz"]) if v > 1)
    bc = "walls" if cfg.get("bc", "periodic") == "neumann" else "periodic"
    fs = cfg.get("fscheme", "rk4").upper()
    return (f"{cfg['pde']} {grid}x{W.ncomp(cfg)} {bc}, N={cfg['N']}, "
            f"F={fs}x{cfg['nF']}, G=Eulerx{cfg['nG']}, M={cfg['M']}, m={cfg['m']}, "
            f"tol={cfg['tol']}, batch={cfg.get('batch', 1)}, max_iters={cfg['max_iters']}")


def line_config(name: str, precision: str, ws: int) -> dict:
    """The ``config`` object of a JSON line: the same for the GPU arm and the
    reference arm of one workload."""
    cfg = bench_config(name)
    grid = "x".join(str(v) for v in (cfg["nx"], cfg["ny"], cfg["nz"]) if v > 1)
    return {"workload": f"{name}: {describe(cfg)}", "grid": f"{grid}x{W.ncomp(cfg)}",
            "N": cfg["N"], "nF": cfg["nF"], "nG": cfg["nG"], "batch": cfg.get("batch", 1),
            "max_iters": cfg["max_iters"], "precision": precision, "exec": "fused",
            "autotune": True, "replica_per_rank": True,
            "l2": "flushed between timed steps (256 MB write)",
            "parallelism": f"replicas x{ws}"}


def replica_seed(rank: int, name: str | None = None) -> int:
    """Seed of the replica a rank solves (weak scaling: one solve per rank)."""
    return W.CONFIGS[name or WORKLOAD]["seed"] + 1000 * rank


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


def cpu_sample_config(name: str) -> tuple[dict, str]:
    """The bounded oracle sample of a workload: the same grid, operator,
    coarse solver, RandNet settings and slice length, one member and at most
    16 slices (t_N shortened so each slice keeps its length), and at most
    2e9 fine cell-updates per iteration (nF cut where needed); a full solve."""
    full = bench_config(name)
    Ns = min(full["N"], 16)
    dT = (full["tN"] - full["t0"]) / full["N"]
    d = W.dim(full)
    nF = min(full["nF"], max(50, int(2e9 // (Ns * d))))
    cfg = bench_config(name, N=Ns, tN=full["t0"] + Ns * dT, nF=nF, batch=1,
                       max_iters=Ns)
    grid = "x".join(str(v) for v in (cfg["nx"], cfg["ny"], cfg["nz"]) if v > 1)
    what = (f"{name} {grid}x{W.ncomp(cfg)}, one member, N={Ns} of {full['N']} slices "
            f"(same slice length), nF={nF} of {full['nF']} RK4 steps per slice")
    return cfg, what


def cpu_baseline(name: str | None = None) -> dict:
    """The FP64 oracle on the host cores: a full solve of the bounded sample
    of the workload (slice-parallel over all cores), in fine cell-updates
    per second."""
    import oracle
    name = name or WORKLOAD
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    cfg, what = cpu_sample_config(name)
    p = oracle.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    t0 = time.perf_counter()
    rc, U, st, _ = oracle.solve(p, u0)
    dt = time.perf_counter() - t0
    return {"value": st.fine_cell_updates / dt, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{what}: full solve, K={st.K}, {dt:.2f} s, FP64, slice-parallel "
                      f"over {cores} threads"}


def timed_precision(name: str, requested: str | None) -> str:
    return requested or TIMED_PRECISION.get(name, "mixed")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    name = getattr(args, "workload", None) or WORKLOAD
    precision = timed_precision(name, getattr(args, "precision", None))
    samples = []
    base = None
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(name)
        if i >= args.warmup:
            samples.append(b["value"])
        base = b
    value = statistics.median(samples) if samples else base["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": line_config(name, precision, args.gpus),
        "cpu_baseline": {"kind": "oracle", "cores": base["cores"], "sample": base["sample"],
                         "value": value, "unit": UNIT},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def roofline(name: str, cells_per_launch: float, launch_s: float, tf: dict,
             slices: float, pk: dict) -> dict:
    """The fine kernel against the roof its workload is stated in, plus the
    same launch against the other roof."""
    kname = (f"k_stencil_mixed{'_wide' if tf['threads'] > 512 else ''}<{name}, "
             f"PX={tf['px']}, RS={tf['rs']}> cluster {tf['cluster']} x {tf['threads']} threads"
             if tf["px"] else f"k_stencil_fused<{name}, double> cluster {tf['cluster']}")
    traffic = traffic_per_launch(name, tf, slices)
    alu_peak = fp32_alu_peak_tflops(pk.get("sm_max_mhz", 2070.0))
    alu_src = (f"152 SMs x 128 FP32 lanes x 2 x max SM clock {pk.get('sm_max_mhz', 2070.0)} MHz "
               "of the measured peaks")
    kind, per = ROOF_UNIT.get(name, ("flops", FLOPS_PER_CELL_UPDATE.get(name, 0.0)))
    if kind == "bytes":
        ach = cells_per_launch * per / launch_s / 1e9
        r = {"kernel": kname, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"],
             "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "traffic": traffic,
             "per_unit": f"{per:g} B per cell-step (FP32 state read + written once)",
             "peak_source": "hbm_gbs of the measured peaks (copy bandwidth)"}
    elif kind == "fp64flops":
        ach = cells_per_launch * per / launch_s / 1e12
        r = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS,
             "unit": "TFLOP/s", "frac": ach / FP64_NOMINAL_TFLOPS, "traffic": traffic,
             "per_unit": f"{per:g} FP64 flop per cell-step",
             "peak_source": "nominal FP64 rate of the GB300 (no measured FP64 peak)"}
    else:
        ach = cells_per_launch * per / launch_s / 1e12
        r = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": alu_peak,
             "unit": "TFLOP/s", "frac": ach / alu_peak, "traffic": traffic,
             "per_unit": f"{per:g} FP32 flop per cell-step", "peak_source": alu_src}
    # the same launch counted with every FP32 operation of the step
    fl = FLOPS_PER_CELL_UPDATE.get(name) if tf["px"] else None
    if fl:
        a2 = cells_per_launch * fl / launch_s / 1e12
        r["alu_recount"] = {"flop_per_cell_step": fl, "achieved": a2, "peak": alu_peak,
                            "unit": "TFLOP/s", "frac": a2 / alu_peak}
    # the measured DRAM bytes over the launch, of the copy bandwidth (the
    # state lives in shared memory, so this stays far below 1)
    if traffic is not None:
        g = traffic / launch_s / 1e9
        r["dram"] = {"achieved_gbs": g, "peak_gbs": pk["hbm_gbs"], "frac": g / pk["hbm_gbs"]}
    return r


def measure(rnp, torch, name, args, rank, ws, dist, dev, stream, flush, headline):
    """Time `steps` solves of one workload; returns the figures of its line."""
    cfg = bench_config(name, seed=replica_seed(rank, name))
    if args.max_iters:
        cfg["max_iters"] = args.max_iters
    d = W.dim(cfg)
    N = cfg["N"]
    B = cfg.get("batch", 1)
    u0_h = torch.as_tensor(W.initial_condition(cfg)).pin_memory()
    u0 = u0_h.to(dev)
    prec = timed_precision(name, args.precision)
    if args.tile and headline:
        # a fixed stencil tiling (cluster, threads), e.g. to profile one
        # configuration: the autotuner's pick can differ under a profiler
        c_, t_ = (int(x) for x in args.tile.split(","))
        prob = rnp.problem(cfg, precision=prec, exec="fused", autotune=0,
                           cluster=c_, threads=t_)
    else:
        prob = rnp.problem(cfg, precision=prec, exec="fused", autotune=1)
    solver = rnp.Solver(prob, stream=stream)
    tiling = {"fine": solver.stencil_config("fine"), "coarse": solver.stencil_config("coarse")}
    steps = args.steps if headline else max(3, min(args.steps, 5))
    for _ in range(args.warmup):
        solver.solve(u0)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    clocks = None
    if headline:
        try:
            gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            gpu_id = dev.index
        clocks = ClockSampler(gpu_id)
    tts, fine_ms, cells, launches, stats = [], [], 0, 0, None
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    if clocks:
        clocks.start()
    t_wall0 = time.perf_counter()
    for _ in range(steps):
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
    clk = clocks.stop() if clocks else None
    t_sum = sum(tts) / 1e3
    # max over ranks of the timed device time, sum of the work
    t_max, cells_all = aggregate(t_sum, float(cells), dist, dev) if headline else \
        (t_sum, float(cells))
    value = cells_all / t_max

    # e2e: the same C ABI call with HOST buffers (pinned): the library copies
    # u0 in and the states out, each member's converged states while later
    # iterations run, the rest at the end
    U_h = torch.empty((B, N + 1, d), dtype=torch.float64).pin_memory()
    e2e_t = []
    st_e = stats
    for _ in range(max(2, min(steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, st_e = solver.solve(u0_h, U=U_h)
        torch.cuda.synchronize(dev)
        e2e_t.append(time.perf_counter() - t0)
    if headline and ws > 1:
        e2e_value = st_e["fine_cell_updates"] * ws / max(e2e_t)
    else:
        e2e_value = st_e["fine_cell_updates"] / statistics.median(e2e_t)

    pk = peaks()
    launch_s = statistics.mean(fine_ms) / 1e3
    cells_per_launch = stats["fine_cell_updates"] / max(stats["K"], 1)
    # slices per fine launch = cell-updates per launch / (nF steps x d unknowns)
    slices = cells_per_launch / (cfg["nF"] * d)
    res = {
        "value": value, "ms_per_step": statistics.mean(tts),
        "time_to_solution_ms": {"p50": statistics.median(tts), "min": min(tts),
                                "max": max(tts)},
        "K": stats["K"], "K_each": stats.get("K_each", [])[:B],
        "fine_ms_per_iteration": statistics.mean(fine_ms),
        "fine_cell_updates_per_solve": stats["fine_cell_updates"],
        "stencil_tiling": tiling,
        "sweep_ms": stats["t_sweep_ms"], "fit_ms": stats["t_fit_ms"],
        "roofline": roofline(name, cells_per_launch, launch_s, tiling["fine"], slices, pk),
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(u0_h.numel() * 8),
                "d2h_bytes_per_step": int(U_h.numel() * 8),
                "ms_per_step": statistics.median(e2e_t) * 1e3},
        "gpu_launches": launches, "wall_s": t_wall, "steps": steps, "precision": prec,
    }
    if clk is not None:
        res["clocks"] = clk
    return res, solver, u0, U, cfg


def compare_forms(rnp, torch, name, cfg, args, stream, dev, u0, U, forms, parareal=True,
                  timed="mixed"):
    """One solve of each other form of the workload on the same input."""
    extra = {}
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    Uf = None
    for label, prec, ex in forms:
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
                extra["timed_vs_fp64_max_abs"] = float((U - U2).abs().max().item())
                extra["timed_vs_fp64_rel"] = float(((U - U2).abs().max() /
                                                    U2.abs().max()).item())
            if label == "mixed_bf16" and Uf is not None:
                extra["mixed_bf16_vs_fp64_rel"] = float(((U2 - Uf).abs().max() /
                                                         Uf.abs().max()).item())
            if label in ("mixed_bf16", "mixed") and label != timed:
                extra[f"{label}_vs_timed_rel"] = float(((U2 - U).abs().max() /
                                                        U.abs().max()).item())
            del U2
    # classic Parareal (the correction of Eq. 4), same workload and mixed
    # precision: the in-repo counterpart of the paper's speed-up over Parareal
    if not parareal:
        return extra
    try:
        with rnp.Solver(rnp.problem(cfg, precision=timed, exec="fused",
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
    return extra


def fp64_fine_sample(rnp, torch, cfg, stream, dev, u0):
    """The fused FP64 fine kernel on one member's slices for 64 steps: its
    cell-updates per second beside the mixed kernel's (a full FP64 solve of
    the headline workload takes minutes)."""
    c = dict(cfg, batch=1, nF=64, max_iters=1)
    with rnp.Solver(rnp.problem(c, precision="fp64", exec="fused", autotune=0),
                    stream=stream) as s:
        starts = u0[:1, None, :].expand(1, c["N"], u0.shape[1]).contiguous()
        s.fine_batch(starts)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        s.fine_batch(starts)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        return {"cell_updates_per_s": c["N"] * W.dim(c) * 64 / (ms / 1e3),
                "sample": f"one member, {c['N']} slices x 64 RK4 steps, {ms:.1f} ms",
                "tiling": s.stencil_config("fine")}


def serving_block(args) -> dict:
    """C5: Poisson streams of shallow-water solves (grids {64^2, 128^2,
    256^2} x 3, N in {32, 64, 128}, seeded Gaussian bumps) served with
    continuous batching, at 0.3, 0.7 and 0.9 x the closed-loop throughput
    measured first on the same request mix: p50 / p99 latency and solves/s.
    `--serve-requests` requests per load (2000 is the full specification)."""
    from paper_2411_06225_gb300 import serve
    n = args.serve_requests
    base = W.serving_stream(n, rate=1.0)
    for r in base:
        r["cfg"]["max_iters"] = min(12, r["cfg"]["N"])
    closed = serve.run_stream([dict(r, arrival=0.0) for r in base[: max(16, n // 4)]],
                              "mixed", 4)
    rate = closed["solves_per_s"]
    out = {"requests_per_load": n, "closed_loop_solves_per_s": rate,
           "stream": "shallow water, grids {64,128,256}^2 x 3, N in {32,64,128}, "
                     "Poisson arrivals, mixed precision, 4 slots per class pool, "
                     "max_iters 12"}
    for frac in (0.3, 0.7, 0.9):
        reqs = W.serving_stream(n, rate=rate * frac)
        for r in reqs:
            r["cfg"]["max_iters"] = min(12, r["cfg"]["N"])
        res = serve.run_stream(reqs, "mixed", 4)
        out[f"{frac:.1f}x"] = {k: res[k] for k in ("p50_ms", "p99_ms", "mean_ms",
                                                    "solves_per_s", "converged", "K_mean",
                                                    "wall_s")}
    return out


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
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    if args.profile:
        # the fine step of the timed form once, inside an NVTX range, on a
        # reduced batch / slice count when --batch / --slices are given
        over = {}
        if args.batch:
            over["batch"] = args.batch
        if args.slices:
            full = bench_config(WORKLOAD)
            dT = (full["tN"] - full["t0"]) / full["N"]
            over.update(N=args.slices, tN=full["t0"] + args.slices * dT,
                        max_iters=min(args.slices, full["max_iters"]))
        cfg = bench_config(WORKLOAD, **over)
        prec = timed_precision(WORKLOAD, args.precision)
        if args.tile:
            c_, t_ = (int(x) for x in args.tile.split(","))
            prob = rnp.problem(cfg, precision=prec, exec="fused", cluster=c_,
                               threads=t_)
        else:
            prob = rnp.problem(cfg, precision=prec, exec="fused", autotune=1)
        u0 = torch.as_tensor(W.initial_condition(cfg)).to(dev)
        with rnp.Solver(prob, stream=stream) as solver:
            U0 = solver.coarse_sweep(0, u0)
            starts = U0[:, :cfg["N"]].contiguous()
            solver.fine_batch(starts)              # untimed first launch
            torch.cuda.synchronize(dev)
            torch.cuda.nvtx.range_push("rnp_fine")
            solver.fine_batch(starts)
            torch.cuda.synchronize(dev)
            torch.cuda.nvtx.range_pop()
            print(json.dumps({"profile": "done", "workload": describe(cfg),
                              "precision": prec,
                              "tiling": solver.stencil_config("fine")}))
        return 0

    res, solver, u0, U, cfg = measure(rnp, torch, WORKLOAD, args, rank, ws, dist, dev,
                                      stream, flush, headline=True)
    extra = {}
    if rank == 0 and not args.skip_extra:
        if WORKLOAD == "bruss3d":
            # the other feature precision on the same workload, and the FP64
            # fine kernel's rate (a full FP64 solve takes minutes)
            other = "mixed" if res["precision"] == "mixed_bf16" else "mixed_bf16"
            extra.update(compare_forms(rnp, torch, WORKLOAD, cfg, args, stream, dev, u0, U,
                                       [(other, other, "fused")], parareal=False,
                                       timed=res["precision"]))
            extra["fp64_fused_fine_sample"] = fp64_fine_sample(rnp, torch, cfg, stream, dev,
                                                               u0)
        else:
            extra.update(compare_forms(rnp, torch, WORKLOAD, cfg, args, stream, dev, u0, U,
                                       [("fp64_plain", "fp64", "plain"),
                                        ("fp64_fused", "fp64", "fused"),
                                        ("mixed_bf16", "mixed_bf16", "fused")],
                                       timed=res["precision"]))
    solver.close()
    del U
    secondary = {}
    if rank == 0 and not args.skip_extra:
        for name, forms in SECONDARY.items():
            if name == WORKLOAD:
                continue
            try:
                r2, s2, u2, U2, cfg2 = measure(rnp, torch, name, args, rank, ws, None, dev,
                                               stream, flush, headline=False)
                r2["config"] = line_config(name, r2["precision"], ws)
                r2.update(compare_forms(rnp, torch, name, cfg2, args, stream, dev, u2, U2,
                                        list(forms), parareal=name == "diffreact2d",
                                        timed=r2["precision"]))
                s2.close()
                del U2
                secondary[name] = r2
            except Exception as e:  # report, do not fail the GPU line
                secondary[name] = {"error": repr(e)[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": ws,
            "steps": res["steps"], "warmup": args.warmup,
            "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+bf16+f64" if res["precision"] == "mixed_bf16" else "f32+f64",
            "data": "synthetic",
            "config": line_config(WORKLOAD, res["precision"], ws),
        }
        for k in ("time_to_solution_ms", "K", "K_each", "fine_ms_per_iteration",
                  "fine_cell_updates_per_solve", "stencil_tiling", "sweep_ms", "fit_ms",
                  "roofline", "e2e", "gpu_launches", "clocks", "wall_s"):
            if k in res:
                line[k] = res[k]
        line.update(extra)
        if secondary:
            line["workloads"] = secondary
        if args.serve_requests > 0 and not args.skip_extra:
            try:
                line["serving"] = serving_block(args)
            except Exception as e:  # report, do not fail the GPU line
                line["serving"] = {"error": repr(e)[:200]}
        if not args.skip_cpu:
            try:
                line["cpu_baseline"] = cpu_baseline(WORKLOAD)
            except Exception as e:  # report, do not fail the GPU line
                line["cpu_baseline"] = {"error": repr(e)}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["mixed", "mixed_bf16", "fp64"],
                    help="timed form (default: the workload's, see TIMED_PRECISION)")
    ap.add_argument("--profile", action="store_true",
                    help="one untimed and one NVTX-ranged ('rnp_fine') fine step of the "
                         "timed form, for ncu; --batch / --slices reduce the launch")
    ap.add_argument("--batch", type=int, default=0, help="members (with --profile)")
    ap.add_argument("--slices", type=int, default=0,
                    help="slices of the same length (with --profile)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-extra", action="store_true",
                    help="no other forms, no secondary workloads")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["bruss3d", "diffreact2d", "burgers1d", "bruss2d", "swe_box"])
    ap.add_argument("--max-iters", type=int, default=0)
    ap.add_argument("--serve-requests", type=int, default=120,
                    help="requests per load level of the serving streams (0: none; "
                         "2000: the full specification)")
    ap.add_argument("--tile", default="",
                    help="fixed stencil tiling 'cluster,threads' instead of the autotuner's")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
