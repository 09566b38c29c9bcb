"""Robustness of RandNet-Parareal to its knobs (the paper's robustness study,
App. "Robustness study", Figs. of K over m and M): the number of iterations
to convergence K over the number of nearest neighbours m, the number of
hidden neurons M and independent draws of the random weights (A, zeta).

Two systems, as in the paper:
  * ``burgers``   1D Burgers as in the paper's Burgers experiment: d = 128,
                  N = 128 slices on [0, 5.9], u0 = 0.5 (cos(9 pi x / 2) + 1),
                  nu = 0.01, G = Euler x 4 per slice; F = RK4 x 100 per slice
                  by default (the fine step only needs to be far more
                  accurate than tol), or with ``--fine rk8`` the paper's
                  RK8 with its 4e4 fine steps spread over the 128 slices
                  (313 per slice);
  * ``diffreact`` diffusion-reaction on a 19 x 19 grid (d = 722, the paper's
                  robustness size), N = 32 on [0, 5], F = RK4 x 200,
                  G = Euler x 4.
The initial condition is fixed per system; only the weight seed, m and M
change.  Every solve runs on the GPU through the library (FP64 by default,
the paper's precision).  The solves of the grid are independent, so a small
pool of host threads runs them concurrently, each on its own CUDA stream.

    python -m paper_2411_06225_gb300.robustness --system burgers --seeds 20

prints one JSON line with the K histograms per m and per M.  The paper's
full grid (m = 2..20, M = 20..500 in steps of 10, 100 seeds) is
``--m 2:21:1 --M 20:501:10 --seeds 100``.
"""
from __future__ import annotations

import collections
import json
import threading
import time

SYSTEMS = ("burgers", "diffreact")


def system_config(name: str, fine: str = "rk4") -> dict:
    import workloads as W
    if fine not in ("rk4", "rk8"):
        raise ValueError(f"unknown fine solver {fine!r}")
    if name == "burgers":
        nF = 100 if fine == "rk4" else 313
        return W.config("burgers1d", N=128, tN=5.9, nF=nF, nG=4, ic="cos9", max_iters=128,
                        fscheme=fine)
    if name == "diffreact":
        return W.config("diffreact2d", nx=19, ny=19, N=32, nF=200, nG=4, tN=5.0, fscheme=fine)
    raise ValueError(f"unknown system {name!r} (one of {SYSTEMS})")


def weight_seeds(n: int, base: int = 7000) -> list[int]:
    """Seeds of the weight draws: base, base + 1, ... (the SplitMix64 streams
    of different seeds are independent)."""
    return [base + i for i in range(n)]


def grid(ms, Ms, seeds) -> list[tuple[int, int, int]]:
    return [(m, M, s) for s in seeds for m in ms for M in Ms]


def histograms(results) -> dict:
    """results: iterable of (m, M, seed, K, outcome) with outcome one of
    "converged", "notconv" (max_iters reached) and "diverged" (a non-finite
    state or ridge system).  Histograms of K per m and per M; the solves that
    did not converge are counted under "nc" and "div"."""
    by_m = collections.defaultdict(collections.Counter)
    by_M = collections.defaultdict(collections.Counter)
    Ks = []
    nc = div = 0
    for m, M, _, K, outcome in results:
        key = {"converged": str(K), "notconv": "nc", "diverged": "div"}[outcome]
        by_m[m][key] += 1
        by_M[M][key] += 1
        if outcome == "converged":
            Ks.append(K)
        elif outcome == "notconv":
            nc += 1
        else:
            div += 1
    rank = {"nc": 1 << 30, "div": (1 << 30) + 1}
    order = lambda c: dict(sorted(c.items(), key=lambda kv: rank.get(kv[0], 0) or int(kv[0])))
    return {
        "K_hist_by_m": {str(m): order(c) for m, c in sorted(by_m.items())},
        "K_hist_by_M": {str(M): order(c) for M, c in sorted(by_M.items())},
        "K_min": min(Ks) if Ks else None,
        "K_max": max(Ks) if Ks else None,
        "K_mean": sum(Ks) / len(Ks) if Ks else None,
        "not_converged": nc,
        "diverged": div,
        "solves": len(Ks) + nc + div,
    }


def run(system: str, points, precision: str = "fp64", workers: int = 8,
        fine: str = "rk4") -> list[tuple]:
    """Solve every (m, M, seed) point on the GPU; returns (m, M, seed, K,
    outcome) per point, in the order of ``points`` (see ``histograms``)."""
    import numpy as np
    import torch

    import workloads as W

    from . import RNP_ENONFINITE, RnpError, Solver, problem
    cfg = system_config(system, fine)
    u0_h = np.ascontiguousarray(W.initial_condition(cfg), dtype=np.float64)
    out = [None] * len(points)
    nxt = [0]
    lock = threading.Lock()
    errors = []

    def worker():
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            u0 = torch.as_tensor(u0_h, device="cuda")
            while True:
                with lock:
                    i = nxt[0]
                    nxt[0] += 1
                if i >= len(points) or errors:
                    return
                m, M, seed = points[i]
                try:
                    with Solver(problem(cfg, precision=precision, m=m, M=M, seed=seed),
                                stream=stream) as s:
                        try:
                            _, st = s.solve(u0, check=False)
                            out[i] = (m, M, seed, st["K"],
                                      "converged" if st["converged"] else "notconv")
                        except RnpError as e:
                            if e.status != RNP_ENONFINITE:
                                raise
                            out[i] = (m, M, seed, None, "diverged")
                except Exception as e:  # reported after the pool drains
                    errors.append(e)
                    return

    threads = [threading.Thread(target=worker) for _ in range(max(1, workers))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return out


def _range(spec: str) -> list[int]:
    """'a:b:c' -> range(a, b, c); 'x,y,z' -> [x, y, z]."""
    if ":" in spec:
        a, b, c = (int(v) for v in spec.split(":"))
        return list(range(a, b, c))
    return [int(v) for v in spec.split(",")]


def main():
    import argparse
    ap = argparse.ArgumentParser(description="K over m, M and weight draws (GPU)")
    ap.add_argument("--system", default="burgers", choices=SYSTEMS)
    ap.add_argument("--m", default="2,4,6,8,10,12,14,16,18,20",
                    help="nearest neighbours: 'a:b:step' or a list")
    ap.add_argument("--M", default="20,50,100,200,300,500", help="neurons: 'a:b:step' or a list")
    ap.add_argument("--seeds", type=int, default=20, help="weight draws")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--fine", default="rk4", choices=["rk4", "rk8"],
                    help="fine solver (rk8: FP64 only)")
    args = ap.parse_args()
    cfg = system_config(args.system, args.fine)
    pts = grid(_range(args.m), _range(args.M), weight_seeds(args.seeds))
    t0 = time.perf_counter()
    res = run(args.system, pts, args.precision, args.workers, args.fine)
    wall = time.perf_counter() - t0
    import workloads as W
    print(json.dumps(dict(system=args.system, d=W.dim(cfg), N=cfg["N"], fine=args.fine,
                          nF=cfg["nF"], precision=args.precision,
                          seeds=args.seeds, wall_s=wall, solves_per_s=len(pts) / wall,
                          **histograms(res))))


if __name__ == "__main__":
    main()
