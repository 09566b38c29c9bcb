"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module only *describes* problems and draws their initial conditions. It
holds none of the method's arithmetic (no right-hand side, integrator,
feature map, neighbour search or ridge solve), so the CUDA path and the CPU
oracle can both consume it without sharing any code of the method.

Every workload mirrors the shape of one of the paper's experiments (Sec. 5,
App. E and Tables 4-7); the paper simulates its own data, so nothing here
stands in for an external dataset:

* ``burgers1d``   1D viscous Burgers, periodic on [-1,1), nu = 0.01, d = 128,
                  N = 16 slices on [0,1], F = RK4 1000 steps, G = Euler 4 steps.
* ``diffreact2d`` 2D FitzHugh-Nagumo diffusion-reaction (Sec. 5.2), 128 x 128
                  periodic on (-1,1)^2, d = 32768, N = 64 on [0,5],
                  F = RK4 2000 steps, G = Euler 8 steps.
* ``bruss2d``     2D Brusselator (App. E), 256 x 256 x 2, periodic, side 16,
                  N = 128 on [0,10], F = RK4 4000, G = Euler 16.
* ``bruss3d``     3D Brusselator, 40^3 x 2, side 16, N = 256 on [0,5],
                  batch of 8 initial conditions, F = RK4 1000, G = Euler 4.
* ``swe2d``       2D shallow water (Sec. 5.3), Gaussian bump, periodic unit
                  square, used by the request stream of the server.
"""
from __future__ import annotations

import copy
import math

import numpy as np

PDE_IDS = {
    "burgers1d": 0,
    "diffreact2d": 1,
    "bruss2d": 2,
    "bruss3d": 3,
    "swe2d": 4,
    "heat": 5,
    "advect1d": 6,
}
NCOMP = {"burgers1d": 1, "diffreact2d": 2, "bruss2d": 2, "bruss3d": 2,
         "swe2d": 3, "heat": 1, "advect1d": 1}

SEED_BASE = 2411

# Canonical full-size workloads.  ``param`` is the PDE coefficient vector:
#   burgers1d: [nu]; diffreact2d: [Du, Dv, c]; bruss*: [a, b, D0, D1];
#   swe2d: [g]; heat: [D]; advect1d: [c].
CONFIGS = {
    "burgers1d": dict(pde="burgers1d", nx=128, ny=1, nz=1, lx=2.0, ly=1.0,
                      lz=1.0, param=[0.01], t0=0.0, tN=1.0, N=16, nF=1000,
                      nG=4, M=100, m=4, lam=1e-7, tol=1e-6, batch=1,
                      ic="fourier4", seed=SEED_BASE + 0),
    "diffreact2d": dict(pde="diffreact2d", nx=128, ny=128, nz=1, lx=2.0,
                        ly=2.0, lz=1.0, param=[1e-3, 5e-3, 5e-3], t0=0.0,
                        tN=5.0, N=64, nF=2000, nG=8, M=100, m=4, lam=1e-7,
                        tol=1e-6, batch=1, ic="normal", seed=SEED_BASE + 1),
    "bruss2d": dict(pde="bruss2d", nx=256, ny=256, nz=1, lx=16.0, ly=16.0,
                    lz=1.0, param=[1.0, 3.0, 0.02, 0.01], t0=0.0, tN=10.0,
                    N=128, nF=4000, nG=16, M=100, m=4, lam=1e-7, tol=1e-6,
                    batch=1, ic="steady_uniform", seed=SEED_BASE + 2),
    "bruss3d": dict(pde="bruss3d", nx=40, ny=40, nz=40, lx=16.0, ly=16.0,
                    lz=16.0, param=[1.0, 3.0, 0.02, 0.01], t0=0.0, tN=5.0,
                    N=256, nF=1000, nG=4, M=100, m=4, lam=1e-7, tol=1e-6,
                    batch=8, ic="steady_uniform", seed=SEED_BASE + 3),
    "swe2d": dict(pde="swe2d", nx=64, ny=64, nz=1, lx=1.0, ly=1.0, lz=1.0,
                  param=[9.81], t0=0.0, tN=0.5, N=32, nF=0, nG=0, M=100, m=4,
                  lam=1e-7, tol=1e-6, batch=1, ic="gauss_bump",
                  seed=SEED_BASE + 4),
    # The paper's radial dam break in a box (Sec. 5.3 and its appendix):
    # [-5,5] x [0,5] (here shifted to [0,10] x [0,5]), reflecting walls, a
    # Gaussian column at (-2.5, 1.5) with covariance 0.25 I, t in [0, 20],
    # N = 235, G = 7 Euler steps per slice, m = 3.  Mesh 100 x 50 cells
    # (the paper's coarsest 101 x 51 points, made even for the FP32 tiles);
    # nF from the CFL rule of swe_steps (the paper's 1e5 RK4 steps per slice
    # is far below the stability limit).  Flat bottom unless a
    # ``bathymetry`` array is added.
    "swe_box": dict(pde="swe2d", nx=100, ny=50, nz=1, lx=10.0, ly=5.0, lz=1.0,
                    param=[9.81], t0=0.0, tN=20.0, N=235, nF=0, nG=7, M=100, m=3,
                    lam=1e-7, tol=1e-6, batch=1, ic="gauss_column", bc="neumann",
                    seed=SEED_BASE + 6),
}


def config(name: str, **overrides) -> dict:
    """A copy of a canonical workload with some fields replaced."""
    cfg = copy.deepcopy(CONFIGS[name])
    cfg.update(overrides)
    if cfg["pde"] == "swe2d" and (cfg["nF"] <= 0 or cfg["nG"] <= 0):
        nf, ng = swe_steps(cfg)
        cfg["nF"] = cfg["nF"] if cfg["nF"] > 0 else nf
        cfg["nG"] = cfg["nG"] if cfg["nG"] > 0 else ng
    cfg.setdefault("max_iters", cfg["N"])
    return cfg


def swe_steps(cfg: dict) -> tuple[int, int]:
    """Fine/coarse step counts per slice from a CFL-style rule:
    dt_F = 0.1 h / 4 and dt_G = 0.4 h / 4 (h the grid spacing)."""
    h = cfg["lx"] / cfg["nx"]
    dT = (cfg["tN"] - cfg["t0"]) / cfg["N"]
    return (int(math.ceil(dT / (0.1 * h / 4.0))),
            int(math.ceil(dT / (0.4 * h / 4.0))))


def ncomp(cfg: dict) -> int:
    return NCOMP[cfg["pde"]]


def dim(cfg: dict) -> int:
    return ncomp(cfg) * cfg["nx"] * cfg["ny"] * cfg["nz"]


def initial_condition(cfg: dict, seed: int | None = None,
                      batch: int | None = None) -> np.ndarray:
    """Seeded initial states, shape [batch, d], float64.

    * ``fourier4``: u0(x) = 1/4 sum_{k=1..4} a_k sin(k pi x + p_k) on [-1,1),
      a_k ~ U(-1,1), p_k ~ U(0, 2 pi).
    * ``normal``: every cell of every species i.i.d. N(0,1) (Sec. 5.2).
    * ``steady_uniform``: Brusselator steady state (a, b/a) plus i.i.d.
      U(0, 0.1) per cell.
    * ``gauss_bump``: shallow-water depth 1 + A exp(-r^2 / (2 w^2)) around the
      domain centre (minimum-image distance), A ~ U(0.1,0.5),
      w ~ U(0.05,0.2), zero momentum.
    * ``gauss_column``: shallow-water depth 1 plus the bivariate normal
      density with mean (0.25 lx, 0.3 ly) and covariance 0.25 (lx / 10)^2 I
      (the paper's column at (-2.5, 1.5), covariance 0.25 I, in a [-5, 5] x
      [0, 5] box), at the cell centres, zero momentum; deterministic.
    * ``sine``: single Fourier mode sin(2 pi k x / lx) (test operators), mode
      number cfg['mode'] (default 1), along each axis that has > 1 point.
    * ``cos9``: u0(x) = 0.5 (cos(9 pi x / 2) + 1) on [-1, 1), the Burgers
      initial condition of the paper's Burgers experiments (Sec. 5.1);
      deterministic.
    """
    seed = cfg["seed"] if seed is None else seed
    batch = cfg.get("batch", 1) if batch is None else batch
    rng = np.random.default_rng(seed)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    n = nx * ny * nz
    nc = ncomp(cfg)
    out = np.empty((batch, nc * n), dtype=np.float64)
    kind = cfg["ic"]
    for b in range(batch):
        if kind == "fourier4":
            x = -1.0 + cfg["lx"] * np.arange(nx) / nx
            a = rng.uniform(-1.0, 1.0, 4)
            ph = rng.uniform(0.0, 2.0 * np.pi, 4)
            u = sum(a[k] * np.sin((k + 1) * np.pi * x + ph[k]) for k in range(4))
            out[b] = 0.25 * u
        elif kind == "normal":
            out[b] = rng.standard_normal(nc * n)
        elif kind == "steady_uniform":
            a, bb = cfg["param"][0], cfg["param"][1]
            out[b, :n] = a + rng.uniform(0.0, 0.1, n)
            out[b, n:] = bb / a + rng.uniform(0.0, 0.1, n)
        elif kind == "gauss_bump":
            amp = rng.uniform(0.1, 0.5)
            w = rng.uniform(0.05, 0.2)
            xs = (np.arange(nx) + 0.5) / nx * cfg["lx"]
            ys = (np.arange(ny) + 0.5) / ny * cfg["ly"]
            dx = xs - 0.5 * cfg["lx"]
            dy = ys - 0.5 * cfg["ly"]
            dx = dx - cfg["lx"] * np.round(dx / cfg["lx"])
            dy = dy - cfg["ly"] * np.round(dy / cfg["ly"])
            r2 = dy[:, None] ** 2 + dx[None, :] ** 2
            out[b, :n] = (1.0 + amp * np.exp(-r2 / (2.0 * w * w))).ravel()
            out[b, n:] = 0.0
        elif kind == "gauss_column":
            var = 0.25 * (cfg["lx"] / 10.0) ** 2
            xs = (np.arange(nx) + 0.5) / nx * cfg["lx"] - 0.25 * cfg["lx"]
            ys = (np.arange(ny) + 0.5) / ny * cfg["ly"] - 0.3 * cfg["ly"]
            r2 = ys[:, None] ** 2 + xs[None, :] ** 2
            out[b, :n] = (1.0 + np.exp(-r2 / (2.0 * var)) / (2.0 * np.pi * var)).ravel()
            out[b, n:] = 0.0
        elif kind == "cos9":
            x = -1.0 + cfg["lx"] * np.arange(nx) / nx
            out[b] = 0.5 * (np.cos(4.5 * np.pi * x) + 1.0)
        elif kind == "sine":
            k = cfg.get("mode", 1)
            x = np.arange(nx) / nx
            f = np.sin(2.0 * np.pi * k * x)[None, None, :]
            if ny > 1:
                f = f * np.sin(2.0 * np.pi * k * np.arange(ny) / ny)[None, :, None]
            if nz > 1:
                f = f * np.sin(2.0 * np.pi * k * np.arange(nz) / nz)[:, None, None]
            out[b] = np.broadcast_to(f, (nz, ny, nx)).ravel()
        else:
            raise ValueError(f"unknown initial condition {kind!r}")
    return out


def serving_stream(n_requests: int, rate: float, seed: int = SEED_BASE + 5,
                   grids=(64, 128, 256), slices=(32, 64, 128)) -> list[dict]:
    """Poisson stream of shallow-water solve requests: exponential
    inter-arrival times at ``rate`` per second, grid side and slice count
    drawn uniformly from ``grids`` and ``slices``, one seeded bump each."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate)
        g = int(rng.choice(grids))
        N = int(rng.choice(slices))
        cfg = config("swe2d", nx=g, ny=g, N=N, nF=0, nG=0,
                     seed=int(rng.integers(1 << 31)))
        reqs.append(dict(id=r, arrival=t, cfg=cfg))
    return reqs
