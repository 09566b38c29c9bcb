"""No-flux (Neumann, finite-volume) walls on the GPU against the FP64 oracle.

Bars as for the periodic operators: FP64 F and G bit-identical to the oracle
(fused, every cluster size the cases force, and plain); FP32 F within 2e-7
and G within 1e-6 of the oracle's FP64 (relative to the largest state
magnitude); solves within 1e-10 (FP64, same K) and 1e-5 (mixed, K within 1).
Cluster sizes 1, 2 and 4+ exercise the wall ranks' own ghost rows, the
one-CTA wall case and the interior ranks' pushes."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import paper_2411_06225_gb300 as rnp
    rnp.build()
    rnp.lib()
    return rnp


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = [
    ("burgers1d", dict(nx=96, N=3, nF=40, nG=40, tN=0.3), 0),
    ("diffreact2d", dict(nx=32, ny=32, N=3, nF=20, tN=0.5), 1),
    ("diffreact2d", dict(nx=32, ny=32, N=3, nF=20, tN=0.5), 2),
    ("diffreact2d", dict(nx=48, ny=40, N=2, nF=15, tN=0.5), 8),
    ("bruss2d", dict(nx=24, ny=24, N=3, nF=15, tN=1.0), 4),
    ("bruss3d", dict(nx=10, ny=10, nz=10, N=2, nF=10, tN=0.5, batch=1), 5),
    ("bruss3d", dict(pde="heat", nx=16, ny=12, nz=8, N=2, nF=10, param=[0.05], ic="sine",
                     lx=1.0, ly=1.0, lz=1.0, tN=0.01, batch=1), 2),
]


def _starts(cfg, B):
    rng = np.random.default_rng(21)
    u0 = W.initial_condition(cfg, batch=B)
    n = cfg["N"]
    if cfg["ic"] == "steady_uniform":
        return np.stack([np.stack([u0[b] + 0.01 * rng.random(u0.shape[1]) * (j + 1)
                                   for j in range(n)]) for b in range(B)])
    return np.stack([np.stack([u0[b] * (1 + 0.01 * rng.standard_normal(u0.shape[1]))
                               for j in range(n)]) for b in range(B)])


@pytest.mark.parametrize("exec_", ["fused", "plain"])
@pytest.mark.parametrize("name,kw,cluster", CASES)
def test_fp64_bitwise(R, orc, name, kw, cluster, exec_):
    cfg = W.config(name, bc="neumann", **kw)
    cfg["cluster"] = cluster
    B = cfg.get("batch", 1)
    p = orc.problem(cfg)
    starts = _starts(cfg, B)
    with R.Solver(R.problem(cfg, precision="fp64", exec=exec_)) as s:
        out = host(s.fine_batch(dev(starts)))
        U = host(s.coarse_sweep(0, dev(starts[:, 0])))
    for b in range(B):
        for j in range(cfg["N"]):
            ref = orc.fine(p, starts[b, j])
            assert np.array_equal(out[b, j], ref), (b, j, np.abs(out[b, j] - ref).max())
        ref = starts[b, 0]
        for i in range(1, cfg["N"] + 1):
            ref = orc.coarse(p, ref)
            assert np.array_equal(U[b, i], ref), (b, i)


@pytest.mark.parametrize("name,kw,cluster,threads", [
    ("diffreact2d", dict(nx=64, ny=64, N=2, nF=100, tN=0.5), 1, 512),
    ("diffreact2d", dict(nx=64, ny=64, N=2, nF=100, tN=0.5), 2, 256),
    ("diffreact2d", dict(nx=128, ny=128, N=2, nF=100, tN=0.2), 8, 256),
    ("diffreact2d", dict(nx=128, ny=128, N=2, nF=100, tN=0.2), 16, 128),
    ("bruss2d", dict(nx=64, ny=64, N=2, nF=150, nG=16, tN=1.0), 4, 0),
    ("bruss3d", dict(nx=16, ny=16, nz=16, N=2, nF=60, nG=8, tN=0.5, batch=1), 4, 0),
])
def test_mixed_fine_and_coarse_error(R, orc, name, kw, cluster, threads):
    cfg = W.config(name, bc="neumann", **kw)
    cfg["cluster"], cfg["threads"] = cluster, threads
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg, batch=1)
    starts = np.stack([u0[0]] * cfg["N"])[None]
    with R.Solver(R.problem(cfg, precision="mixed")) as s:
        assert s.stencil_config("fine")["px"] > 0        # the FP32 kernel ran
        out = host(s.fine_batch(dev(starts)))
        U = host(s.coarse_sweep(0, dev(u0)))
    e_f = rel(out[0, 0], orc.fine(p, u0[0]))
    g, e_g = u0[0], 0.0
    for i in range(1, cfg["N"] + 1):
        g = orc.coarse(p, g)
        e_g = max(e_g, rel(U[0, i], g))
    assert e_f <= 2e-7, e_f
    assert e_g <= 1e-6, e_g


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_against_oracle(R, orc, precision):
    cfg = W.config("diffreact2d", bc="neumann", nx=32, ny=32, N=16, nF=200)
    u0 = W.initial_condition(cfg)
    orc.set_threads(8)
    rc, Uo, so, _ = orc.solve(orc.problem(cfg), u0[0])
    assert rc == 0
    with R.Solver(R.problem(cfg, precision=precision)) as s:
        U, st = s.solve(dev(u0))
        U = host(U)[0]
    if precision == "fp64":
        assert st["K"] == so.K
        assert rel(U, Uo) <= 1e-10
    else:
        assert abs(st["K"] - so.K) <= 1
        assert rel(U, Uo) <= 1e-5

