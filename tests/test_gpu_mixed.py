"""Mixed precision (FP32 stencil arithmetic with a compensated FP32 state,
FP64 correction, ridge and norm) against the FP64 oracle.

Stated error bounds (relative to the largest state magnitude):
  * one fine slice F (RK4, up to 2000 steps):           <= 2e-7
  * one coarse slice G (Euler):                          <= 1e-6 (large
    coarse steps make dt*|h(u)| comparable to |u|, so the FP32 right-hand
    side error is not damped by the step size)
  * a converged RandNet-Parareal solve at tol 1e-6:     <= 1e-5 (max-abs over
    all slices against the FP64 oracle's solve), K within 1 of the oracle.
The full-size test runs the benchmark workload (2D diffusion-reaction,
128 x 128 x 2, N = 64, 2000 RK4 steps per slice) in the launch configuration
bench.py times and checks sampled slices one by one against the oracle.
"""
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
    ("burgers1d", dict(nx=128, N=4, nF=250, nG=200)),
    ("diffreact2d", dict(nx=32, ny=32, N=3, nF=100, tN=0.5)),
    ("diffreact2d", dict(nx=128, ny=128, N=2, nF=200, tN=0.2)),
    ("bruss2d", dict(nx=64, ny=64, N=2, nF=300, nG=16, tN=1.0)),
    ("bruss3d", dict(nx=16, ny=16, nz=16, N=2, nF=100, nG=8, tN=0.5, batch=1)),
    ("swe2d", dict(nx=64, ny=64, N=4, nF=60, nG=60)),
]


@pytest.mark.parametrize("name,kw", CASES)
def test_mixed_fine_and_coarse_error(R, orc, name, kw):
    cfg = W.config(name, **kw)
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg, batch=1)
    n = cfg["N"]
    starts = np.stack([u0[0]] * n)[None]
    with R.Solver(R.problem(cfg, precision="mixed")) as s:
        out = host(s.fine_batch(dev(starts)))
        U = host(s.coarse_sweep(0, dev(u0)))
    ref = orc.fine(p, u0[0])
    e_f = rel(out[0, 0], ref)
    g = u0[0]
    e_g = 0.0
    for i in range(1, n + 1):
        g = orc.coarse(p, g)
        e_g = max(e_g, rel(U[0, i], g))
    print(f"{name}: F rel err {e_f:.2e}, G rel err {e_g:.2e}")
    assert e_f <= 2e-7, e_f
    assert e_g <= 1e-6, e_g
    for j in range(1, n):
        assert np.array_equal(out[0, j], out[0, 0])  # same input, same output


@pytest.mark.parametrize("name,kw", [
    # the 128-point Burgers workload with 4 Euler steps per slice has an
    # unstable coarse step (diffusion number 2.56 > 2): it is an all-FP64
    # configuration, FP32 rounding noise overflows; a stable coarse step here
    ("burgers1d", dict(nG=16)),
    ("diffreact2d", dict(nx=32, ny=32, N=16, nF=200)),
    ("diffreact2d", dict(nx=64, ny=64, N=16, nF=100, batch=2)),
    ("bruss2d", dict(nx=32, ny=32, N=12, nF=150, nG=4, tN=2.0)),
    ("bruss3d", dict(nx=16, ny=16, nz=16, N=8, nF=60, nG=3, tN=0.5, batch=2)),
    ("swe2d", dict(nx=32, ny=32, N=8, nF=40, nG=20)),
])
def test_mixed_solve_error_against_fp64_oracle(R, orc, name, kw):
    cfg = W.config(name, **kw)
    B = cfg.get("batch", 1)
    u0 = W.initial_condition(cfg, batch=B)
    orc.set_threads(8)
    p = orc.problem(cfg)
    with R.Solver(R.problem(cfg, precision="mixed")) as s:
        U, st = s.solve(dev(u0))
        U = host(U)
    for b in range(B):
        rc, Uo, so, _ = orc.solve(p, u0[b])
        e = rel(U[b], Uo)
        print(f"{name} b={b}: K mixed {st['K_each'][b]} fp64 {so.K}, rel err {e:.2e}")
        assert abs(st["K_each"][b] - so.K) <= 1
        assert e <= 1e-5, e


def test_full_size_benchmark_workload_sampled(R, orc):
    """The bench workload at full size, in the bench's launch configuration:
    F on all 64 slice starts in one launch, two slices checked against the
    FP64 oracle; then a full mixed solve whose converged states satisfy
    |U_i - F(U_{i-1})| <= 10 tol on sampled slices (oracle F, FP64)."""
    cfg = W.config("diffreact2d")
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)
    d = W.dim(cfg)
    orc.set_threads(8)
    with R.Solver(R.problem(cfg, precision="mixed")) as s:
        U0 = host(s.coarse_sweep(0, dev(u0)))
        starts = U0[:, :cfg["N"]].copy()
        Fv = host(s.fine_batch(dev(starts)))
        for j in (0, 37):
            e = rel(Fv[0, j], orc.fine(p, starts[0, j]))
            assert e <= 2e-7, (j, e)
        s.reset()
        U, st = s.solve(dev(u0))
        U = host(U)[0]
    assert st["converged"]
    for i in (5, 40, 64):
        r = np.abs(U[i] - orc.fine(p, U[i - 1])).max()
        assert r <= 10 * cfg["tol"], (i, r)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotuned_tiling_gives_the_same_results(R, precision):
    cfg = W.config("diffreact2d", nx=64, ny=64, N=8, nF=60, tN=0.5)
    u0 = W.initial_condition(cfg)
    starts = np.stack([u0[0] * (1 + 0.01 * j) for j in range(cfg["N"])])[None]
    outs = []
    for tune in (0, 1):
        with R.Solver(R.problem(cfg, precision=precision, autotune=tune)) as s:
            conf = s.stencil_config("fine")
            assert conf["tuned"] == bool(tune)
            outs.append(host(s.fine_batch(dev(starts))))
    if precision == "fp64":
        assert np.array_equal(outs[0], outs[1])
    else:
        assert rel(outs[1], outs[0]) <= 2e-7


def test_large_shallow_water_grid_runs_an_fp32_tile(R, orc):
    """256 x 256 x 3 has no spill-free FP32 tile of <= 512 threads; the mixed
    context must still pick an FP32 tile (not the FP64 kernel)."""
    cfg = W.config("swe2d", nx=256, ny=256, N=64, nF=0, nG=0)   # CFL-rule step counts
    u0 = W.initial_condition(cfg)
    with R.Solver(R.problem(cfg, precision="mixed")) as s:
        assert s.stencil_config("fine")["px"] > 0
        assert s.stencil_config("coarse")["px"] > 0
        out = host(s.fine_batch(dev(np.stack([u0[0]] * 2)[None])))
    e = rel(out[0, 0], orc.fine(orc.problem(cfg), u0[0]))
    assert e <= 2e-7, e
