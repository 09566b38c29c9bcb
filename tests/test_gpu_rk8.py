"""The eighth-order fine solver (Cooper & Verner RK8, FP64) on the GPU
against the FP64 oracle.

Bars: F bit-identical to the oracle in both executions (the fused kernel
at every cluster size the cases force, and the plain per-stage kernels),
periodic and no-flux; G unchanged; a solve reaches the oracle's K with
U within 1e-10, and with eps = 0 it reproduces the serial RK8 solution bit
for bit.  Unsupported combinations are refused at rnp_create."""
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


CASES = [
    # tN short enough that G's forward Euler is stable (4 nu dt_G / h^2 < 2)
    ("burgers1d", dict(nx=128, N=3, nF=40, nG=8, tN=0.1), 0, "periodic"),
    ("burgers1d", dict(nx=96, N=2, nF=30, nG=8, tN=0.1), 0, "neumann"),
    ("diffreact2d", dict(nx=32, ny=32, N=3, nF=12, tN=0.5), 1, "periodic"),
    ("diffreact2d", dict(nx=32, ny=32, N=3, nF=12, tN=0.5), 4, "periodic"),
    ("diffreact2d", dict(nx=48, ny=40, N=2, nF=10, tN=0.5), 8, "neumann"),
    ("bruss2d", dict(nx=24, ny=24, N=2, nF=10, tN=1.0), 2, "periodic"),
    ("bruss3d", dict(nx=10, ny=10, nz=10, N=2, nF=6, tN=0.5, batch=1), 5, "periodic"),
    ("swe2d", dict(nx=24, ny=24, N=2, nF=10, nG=4, tN=0.05), 2, "periodic"),
    ("bruss3d", dict(pde="heat", nx=16, ny=12, nz=8, N=2, nF=10, param=[0.05], ic="sine",
                     lx=1.0, ly=1.0, lz=1.0, tN=0.01, batch=1), 2, "neumann"),
]


def _starts(cfg, B):
    rng = np.random.default_rng(8)
    u0 = W.initial_condition(cfg, batch=B)
    n = cfg["N"]
    if cfg["ic"] == "steady_uniform":
        return np.stack([np.stack([u0[b] + 0.01 * rng.random(u0.shape[1]) * (j + 1)
                                   for j in range(n)]) for b in range(B)])
    return np.stack([np.stack([u0[b] * (1 + 0.01 * rng.standard_normal(u0.shape[1]))
                               for j in range(n)]) for b in range(B)])


@pytest.mark.parametrize("exec_", ["fused", "plain"])
@pytest.mark.parametrize("name,kw,cluster,bc", CASES)
def test_fine_rk8_bitwise(R, orc, name, kw, cluster, bc, exec_):
    cfg = W.config(name, bc=bc, fscheme="rk8", **kw)
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


def test_rk8_is_more_accurate_than_rk4(R, orc):
    # same step count: the RK8 slice lands far closer to the exact flow
    # (approximated by the oracle's RK4 with 400 times more steps)
    cfg = W.config("burgers1d", nx=64, N=2, nF=10, nG=4)
    u0 = W.initial_condition(cfg)
    starts = np.stack([u0[0], u0[0]])[None]
    dT = (cfg["tN"] - cfg["t0"]) / cfg["N"]
    exact = orc.rk4(orc.problem(cfg), u0[0], dT / 4000, 4000)
    err = {}
    for fs in ("rk4", "rk8"):
        with R.Solver(R.problem(dict(cfg, fscheme=fs), precision="fp64")) as s:
            err[fs] = np.abs(host(s.fine_batch(dev(starts)))[0, 0] - exact).max()
    assert err["rk8"] < 1e-2 * err["rk4"], err     # about 7e-4 here


@pytest.mark.parametrize("exec_", ["fused", "plain"])
def test_solve_rk8_against_oracle(R, orc, exec_):
    cfg = W.config("burgers1d", nx=128, N=16, nF=60, nG=4, fscheme="rk8")
    u0 = W.initial_condition(cfg)
    orc.set_threads(8)
    rc, Uo, so, _ = orc.solve(orc.problem(cfg), u0[0])
    assert rc == 0
    with R.Solver(R.problem(cfg, precision="fp64", exec=exec_)) as s:
        U, st = s.solve(dev(u0))
        U = host(U)[0]
    assert st["K"] == so.K
    assert np.abs(U - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_solve_rk8_tol0_is_serial_fine(R, orc):
    cfg = W.config("diffreact2d", nx=16, ny=16, N=5, nF=8, tol=0.0, fscheme="rk8")
    u0 = W.initial_condition(cfg)
    p = orc.problem(cfg)
    with R.Solver(R.problem(cfg, precision="fp64")) as s:
        U, st = s.solve(dev(u0), check=False)
        U = host(U)[0]
    assert st["K"] == cfg["N"]
    assert np.array_equal(U, orc.serial_fine(p, u0[0]))


def test_rk8_refusals(R):
    cfg = W.config("diffreact2d", nx=32, ny=32, N=2, nF=4, fscheme="rk8")
    with pytest.raises(R.RnpError) as e:
        R.Solver(R.problem(cfg, precision="mixed"))
    assert e.value.status == R.RNP_EINVAL
    # fused RK8 keeps at most 2 x 512 cells per CTA of a 16-CTA cluster
    big = W.config("diffreact2d", nx=256, ny=256, N=2, nF=4, fscheme="rk8")
    with pytest.raises(R.RnpError) as e:
        R.Solver(R.problem(big, precision="fp64"))
    assert e.value.status == R.RNP_EINVAL
    # the plain execution has no such limit
    with R.Solver(R.problem(big, precision="fp64", exec="plain")) as s:
        assert s is not None


def test_rk8_robustness_burgers_full_size_sampled(R, orc):
    """The robustness study's Burgers with the paper's RK8 (d = 128,
    N = 128 on [0, 5.9], 313 steps per slice): F on all 128 slices in one
    fused launch, sampled slices bit-identical to the oracle."""
    from paper_2411_06225_gb300.robustness import system_config
    cfg = system_config("burgers", fine="rk8")
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)
    with R.Solver(R.problem(cfg, precision="fp64")) as s:
        U0 = host(s.coarse_sweep(0, dev(u0)))
        starts = U0[:, :cfg["N"]].copy()
        Fv = host(s.fine_batch(dev(starts)))
    for j in (0, 64, 127):
        assert np.array_equal(Fv[0, j], orc.fine(p, starts[0, j])), j
