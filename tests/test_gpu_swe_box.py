"""Shallow water in a box (reflecting walls) and over a bottom b on the GPU
against the FP64 oracle (Sec. 5.3).

Bars as for the other operators: FP64 F and G bit-identical to the oracle
(fused at the cluster sizes the cases force, and plain); FP32 F within 2e-7
and G within 1e-6 of the oracle's FP64 (relative to the largest state
magnitude); solves at the oracle's K within 1e-10 (FP64) and within one
iteration and 1e-5 (mixed).  Walls keep the mass in the box."""
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


def _bottom(nx, ny, seed=4, amp=0.15):
    """A smooth seeded bottom: a hump plus a gentle slope."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    cx, cy, w = rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7), rng.uniform(0.1, 0.2)
    X, Y = np.meshgrid(x, y)
    return amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * w * w)) + 0.05 * X


def _cfg(nx, ny, bc="neumann", bottom=False, **kw):
    c = W.config("swe_box", nx=nx, ny=ny, bc=bc, **kw)
    if bottom:
        c["bathymetry"] = _bottom(nx, ny)
    return c


def _starts(cfg):
    rng = np.random.default_rng(13)
    u0 = W.initial_condition(cfg)[0]
    n = cfg["nx"] * cfg["ny"]
    out = []
    for j in range(cfg["N"]):
        v = u0.copy()
        v[:n] *= 1 + 0.01 * rng.random(n)
        v[n:] = 0.02 * rng.standard_normal(2 * n)   # some momentum at the walls
        out.append(v)
    return np.stack(out)[None]


CASES = [
    (dict(nx=24, ny=20, N=3, nF=20, nG=4, tN=0.3), 1, "neumann", False),
    (dict(nx=24, ny=20, N=3, nF=20, nG=4, tN=0.3), 4, "neumann", True),
    (dict(nx=30, ny=25, N=2, nF=15, nG=3, tN=0.3), 5, "neumann", True),
    (dict(nx=32, ny=16, N=2, nF=15, nG=3, tN=0.3), 2, "periodic", True),
]


@pytest.mark.parametrize("exec_", ["fused", "plain"])
@pytest.mark.parametrize("kw,cluster,bc,bottom", CASES)
def test_fp64_bitwise(R, orc, kw, cluster, bc, bottom, exec_):
    cfg = _cfg(bc=bc, bottom=bottom, **kw)
    cfg["cluster"] = cluster
    p = orc.problem(cfg)
    starts = _starts(cfg)
    with R.Solver(R.problem(cfg, precision="fp64", exec=exec_)) as s:
        out = host(s.fine_batch(dev(starts)))
        U = host(s.coarse_sweep(0, dev(starts[:, 0])))
    for j in range(cfg["N"]):
        ref = orc.fine(p, starts[0, j])
        assert np.array_equal(out[0, j], ref), (j, np.abs(out[0, j] - ref).max())
    ref = starts[0, 0]
    for i in range(1, cfg["N"] + 1):
        ref = orc.coarse(p, ref)
        assert np.array_equal(U[0, i], ref), i


@pytest.mark.parametrize("kw,cluster,threads,bottom", [
    (dict(nx=64, ny=32, N=2, nF=60, nG=8, tN=0.3), 1, 0, False),
    (dict(nx=64, ny=32, N=2, nF=60, nG=8, tN=0.3), 4, 0, True),
    # the paper's mesh spacing and slice length (20 / 235): G's Euler step
    # stays inside its CFL limit
    (dict(nx=100, ny=50, N=2, nF=40, nG=7, tN=0.17), 5, 0, True),
    (dict(nx=100, ny=50, N=2, nF=40, nG=7, tN=0.17), 10, 0, False),
])
def test_mixed_fine_and_coarse_error(R, orc, kw, cluster, threads, bottom):
    cfg = _cfg(bottom=bottom, **kw)
    cfg["cluster"], cfg["threads"] = cluster, threads
    p = orc.problem(cfg)
    starts = _starts(cfg)
    with R.Solver(R.problem(cfg, precision="mixed")) as s:
        assert s.stencil_config("fine")["px"] > 0        # the FP32 kernel ran
        out = host(s.fine_batch(dev(starts)))
        U = host(s.coarse_sweep(0, dev(starts[:, 0])))
    e_f = max(rel(out[0, j], orc.fine(p, starts[0, j])) for j in range(cfg["N"]))
    g, e_g = starts[0, 0], 0.0
    for i in range(1, cfg["N"] + 1):
        g = orc.coarse(p, g)
        e_g = max(e_g, rel(U[0, i], g))
    assert e_f <= 2e-7, e_f
    assert e_g <= 1e-6, e_g


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_walls_keep_the_mass(R, precision):
    cfg = _cfg(64, 32, bottom=True, N=2, nF=200, nG=8, tN=1.0)
    n = 64 * 32
    starts = _starts(cfg)
    with R.Solver(R.problem(cfg, precision=precision)) as s:
        out = host(s.fine_batch(dev(starts)))
    for j in range(cfg["N"]):
        m0, m1 = starts[0, j, :n].sum(), out[0, j, :n].sum()
        assert abs(m1 - m0) <= (1e-12 if precision == "fp64" else 1e-6) * m0, (m0, m1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_against_oracle(R, orc, precision):
    cfg = _cfg(40, 20, bottom=True, N=16, nF=0, nG=7, tN=2.0)
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


def test_bathymetry_refused_for_other_pdes(R):
    cfg = W.config("diffreact2d", nx=16, ny=16, N=2, nF=4)
    cfg["bathymetry"] = np.zeros((16, 16))
    with pytest.raises(R.RnpError) as e:
        R.Solver(R.problem(cfg))
    assert e.value.status == R.RNP_EINVAL


def test_full_size_box_sampled(R, orc):
    """The paper's dam-break workload at full size, in the bench's launch
    configuration (F on all 235 slice starts in one launch, autotuned
    tiling): sampled slices within the FP32 bound of the FP64 oracle, and
    a full mixed solve whose states satisfy |U_i - F(U_{i-1})| <= 10 tol
    on sampled slices."""
    cfg = W.config("swe_box")
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)
    with R.Solver(R.problem(cfg, precision="mixed", autotune=1)) as s:
        U0 = host(s.coarse_sweep(0, dev(u0)))
        starts = U0[:, :cfg["N"]].copy()
        Fv = host(s.fine_batch(dev(starts)))
        for j in (0, 117, 234):
            assert rel(Fv[0, j], orc.fine(p, starts[0, j])) <= 2e-7, j
        s.reset()
        U, st = s.solve(dev(u0))
        U = host(U)[0]
    assert st["converged"]
    for i in (3, 120, 235):
        assert np.abs(U[i] - orc.fine(p, U[i - 1])).max() <= 10 * cfg["tol"], i
