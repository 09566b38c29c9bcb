"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars:
  * F and G in FP64 (fused and plain): bit-identical to the oracle.
  * random weights A, zeta: bit-identical (same counter generator).
  * scaling: bit-identical (min/max are exact).
  * predictions and end-to-end FP64 iterates: within 1e-10 relative to the
    largest state magnitude (the GPU sums long dot products as chunked trees,
    the oracle left to right), with identical iteration counts.
  * mixed precision (FP32 stencils): error against FP64 stated in
    test_gpu_mixed.py.
Sizes span several CTAs of a cluster and ragged thread tails.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-10


@pytest.fixture(scope="module")
def R():
    import torch
    import paper_2411_06225_gb300 as rnp
    rnp.build()
    rnp.lib()
    assert torch.cuda.is_available()
    return rnp


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


FINE_CASES = [
    ("burgers1d", dict(nx=128, N=4, nF=30, nG=200), 1, 0),
    ("burgers1d", dict(nx=300, N=3, nF=200, nG=300), 1, 0),
    ("burgers1d", dict(pde="advect1d", nx=64, N=2, nF=20, param=[0.7]), 1, 0),
    ("diffreact2d", dict(nx=32, ny=32, N=3, nF=15, tN=0.5), 1, 0),
    ("diffreact2d", dict(nx=32, ny=32, N=3, nF=15, tN=0.5), 1, 4),
    ("diffreact2d", dict(nx=48, ny=40, N=2, nF=10, tN=0.5), 2, 8),
    ("bruss2d", dict(nx=24, ny=24, N=3, nF=15, tN=1.0), 1, 2),
    ("bruss3d", dict(nx=10, ny=10, nz=10, N=2, nF=10, tN=0.5, batch=1), 1, 5),
    ("bruss3d", dict(nx=8, ny=9, nz=12, N=2, nF=10, tN=0.5, batch=2), 2, 0),
    ("swe2d", dict(nx=32, ny=32, N=4, nF=24, nG=40), 1, 4),
    ("bruss3d", dict(pde="heat", nx=16, ny=12, nz=8, N=2, nF=10, param=[0.05], ic="sine",
                     lx=1.0, ly=1.0, lz=1.0, tN=0.01), 1, 2),
]


@pytest.mark.parametrize("exec_", ["fused", "plain"])
@pytest.mark.parametrize("name,kw,B,cluster", FINE_CASES)
def test_fine_and_coarse_fp64_bitwise(R, orc, name, kw, B, cluster, exec_):
    cfg = W.config(name, **kw)
    cfg["batch"] = B
    cfg["cluster"] = cluster
    p_orc = orc.problem(cfg)
    rng = np.random.default_rng(11)
    u0 = W.initial_condition(cfg, batch=B)
    n = cfg["N"]
    starts = np.stack([np.stack([u0[b] * (1 + 0.01 * rng.standard_normal(u0.shape[1]))
                                 if cfg["ic"] != "steady_uniform" and cfg["pde"] != "swe2d"
                                 else u0[b] + 0.01 * rng.random(u0.shape[1]) * (j + 1)
                                 for j in range(n)]) for b in range(B)])
    with R.Solver(R.problem(cfg, precision="fp64", exec=exec_)) as s:
        out = host(s.fine_batch(dev(starts)))
        for b in range(B):
            for j in range(n):
                ref = orc.fine(p_orc, starts[b, j])
                assert np.array_equal(out[b, j], ref), (b, j, np.abs(out[b, j] - ref).max())
        # G through the k = 0 coarse sweep
        U = host(s.coarse_sweep(0, dev(starts[:, 0])))
        for b in range(B):
            ref = starts[b, 0]
            for i in range(1, n + 1):
                ref = orc.coarse(p_orc, ref)
                assert np.array_equal(U[b, i], ref), (b, i)


def test_weights_bitwise(R, orc):
    for cfg in (W.config("burgers1d"), W.config("diffreact2d", nx=64, ny=64, M=37)):
        A0, z0 = orc.weights(orc.problem(cfg))
        with R.Solver(R.problem(cfg)) as s:
            A, z = s.weights()
            assert np.array_equal(host(A), A0)
            assert np.array_equal(host(z), z0)


def test_weights_full_size_sampled(R, orc):
    cfg = W.config("bruss2d")
    d = W.dim(cfg)
    with R.Solver(R.problem(cfg, max_iters=1)) as s:
        A, z = s.weights()
        A = host(A)
        rng = np.random.default_rng(3)
        for _ in range(2000):
            w, j = int(rng.integers(cfg["M"])), int(rng.integers(d))
            assert A[w, j] == 2.0 * orc.uniform(cfg["seed"], 0, w * d + j) - 1.0


def test_scaling_from_k0_sweep_bitwise(R, orc):
    cfg = W.config("diffreact2d", nx=32, ny=32, N=6, nF=10, tN=0.5, batch=2)
    u0 = W.initial_condition(cfg)
    p = orc.problem(cfg)
    with R.Solver(R.problem(cfg)) as s:
        U = host(s.coarse_sweep(0, dev(u0)))
        c, r = s.scaling()
        for b in range(2):
            ref = [u0[b]]
            for i in range(cfg["N"]):
                ref.append(orc.coarse(p, ref[-1]))
            ref = np.stack(ref)
            assert np.array_equal(U[b], ref)
            c0, r0 = orc.scaling(p, ref)
            assert np.array_equal(c[b, :2], c0[:2]) and np.array_equal(r[b, :2], r0[:2])


@pytest.mark.parametrize("name,kw,P", [
    ("burgers1d", dict(nx=128, M=100), 23),
    ("diffreact2d", dict(nx=40, ny=36, M=64), 9),
    ("diffreact2d", dict(nx=128, ny=128, M=100), 70),
    ("bruss3d", dict(nx=10, ny=10, nz=10, M=50, batch=2), 5),
])
def test_fit_predict_matches_oracle(R, orc, name, kw, P):
    cfg = W.config(name, **kw)
    B = cfg.get("batch", 1)
    p = orc.problem(cfg)
    d = W.dim(cfg)
    rng = np.random.default_rng(5)
    Uin = rng.standard_normal((B, P, d))
    Y = rng.standard_normal((B, P, d))
    # duplicated rows and an exact query hit exercise the ties and the penalty
    Uin[:, 3] = Uin[:, 1]
    Y[:, 3] = Y[:, 1]          # a repeated input has the same target
    q = Uin[:, 2] + 1e-3 * rng.standard_normal((B, d))
    q[0] = Uin[0, 1]
    c = np.tile(np.array([0.25, -0.5, 0.0]), (B, 1))
    r = np.tile(np.array([2.0, 3.0, 1.0]), (B, 1))
    A, z = orc.weights(p)
    with R.Solver(R.problem(cfg, max_pairs=P + 4)) as s:
        s.set_scaling(c, r)
        s.randnet_fit(dev(Uin), dev(Y))
        assert s.pairs() == [P] * B
        out = host(s.randnet_predict(dev(q)))
    for b in range(B):
        S = np.stack([orc.scale(p, c[b], r[b], u) for u in Uin[b]])
        Phi = np.stack([orc.features(A, z, sr) for sr in S])
        rc, ref, nn = orc.predict(p, S, Y[b], Phi, A, z, c[b], r[b], q[b])
        assert rc >= 0
        assert rel_err(out[b], ref) < REL, (b, rel_err(out[b], ref))


def test_predict_with_empty_dataset_is_zero(R):
    cfg = W.config("burgers1d")
    with R.Solver(R.problem(cfg)) as s:
        out = host(s.randnet_predict(dev(np.ones((1, 128)))))
        assert np.all(out == 0.0)


SOLVE_CASES = [
    ("burgers1d", dict(), "randnet"),
    ("burgers1d", dict(), "parareal"),
    ("burgers1d", dict(nx=200, N=10, nF=300, nG=25, m=3, M=60), "randnet"),
    ("diffreact2d", dict(nx=32, ny=32, N=16, nF=200), "randnet"),
    ("diffreact2d", dict(nx=64, ny=64, N=16, nF=100, batch=2), "randnet"),
    ("bruss2d", dict(nx=32, ny=32, N=12, nF=150, nG=4, tN=2.0), "randnet"),
    ("bruss3d", dict(nx=10, ny=10, nz=10, N=8, nF=60, nG=3, tN=0.5, batch=2), "randnet"),
    ("swe2d", dict(nx=32, ny=32, N=8, nF=40, nG=20), "randnet"),
    ("swe2d", dict(nx=32, ny=32, N=8, nF=40, nG=20), "parareal"),
]


@pytest.mark.parametrize("exec_", ["fused", "plain"])
@pytest.mark.parametrize("name,kw,corr", SOLVE_CASES)
def test_solve_fp64_matches_oracle(R, orc, name, kw, corr, exec_):
    if exec_ == "plain" and kw.get("batch", 1) > 1:
        pytest.skip("plain path covered with batch 1")
    cfg = W.config(name, corr=corr, **kw)
    B = cfg.get("batch", 1)
    u0 = W.initial_condition(cfg, batch=B)
    orc.set_threads(8)
    p = orc.problem(cfg)
    with R.Solver(R.problem(cfg, precision="fp64", exec=exec_)) as s:
        U, st = s.solve(dev(u0))
        U = host(U)
    for b in range(B):
        rc, Uo, so, _ = orc.solve(p, u0[b])
        assert rc == orc.ORC_OK
        assert st["K_each"][b] == so.K
        assert rel_err(U[b], Uo) < REL, rel_err(U[b], Uo)
    assert st["converged"] == 1


@pytest.mark.parametrize("corr", ["randnet", "parareal"])
def test_solve_tol0_is_serial_fine_bitwise(R, orc, corr):
    cfg = W.config("diffreact2d", nx=16, ny=16, N=6, nF=30, tN=0.5, tol=0.0, corr=corr)
    u0 = W.initial_condition(cfg)
    with R.Solver(R.problem(cfg, precision="fp64")) as s:
        U, st = s.solve(dev(u0))
    assert st["K"] == cfg["N"]
    assert np.array_equal(host(U)[0], orc.serial_fine(orc.problem(cfg), u0[0]))


def test_batch_members_are_independent(R):
    cfg = W.config("diffreact2d", nx=32, ny=32, N=10, nF=80, batch=3)
    u0 = W.initial_condition(cfg)
    with R.Solver(R.problem(cfg, precision="fp64")) as s:
        Ub, stb = s.solve(dev(u0))
    Ub = host(Ub)
    cfg1 = dict(cfg, batch=1)
    for b in range(3):
        with R.Solver(R.problem(cfg1, precision="fp64")) as s:
            U1, st1 = s.solve(dev(u0[b:b + 1]))
        assert np.array_equal(host(U1)[0], Ub[b])
        assert st1["K"] == stb["K_each"][b]


def test_not_converged_and_bad_arguments(R):
    import torch
    cfg = W.config("burgers1d", max_iters=2, tol=1e-15)
    u0 = W.initial_condition(cfg)
    with R.Solver(R.problem(cfg)) as s:
        with pytest.raises(R.RnpError) as e:
            s.solve(dev(u0))
        assert e.value.status == R.RNP_ENOTCONV
        U, st = s.solve(dev(u0), check=False)
        assert st["K"] == 2 and not st["converged"] and torch.isfinite(U).all()
        with pytest.raises(ValueError):
            s.solve(dev(np.ones((1, 7))))
    bad = W.config("burgers1d")
    bad["nF"] = 0
    with pytest.raises(R.RnpError):
        R.Solver(R.problem(bad))


def test_nonfinite_state_is_reported(R):
    cfg = W.config("burgers1d", nx=64, N=4, nF=10, nG=2)
    u0 = W.initial_condition(cfg)
    u0[0, 5] = np.nan
    with R.Solver(R.problem(cfg)) as s:
        with pytest.raises(R.RnpError) as e:
            s.solve(dev(u0))
        assert e.value.status == R.RNP_ENONFINITE


@pytest.mark.parametrize("name,kw", [
    ("diffreact2d", dict(nx=16, ny=16, N=8, nF=40, M=32, m=3, tN=0.5)),
    ("burgers1d", dict(nx=64, N=10, nF=200, nG=16, M=40, m=4)),
])
def test_stepwise_replay_of_one_sweep(R, orc, name, kw):
    """One sweep of Eq. 3 in isolation: the oracle's k = 0 trajectory, the
    pairs (U_i, F(U_i) - G(U_i)) that iteration 1 appends and the scaling of
    Alg. 1 are given to the GPU context, which runs the sweep
    U_i = G(U_{i-1}) + f_hat(U_{i-1}) from the exact leftmost slice.  Each
    state matches the oracle replaying the same step (its G and its
    prediction from the same dataset) within 1e-10, so a near-tie flip of
    the m-nearest selection or a drift of the correction shows at its step
    rather than as a changed K."""
    cfg = W.config(name, **kw)
    p = orc.problem(cfg)
    N, nc = cfg["N"], W.ncomp(cfg)
    u0 = W.initial_condition(cfg)[0]
    U0 = [u0]
    for _ in range(N):
        U0.append(orc.coarse(p, U0[-1]))
    U0 = np.stack(U0)
    c, r = orc.scaling(p, U0)
    c[nc:], r[nc:] = 0.0, 1.0
    A, z = orc.weights(p)
    starts = U0[:N]
    Y = np.stack([orc.fine(p, s) - orc.coarse(p, s) for s in starts])
    S = np.stack([orc.scale(p, c, r, s) for s in starts])
    Phi = np.stack([orc.features(A, z, sr) for sr in S])
    ref = [u0, orc.fine(p, u0)]
    for _ in range(2, N + 1):
        prev = ref[-1]
        rc, corr, _ = orc.predict(p, S, Y, Phi, A, z, c, r, prev)
        assert rc >= 0
        ref.append(orc.coarse(p, prev) + corr)
    ref = np.stack(ref)
    with R.Solver(R.problem(cfg, precision="fp64", max_pairs=N)) as s:
        s.set_scaling(c[None], r[None])
        s.randnet_fit(dev(starts[None]), dev(Y[None]))
        U = host(s.coarse_sweep(1, dev(ref[1][None])))[0]
    for i in range(1, N + 1):
        e = np.abs(U[i] - ref[i]).max() / np.abs(ref[i]).max()
        assert e <= 1e-10, (i, e)
