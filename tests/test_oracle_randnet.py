"""Pins for the oracle's RandNet pieces: Eq. HA (features), App. B (m nearest
neighbours with ties), Eq. ridgeless (readout, dual vs primal vs the
pseudo-inverse limit), the Cholesky solve and the per-species rescaling of
Alg. 1/Alg. 3.  References are numpy/scipy library routines, brute force and
closed forms."""
import numpy as np
import pytest

import workloads as W


def test_features_are_relu_of_affine_map(orc):
    rng = np.random.default_rng(0)
    M, d = 37, 513
    A = rng.uniform(-1, 1, (M, d))
    z = rng.uniform(-1, 1, M)
    s = rng.uniform(-1, 1, d)
    ref = np.maximum(A @ s + z, 0.0)
    phi = orc.features(A, z, s)
    assert np.abs(phi - ref).max() < 1e-12 * max(1.0, np.abs(A @ s).max())
    assert np.all(phi >= 0) and np.any(phi == 0) and np.any(phi > 0)


def test_scaling_maps_each_species_onto_minus1_1(orc):
    cfg = W.config("diffreact2d", nx=8, ny=8)
    p = orc.problem(cfg)
    rng = np.random.default_rng(1)
    U = rng.normal(size=(5, 128))
    U[:, 64:] = 3.0 + 0.1 * U[:, 64:]
    c, r = orc.scaling(p, U)
    for q, sl in enumerate((slice(0, 64), slice(64, 128))):
        lo, hi = U[:, sl].min(), U[:, sl].max()
        s_lo = orc.scale(p, c, r, np.full(128, lo))[sl]
        s_hi = orc.scale(p, c, r, np.full(128, hi))[sl]
        assert np.allclose(s_lo, -1.0, atol=1e-15) and np.allclose(s_hi, 1.0, atol=1e-15)
    # a constant species keeps r = 1
    U2 = np.ones((3, 128))
    c2, r2 = orc.scaling(p, U2)
    assert r2[0] == 1.0 and c2[0] == 1.0
    p_none = orc.problem(cfg, scale="none")
    c3, r3 = orc.scaling(p_none, U)
    assert np.all(c3[:2] == 0.0) and np.all(r3[:2] == 1.0)


def test_nearest_neighbours_brute_force_with_ties(orc):
    rng = np.random.default_rng(2)
    P, d, m = 40, 17, 6
    S = rng.integers(-2, 3, (P, d)).astype(np.float64)
    S[7] = S[3]
    S[20] = S[3]
    S[33] = S[11]
    for trial in range(20):
        q = S[rng.integers(P)] + rng.integers(-1, 2, d) * (trial % 2)
        dist = ((S - q) ** 2).sum(axis=1)
        order = np.lexsort((np.arange(P), dist))[:m]
        idx, dd = orc.nn(S, q, m)
        assert np.array_equal(idx, order)
        assert np.array_equal(dd, dist[order])


def test_nearest_neighbours_fewer_points_than_m(orc):
    S = np.arange(6, dtype=np.float64).reshape(3, 2)
    idx, _ = orc.nn(S, np.array([4.0, 5.0]), 5)
    assert list(idx) == [2, 1, 0]
    idx0, _ = orc.nn(np.zeros((0, 2)), np.zeros(2), 4)
    assert idx0.size == 0


def test_cholesky_solve_matches_numpy(orc):
    rng = np.random.default_rng(3)
    for n in (1, 2, 4, 9):
        B = rng.normal(size=(n, n))
        K = B @ B.T + n * np.eye(n)
        b = rng.normal(size=n)
        rc, x = orc.cholesky_solve(K, b)
        assert rc == 0
        assert np.abs(x - np.linalg.solve(K, b)).max() < 1e-12
    rc, _ = orc.cholesky_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2))
    assert rc == -1


def test_ridge_dual_equals_primal(orc):
    # push-through identity: Y^T (X X^T + l I_m)^{-1} X phi = W^T phi with
    # W = (X^T X + l I_M)^{-1} X^T Y  (Eq. ridgeless, any l > 0)
    rng = np.random.default_rng(4)
    m, M, d = 3, 5, 4
    X = rng.uniform(0, 1, (m, M))
    Y = rng.normal(size=(m, d))
    phiq = rng.uniform(0, 1, M)
    for lam in (1e-3, 1e-1, 1.0):
        esc, alpha = orc.ridge_dual(X, phiq, lam)
        assert esc == 0
        rc, pred = orc.ridge_primal(X, Y, phiq, lam)
        assert rc == 0
        assert np.abs(alpha @ Y - pred).max() < 1e-10 * np.abs(pred).max()
        Wn = np.linalg.solve(X.T @ X + lam * np.eye(M), X.T @ Y)
        assert np.abs(Wn.T @ phiq - pred).max() < 1e-10 * np.abs(pred).max()


def test_ridgeless_limit_is_the_pseudo_inverse(orc):
    rng = np.random.default_rng(5)
    m, M, d = 4, 100, 6
    X = np.maximum(rng.uniform(-1, 1, (m, M)) * 5, 0)
    Y = rng.normal(size=(m, d))
    phiq = np.maximum(rng.uniform(-1, 1, M) * 5, 0)
    esc, alpha = orc.ridge_dual(X, phiq, 1e-9)
    assert esc == 0
    W_pinv = np.linalg.pinv(X) @ Y               # min-norm least squares
    ref = W_pinv.T @ phiq
    assert np.abs(alpha @ Y - ref).max() < 1e-7 * np.abs(ref).max()
    lst = np.linalg.lstsq(X, Y, rcond=None)[0]
    assert np.abs(lst.T @ phiq - ref).max() < 1e-9 * np.abs(ref).max()


def test_ridgeless_interpolates_the_training_targets(orc):
    rng = np.random.default_rng(6)
    m, M, d = 4, 100, 9
    X = np.maximum(rng.uniform(-1, 1, (m, M)) * 3, 0)
    Y = rng.normal(size=(m, d))
    for l in range(m):
        esc, alpha = orc.ridge_dual(X, X[l], 1e-10)
        assert np.abs(alpha @ Y - Y[l]).max() < 1e-8


def test_ridge_failure_after_escalations(orc):
    X = np.zeros((3, 4))
    esc, _ = orc.ridge_dual(X, np.ones(4), 0.0)
    assert esc == -1
    # a duplicated row is rescued by the penalty itself; the query equals the
    # duplicated row, so the interpolant puts total weight 1 on it
    X = np.array([[1.0, 2.0, 0.0], [1.0, 2.0, 0.0], [0.0, 1.0, 1.0]])
    esc, alpha = orc.ridge_dual(X, np.array([1.0, 2.0, 0.0]), 1e-7)
    assert esc == 0
    assert abs(alpha[0] + alpha[1] - 1.0) < 1e-6 and abs(alpha[2]) < 1e-6


def test_prediction_is_the_composition_of_the_pieces(orc):
    cfg = W.config("diffreact2d", nx=6, ny=6, M=30, m=4, lam=1e-7)
    p = orc.problem(cfg)
    d = 72
    rng = np.random.default_rng(7)
    P = 11
    U = rng.normal(size=(P, d))
    c, r = np.array([0.1, -0.2, 0.0]), np.array([2.0, 3.0, 1.0])
    A, z = orc.weights(p)
    S = np.stack([orc.scale(p, c, r, u) for u in U])
    Y = rng.normal(size=(P, d))
    Phi = np.maximum(S @ A.T + z, 0)
    q = U[4] + 0.01 * rng.normal(size=d)
    rc, out, nnv = orc.predict(p, S, Y, Phi, A, z, c, r, q)
    assert rc == 0
    sq = np.concatenate([(q[:36] - c[0]) / r[0], (q[36:] - c[1]) / r[1]])
    dist = ((S - sq) ** 2).sum(1)
    order = np.lexsort((np.arange(P), dist))[:4]
    assert np.array_equal(nnv[:4], order)
    X = Phi[order]
    phiq = np.maximum(A @ sq + z, 0)
    alpha = np.linalg.solve(X @ X.T + 1e-7 * np.eye(4), X @ phiq)
    ref = alpha @ Y[order]
    assert np.abs(out - ref).max() < 1e-6 * np.abs(ref).max()
