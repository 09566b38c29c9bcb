"""Pins for the oracle's eighth-order fine solver (the paper's F = RK8 of
Sec. 5.1 and 5.2; here the eleven-stage explicit method of Cooper & Verner,
SIAM J. Numer. Anal. 9, 1972).

* The tableau: every one of the 200 Butcher order conditions up to order 8
  (one per rooted tree t: b . Phi(t) = 1 / gamma(t)) holds, and an order-9
  condition fails, so the coefficients are those of an order-8 method and
  a mistyped entry cannot pass.
* The stepper's use of the tableau: a Fourier mode of the periodic heat
  operator is multiplied per step by the stability function
  R(z) = 1 + z b^T (I - z A)^{-1} 1 built from the tableau alone.
* Nonlinear convergence: on Burgers the error against a much finer RK4
  solution falls by 2^8 per halving of the step.
* F over a slice is nF such steps; with eps = 0 the solve reproduces the
  serial RK8 fine solution bit for bit."""
import math

import numpy as np
import pytest

import workloads as W


def _trees(n, _cache={}):
    """All rooted trees with n nodes, each a sorted tuple of child trees."""
    if n in _cache:
        return _cache[n]
    if n == 1:
        _cache[n] = [()]
        return _cache[n]
    out = set()

    def parts(rem, maxkey):
        if rem == 0:
            yield ()
            return
        for k in range(rem, 0, -1):
            for t in _trees(k):
                key = (k, t)
                if maxkey is not None and key > maxkey:
                    continue
                for rest in parts(rem - k, key):
                    yield (t,) + rest

    for p in parts(n - 1, None):
        out.add(tuple(sorted(p)))
    _cache[n] = sorted(out)
    return _cache[n]


def _size(t):
    return 1 + sum(_size(x) for x in t)


def _gamma(t):
    g = _size(t)
    for x in t:
        g *= _gamma(x)
    return g


def _phi(A, t):
    """Elementary weight vector: 1 for the single node, else the product
    over the children of A Phi(child)."""
    v = np.ones(A.shape[0])
    for x in t:
        v = v * (A @ _phi(A, x))
    return v


def test_tree_counts():
    # number of rooted trees with n nodes (OEIS A000081)
    assert [len(_trees(n)) for n in range(1, 10)] == [1, 1, 2, 4, 9, 20, 48, 115, 286]


def test_rk8_order_conditions(orc):
    A, b, c = orc.rk8_tableau()
    assert np.allclose(A.sum(axis=1), c, rtol=0, atol=1e-14)
    assert np.all(np.triu(A) == 0)                       # explicit
    worst = 0.0
    for n in range(1, 9):
        for t in _trees(n):
            worst = max(worst, abs(b @ _phi(A, t) - 1.0 / _gamma(t)))
    assert worst < 1e-13, worst
    # order exactly 8: some order-9 condition fails
    bad9 = max(abs(b @ _phi(A, t) - 1.0 / _gamma(t)) for t in _trees(9))
    assert bad9 > 1e-6, bad9


def _heat1d(n, D, L=1.0):
    return dict(pde="heat", nx=n, ny=1, nz=1, lx=L, ly=L, lz=L, param=[D], t0=0.0,
                tN=1.0, N=1, nF=1, nG=1, M=4, m=2, lam=1e-7, tol=1e-6, seed=1,
                batch=1, ic="sine", fscheme="rk8")


@pytest.mark.parametrize("k,nsteps", [(1, 7), (5, 25), (11, 40), (15, 40)])
def test_rk8_fourier_mode(orc, k, nsteps):
    n, D, L = 32, 0.05, 1.0
    p = orc.problem(_heat1d(n, D, L))
    h = L / n
    mu = D * (2.0 * math.cos(2 * math.pi * k / n) - 2.0) / h**2
    x = np.arange(n) * h
    u0 = np.sin(2 * math.pi * k * x / L) + 0.5 * np.cos(2 * math.pi * k * x / L)
    # every mode of the grid inside the stability region (z >= -2.5), so
    # rounding noise in the other modes stays small
    dt = 2.5 / (4.0 * D / h**2)
    A, b, _ = orc.rk8_tableau()
    z = dt * mu
    R = 1.0 + z * (b @ np.linalg.solve(np.eye(11) - z * A, np.ones(11)))
    got = orc.rk8(p, u0, dt, nsteps)
    want = u0 * R**nsteps
    assert np.abs(got - want).max() <= 1e-13 * np.abs(u0).max(), np.abs(got - want).max()
    # the stability function agrees with exp(z) to eighth order
    taylor = sum(z**j / math.factorial(j) for j in range(9))
    assert abs(R - taylor) <= 1e-4 * abs(z) ** 9


def test_rk8_nonlinear_order(orc):
    cfg = W.config("burgers1d", nx=32, N=1, tN=0.25, param=[0.05], fscheme="rk8")
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    T = 0.25
    ref = orc.rk4(p, u0, T / 20000, 20000)
    errs = []
    for n in (4, 8, 16):
        errs.append(np.abs(orc.rk8(p, u0, T / n, n) - ref).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 120 < r1 < 600 and 120 < r2 < 600, (errs, r1, r2)
    # RK4 at the same steps converges by 2^4 only
    e4 = [np.abs(orc.rk4(p, u0, T / n, n) - ref).max() for n in (8, 16)]
    assert 10 < e4[0] / e4[1] < 25


def test_fine_runs_rk8(orc):
    cfg = W.config("burgers1d", nx=16, N=4, nF=30, fscheme="rk8")
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    dt = (cfg["tN"] - cfg["t0"]) / cfg["N"] / cfg["nF"]
    assert np.array_equal(orc.fine(p, u0), orc.rk8(p, u0, dt, cfg["nF"]))
    p4 = orc.problem(dict(cfg, fscheme="rk4"))
    assert not np.array_equal(orc.fine(p4, u0), orc.fine(p, u0))


def test_exact_at_zero_tolerance_rk8(orc):
    cfg = W.config("burgers1d", nx=16, N=6, nF=20, tol=0.0, fscheme="rk8")
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    rc, U, st, _ = orc.solve(p, u0)
    assert st.K == cfg["N"]
    assert np.array_equal(U, orc.serial_fine(p, u0))


@pytest.mark.parametrize("k", [1, 4, 9])
def test_rk8_noflux_cosine_mode(orc, k):
    """With no-flux walls (cell-centred grid) cos(pi k x / L) is an
    eigenvector of the heat operator with eigenvalue
    -(4 D / h^2) sin^2(pi k h / 2L); one RK8 step multiplies it by the
    tableau's stability function."""
    n, D, L = 24, 0.05, 1.0
    cfg = _heat1d(n, D, L)
    cfg["bc"] = "neumann"
    p = orc.problem(cfg)
    h = L / n
    x = (np.arange(n) + 0.5) * h
    u0 = np.cos(math.pi * k * x / L)
    lam = -(4.0 * D / h**2) * math.sin(math.pi * k * h / (2.0 * L)) ** 2
    dt = 2.5 / (4.0 * D / h**2)
    A, b, _ = orc.rk8_tableau()
    z = dt * lam
    R = 1.0 + z * (b @ np.linalg.solve(np.eye(11) - z * A, np.ones(11)))
    got = orc.rk8(p, u0, dt, 30)
    assert np.abs(got - u0 * R**30).max() <= 1e-13
