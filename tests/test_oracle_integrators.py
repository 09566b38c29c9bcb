"""Pins for the oracle's right-hand sides h(u) (Eq. 1) and its integrators
F = RK4, G = forward Euler (Sec. 2, Tables 4-7).

Pins: closed-form Fourier solutions of the discrete linear operators
(RK4/Euler amplification polynomials), convergence orders in time and space,
conservation laws, exact steady states, the ODE reached by spatially uniform
states (against scipy's DOP853), the characteristic solution of inviscid
Burgers, and first-order consistency of the shallow-water flux with the PDE
(against sympy's analytic divergence)."""
import math

import numpy as np
import pytest

import workloads as W


def _cfg(pde, nx, ny=1, nz=1, L=1.0, param=(0.1,), **kw):
    c = dict(pde=pde, nx=nx, ny=ny, nz=nz, lx=L, ly=L, lz=L, param=list(param),
             t0=0.0, tN=1.0, N=1, nF=1, nG=1, M=4, m=2, lam=1e-7, tol=1e-6,
             seed=1, batch=1, ic="sine")
    c.update(kw)
    return c


def R4(z):
    return 1 + z + z * z / 2 + z**3 / 6 + z**4 / 24


def _heat_mode(orc, dims, n, k, D=0.1):
    cfg = _cfg("heat", n, n if dims >= 2 else 1, n if dims >= 3 else 1,
               param=(D,), mode=k)
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    h = 1.0 / n
    lam = dims * (-4.0 * D / h**2) * math.sin(math.pi * k / n) ** 2
    return p, u0, lam


@pytest.mark.parametrize("dims", [1, 2, 3])
def test_heat_mode_rk4_closed_form(orc, dims):
    n = {1: 64, 2: 32, 3: 12}[dims]
    p, u0, lam = _heat_mode(orc, dims, n, 3)
    dt, steps = 2e-4, 50
    u = orc.rk4(p, u0, dt, steps)
    exact = R4(dt * lam) ** steps * u0
    assert np.abs(u - exact).max() < 1e-13


@pytest.mark.parametrize("dims", [1, 2])
def test_heat_mode_euler_closed_form(orc, dims):
    n = 32
    p, u0, lam = _heat_mode(orc, dims, n, 5)
    dt, steps = 1e-4, 40
    u = orc.euler(p, u0, dt, steps)
    assert np.abs(u - (1 + dt * lam) ** steps * u0).max() < 1e-13


def test_rk4_is_fourth_order_in_time(orc):
    p, u0, lam = _heat_mode(orc, 1, 32, 2)
    T = 0.05
    errs = []
    for steps in (8, 16, 32):
        u = orc.rk4(p, u0, T / steps, steps)
        errs.append(np.abs(u - math.exp(lam * T) * u0).max())
    for a, b in zip(errs, errs[1:]):
        assert 14.0 < a / b < 18.0


def test_laplacian_is_second_order_in_space(orc):
    # discrete eigenvalue vs the PDE's -D (2 pi k)^2
    D, k = 0.1, 3
    errs = []
    for n in (32, 64, 128):
        p, u0, lam = _heat_mode(orc, 1, n, k, D)
        lam_num = (orc.rhs(p, u0) @ u0) / (u0 @ u0)
        assert abs(lam_num - lam) < 1e-9 * abs(lam)
        errs.append(abs(lam - (-D * (2 * math.pi * k) ** 2)))
    for a, b in zip(errs, errs[1:]):
        assert 3.8 < a / b < 4.2


def test_advection_mode_closed_form(orc):
    n, k, c = 64, 4, 0.7
    cfg = _cfg("advect1d", n, param=(c,), mode=k)
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    h = 1.0 / n
    theta = 2 * math.pi * k / n
    lam = -1j * c * math.sin(theta) / h
    dt, steps = 1e-3, 200
    u = orc.rk4(p, u0, dt, steps)
    exact = np.imag(R4(dt * lam) ** steps * np.exp(1j * theta * np.arange(n)))
    assert np.abs(u - exact).max() < 1e-12


def _burgers(orc, nx, nu):
    cfg = W.config("burgers1d", nx=nx, param=[nu])
    return orc.problem(cfg)


def test_burgers_conserves_mass(orc):
    p = _burgers(orc, 128, 0.01)
    u0 = W.initial_condition(W.config("burgers1d"))[0]
    u = orc.rk4(p, u0, 1e-3, 500)
    assert abs(u.sum() - u0.sum()) < 1e-12 * max(1.0, np.abs(u0).sum())
    assert np.abs(u - u0).max() > 1e-3  # it did evolve


def test_burgers_small_amplitude_is_heat(orc):
    n, nu, eps = 64, 0.05, 1e-7
    p = _burgers(orc, n, nu)
    x = -1.0 + 2.0 * np.arange(n) / n
    u0 = eps * np.sin(np.pi * x)
    h = 2.0 / n
    lam = -4.0 * nu / h**2 * math.sin(math.pi / n) ** 2
    dt, steps = 1e-3, 300
    u = orc.rk4(p, u0, dt, steps)
    lin = R4(dt * lam) ** steps * u0
    assert np.abs(u - lin).max() < 1e-5 * eps


def _characteristics(x, t):
    # v(x,t) = v0(xi), x = xi + v0(xi) t, v0 = 0.5 + 0.25 sin(pi xi)
    xi = x - (0.5 + 0.25 * np.sin(np.pi * x)) * t
    for _ in range(60):
        f = xi + (0.5 + 0.25 * np.sin(np.pi * xi)) * t - x
        fp = 1 + 0.25 * np.pi * np.cos(np.pi * xi) * t
        xi = xi - f / fp
    return 0.5 + 0.25 * np.sin(np.pi * xi)


def test_inviscid_burgers_matches_characteristics(orc):
    T = 0.4  # shock time is 4 / pi ~ 1.27
    errs = []
    for n in (128, 256):
        p = _burgers(orc, n, 0.0)
        x = -1.0 + 2.0 * np.arange(n) / n
        u0 = 0.5 + 0.25 * np.sin(np.pi * x)
        steps = 400
        u = orc.rk4(p, u0, T / steps, steps)
        errs.append(np.abs(u - _characteristics(x, T)).max())
    assert errs[1] < 2e-4
    assert 3.5 < errs[0] / errs[1] < 4.5


def _ode_ref(f, y0, T):
    from scipy.integrate import solve_ivp
    r = solve_ivp(f, (0.0, T), y0, method="DOP853", rtol=1e-13, atol=1e-15)
    return r.y[:, -1]


def _uniform_state(cfg, vals):
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    return np.concatenate([np.full(n, v) for v in vals])


def test_diffreact_uniform_state_is_the_fitzhugh_nagumo_ode(orc):
    cfg = W.config("diffreact2d", nx=8, ny=8)
    p = orc.problem(cfg)
    c = cfg["param"][2]
    f = lambda t, y: [y[0] - y[0] ** 3 - c - y[1], y[0] - y[1]]
    y0 = [0.8, -0.3]
    T = 1.0
    ref = _ode_ref(f, y0, T)
    errs = []
    for steps in (50, 100):
        u = orc.rk4(p, _uniform_state(cfg, y0), T / steps, steps)
        n = 64
        assert np.ptp(u[:n]) == 0.0 and np.ptp(u[n:]) == 0.0
        errs.append(max(abs(u[0] - ref[0]), abs(u[n] - ref[1])))
    assert errs[1] < 1e-9
    assert 12.0 < errs[0] / errs[1] < 20.0


@pytest.mark.parametrize("name", ["bruss2d", "bruss3d"])
def test_brusselator_uniform_state_is_the_ode(orc, name):
    cfg = W.config(name, nx=6, ny=6, nz=6 if name == "bruss3d" else 1)
    p = orc.problem(cfg)
    a, b = cfg["param"][0], cfg["param"][1]
    f = lambda t, y: [a - (1 + b) * y[0] + y[1] * y[0] ** 2, b * y[0] - y[1] * y[0] ** 2]
    y0 = [1.3, 2.1]
    T = 0.5
    ref = _ode_ref(f, y0, T)
    u = orc.rk4(p, _uniform_state(cfg, y0), T / 200, 200)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    assert abs(u[0] - ref[0]) < 1e-10 and abs(u[n] - ref[1]) < 1e-10


@pytest.mark.parametrize("name", ["bruss2d", "bruss3d"])
def test_brusselator_steady_state_is_exact(orc, name):
    cfg = W.config(name, nx=5, ny=5, nz=5 if name == "bruss3d" else 1)
    p = orc.problem(cfg)
    a, b = cfg["param"][0], cfg["param"][1]
    u0 = _uniform_state(cfg, [a, b / a])
    assert np.all(orc.rhs(p, u0) == 0.0)
    assert np.array_equal(orc.rk4(p, u0, 1e-2, 10), u0)


def test_swe_lake_at_rest_is_exact(orc):
    cfg = W.config("swe2d", nx=16, ny=16)
    p = orc.problem(cfg)
    u0 = _uniform_state(cfg, [1.7, 0.0, 0.0])
    assert np.all(orc.rhs(p, u0) == 0.0)


def test_swe_conserves_mass_and_momentum_and_symmetry(orc):
    cfg = W.config("swe2d", nx=32, ny=32)
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    u = orc.rk4(p, u0, 0.1 * (1 / 32) / 4, 100)
    n = 32 * 32
    for q in range(3):
        assert abs(u[q * n:(q + 1) * n].sum() - u0[q * n:(q + 1) * n].sum()) < 1e-11 * n
    h = u[:n].reshape(32, 32)
    hu = u[n:2 * n].reshape(32, 32)
    hv = u[2 * n:].reshape(32, 32)
    # the centred radial bump is symmetric under x <-> y
    assert np.abs(h - h.T).max() < 1e-13
    assert np.abs(hu - hv.T).max() < 1e-13
    assert np.abs(h - u0[:n].reshape(32, 32)).max() > 1e-4


def test_swe_flux_is_first_order_consistent_with_the_pde(orc):
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    g = 9.81
    H = 1 + sp.Rational(1, 10) * sp.sin(2 * sp.pi * x) * sp.cos(2 * sp.pi * y)
    QX = sp.Rational(1, 5) + sp.Rational(1, 20) * sp.cos(2 * sp.pi * x)
    QY = sp.Rational(1, 10) + sp.Rational(1, 20) * sp.sin(2 * sp.pi * y)
    rhs = [
        -sp.diff(QX, x) - sp.diff(QY, y),
        -sp.diff(QX**2 / H + g * H**2 / 2, x) - sp.diff(QX * QY / H, y),
        -sp.diff(QX * QY / H, x) - sp.diff(QY**2 / H + g * H**2 / 2, y),
    ]
    fs = [sp.lambdify((x, y), e, "numpy") for e in (H, QX, QY)]
    rs = [sp.lambdify((x, y), e, "numpy") for e in rhs]
    errs = []
    for n in (64, 128, 256):
        cfg = W.config("swe2d", nx=n, ny=n)
        p = orc.problem(cfg)
        X, Y = np.meshgrid(np.arange(n) / n, np.arange(n) / n)
        u = np.concatenate([np.broadcast_to(f(X, Y), (n, n)).ravel() for f in fs])
        out = orc.rhs(p, u)
        ex = np.concatenate([np.broadcast_to(r(X, Y), (n, n)).ravel() for r in rs])
        errs.append(np.abs(out - ex).max())
    for a, b in zip(errs, errs[1:]):
        assert 1.7 < a / b < 2.3
