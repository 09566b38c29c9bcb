"""Pins for the oracle's no-flux (homogeneous Neumann, finite-volume)
boundary (Sec. 5.2: no-flow Neumann boundary on a finite-volume grid).

On a cell-centred grid x_i = (i + 1/2) h, i = 0..n-1, the no-flux
second difference (the wall neighbour is the cell itself) has the cosine
eigenvectors cos(pi k x_i / L) with eigenvalues -(4/h^2) sin^2(pi k h / 2L),
k = 0..n-1 -- a mode that the periodic operator does not have for odd k.
Pins: the RK4 / Euler closed forms of such modes (1D, 2D, 3D), exact mass
conservation of the diffusion operator, the boundary stencil itself, the
Burgers/advection wall differences.  Shallow-water walls (reflecting) are
pinned in test_oracle_swe_box.py."""
import math

import numpy as np
import pytest

import workloads as W


def R4(z):
    return 1 + z + z * z / 2 + z**3 / 6 + z**4 / 24


def _cfg(pde, nx, ny=1, nz=1, L=1.0, param=(0.1,), **kw):
    c = dict(pde=pde, nx=nx, ny=ny, nz=nz, lx=L, ly=L, lz=L, param=list(param),
             t0=0.0, tN=1.0, N=1, nF=1, nG=1, M=4, m=2, lam=1e-7, tol=1e-6,
             seed=1, batch=1, ic="sine", bc="neumann")
    c.update(kw)
    return c


def _cos_mode(n, k, L=1.0):
    x = (np.arange(n) + 0.5) * (L / n)
    return np.cos(math.pi * k * x / L)


def _lam(n, k, D, L=1.0):
    h = L / n
    return -(4.0 * D / h**2) * math.sin(math.pi * k * h / (2.0 * L)) ** 2


@pytest.mark.parametrize("dims,k", [(1, 3), (1, 1), (2, 5), (3, 3)])
def test_cosine_mode_rk4_closed_form(orc, dims, k):
    n = {1: 48, 2: 24, 3: 10}[dims]
    D = 0.1
    cfg = _cfg("heat", n, n if dims >= 2 else 1, n if dims >= 3 else 1, param=(D,))
    p = orc.problem(cfg)
    f = _cos_mode(n, k)
    u0 = f
    if dims >= 2:
        u0 = np.multiply.outer(f, f)           # (y, x)
    if dims >= 3:
        u0 = np.multiply.outer(f, np.multiply.outer(f, f))
    u0 = u0.ravel()
    lam = dims * _lam(n, k, D)
    dt, steps = 2e-4, 40
    u = orc.rk4(p, u0, dt, steps)
    assert np.abs(u - R4(dt * lam) ** steps * u0).max() < 1e-13
    # the same odd mode is not an eigenvector of the periodic operator
    if k % 2 == 1:
        up = orc.rk4(orc.problem(dict(cfg, bc="periodic")), u0, dt, steps)
        assert np.abs(up - R4(dt * lam) ** steps * u0).max() > 1e-6


def test_cosine_mode_euler_closed_form(orc):
    n, k, D = 40, 7, 0.05
    p = orc.problem(_cfg("heat", n, param=(D,)))
    u0 = _cos_mode(n, k)
    dt, steps = 1e-4, 30
    u = orc.euler(p, u0, dt, steps)
    assert np.abs(u - (1 + dt * _lam(n, k, D)) ** steps * u0).max() < 1e-13


def test_wall_stencil(orc):
    # h(u) at the wall cells is D (u_1 - u_0) / h^2 and D (u_{n-2} - u_{n-1}) / h^2
    n, D = 16, 0.3
    p = orc.problem(_cfg("heat", n, param=(D,)))
    u = np.random.default_rng(3).standard_normal(n)
    r = orc.rhs(p, u)
    h2 = (1.0 / n) ** 2
    assert r[0] == pytest.approx(D * (u[1] - u[0]) / h2, rel=1e-14)
    assert r[-1] == pytest.approx(D * (u[-2] - u[-1]) / h2, rel=1e-14)
    assert r[5] == pytest.approx(D * (u[6] - 2 * u[5] + u[4]) / h2, rel=1e-12)


@pytest.mark.parametrize("pde,shape,param", [
    ("heat", (20, 1, 1), (0.2,)),
    ("heat", (12, 10, 1), (0.2,)),
    ("heat", (6, 5, 4), (0.2,)),
    ("diffreact2d", (12, 9, 1), (1e-3, 5e-3, 0.0)),
])
def test_diffusion_conserves_mass(orc, pde, shape, param):
    # the no-flux operator moves mass between cells only: sum(h(u)) = 0 for
    # pure diffusion (diffusion-reaction with the reaction's u - u^3 - v and
    # u - v parts removed by testing the u - v symmetric combination below)
    nx, ny, nz = shape
    cfg = _cfg(pde, nx, ny, nz, L=2.0, param=param)
    p = orc.problem(cfg)
    n = nx * ny * nz
    rng = np.random.default_rng(5)
    if pde == "heat":
        u = rng.standard_normal(n)
        r = orc.rhs(p, u)
        assert abs(r.sum()) < 1e-9 * np.abs(r).max() * n
    else:
        # with u = v everywhere the reaction parts are u - u^3 - c - u and 0
        a = rng.uniform(-1, 1, n)
        u = np.concatenate([a, a])
        r = orc.rhs(p, u)
        assert abs(r[n:].sum()) < 1e-9 * np.abs(r[n:]).max() * n
        assert np.allclose(r[:n].sum(), (-(a ** 3) - param[2]).sum(), rtol=1e-9)


def test_burgers_wall_differences(orc):
    n, nu = 16, 0.01
    p = orc.problem(_cfg("burgers1d", n, L=2.0, param=(nu,)))
    u = np.random.default_rng(7).standard_normal(n)
    r = orc.rhs(p, u)
    h = 2.0 / n
    exp0 = nu * (u[1] - u[0]) / h**2 - u[0] * ((u[1] - u[0]) * (0.5 / h))
    expn = nu * (u[-2] - u[-1]) / h**2 - u[-1] * ((u[-1] - u[-2]) * (0.5 / h))
    assert r[0] == pytest.approx(exp0, rel=1e-13)
    assert r[-1] == pytest.approx(expn, rel=1e-13)

