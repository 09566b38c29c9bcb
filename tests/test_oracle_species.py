"""Pins for which diffusion coefficient multiplies which species' Laplacian
in the oracle's two-species right-hand sides.

Sec. 5.2 writes the diffusion-reaction system as u_t = D_u lap u + R_u(u, v),
v_t = D_v lap v + R_v(u, v) (D_u for the activator u, D_v for the inhibitor
v); App. E writes the Brusselator as u_t = D_0 lap u + ..., v_t = D_1 lap v
+ ....  The workloads store the coefficients as param = [Du, Dv, c] and
[a, b, D0, D1].

The reaction terms act point by point, so around a spatially uniform state
the linear response of h(u) to a perturbation of species q has the same
reaction part for every perturbation shape: only the diffusion part tells
shapes apart.  For an eigenvector phi of the discrete Laplacian (eigenvalue
lam, closed form), the response to eps * phi in species q minus phi times
the response to eps * 1 in species q is therefore lam * D_q * phi in
species q and zero in the other species.  Responses are central differences
of h(u), exact up to eps^2 times the reaction's third derivative.  A swap of
the two coefficients, or a Laplacian taken of the wrong species, fails
these tests (the uniform-state tests of the reaction ODE cannot see it: the
Laplacian of a uniform state is zero).
"""
import math

import numpy as np
import pytest

import workloads as W

EPS = 1e-4


def _mode(cfg, k):
    """cos(2 pi k x / n) along every axis with more than one point, and the
    eigenvalue of the periodic second-difference Laplacian for it."""
    f = np.ones((cfg["nz"], cfg["ny"], cfg["nx"]))
    lam = 0.0
    for axis, (n, L) in enumerate(((cfg["nz"], cfg["lz"]), (cfg["ny"], cfg["ly"]),
                                   (cfg["nx"], cfg["lx"]))):
        if n == 1:
            continue
        h = L / n
        shape = [1, 1, 1]
        shape[axis] = n
        f = f * np.cos(2.0 * math.pi * k * np.arange(n) / n).reshape(shape)
        lam += -4.0 / (h * h) * math.sin(math.pi * k / n) ** 2
    return f.ravel(), lam


def _response(orc, p, base, q, shape):
    n = shape.size
    pert = np.zeros_like(base)
    pert[q * n:(q + 1) * n] = shape
    return (orc.rhs(p, base + EPS * pert) - orc.rhs(p, base - EPS * pert)) / (2.0 * EPS)


CASES = [
    # name, grid overrides, uniform base state, index of D_u / D_0 and D_v / D_1 in param
    ("diffreact2d", dict(nx=8, ny=8), (0.8, -0.3), (0, 1)),
    ("bruss2d", dict(nx=8, ny=8), (1.0, 3.0), (2, 3)),
    ("bruss2d", dict(nx=8, ny=8), (1.3, 2.1), (2, 3)),
    ("bruss3d", dict(nx=6, ny=6, nz=6), (1.3, 2.1), (2, 3)),
]


@pytest.mark.parametrize("name,grid,base_vals,didx", CASES)
def test_each_species_diffuses_with_its_own_coefficient(orc, name, grid, base_vals, didx):
    cfg = W.config(name, **grid)
    p = orc.problem(cfg)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    base = np.concatenate([np.full(n, v) for v in base_vals])
    D = [cfg["param"][didx[0]], cfg["param"][didx[1]]]
    assert D[0] != D[1]
    for k in (1, 2):
        phi, lam = _mode(cfg, k)
        assert lam < 0
        for q in (0, 1):
            r_mode = _response(orc, p, base, q, phi)
            r_one = _response(orc, p, base, q, np.ones(n))
            diff = r_mode - np.concatenate([phi * r_one[:n], phi * r_one[n:]])
            own = diff[q * n:(q + 1) * n]
            other = diff[(1 - q) * n:(2 - q) * n]
            scale = abs(lam) * max(D)
            # species q diffuses with D_q ...
            assert np.abs(own - lam * D[q] * phi).max() < 1e-6 * scale, (k, q)
            # ... and its Laplacian does not enter the other species' equation
            assert np.abs(other).max() < 1e-6 * scale, (k, q)


def test_swapped_coefficients_would_be_seen(orc):
    """The pin's resolution: the two coefficients' contributions differ by
    far more than the tolerance used above, for each workload."""
    for name, grid, base_vals, didx in CASES:
        cfg = W.config(name, **grid)
        _, lam = _mode(cfg, 1)
        D = [cfg["param"][didx[0]], cfg["param"][didx[1]]]
        assert abs(lam) * abs(D[0] - D[1]) > 1e3 * 1e-6 * abs(lam) * max(D)


@pytest.mark.parametrize("name,grid,didx", [("diffreact2d", dict(nx=8, ny=8), (0, 1)),
                                            ("bruss3d", dict(nx=6, ny=6, nz=6, lx=2.0, ly=2.0, lz=2.0),
                                             (2, 3))])
def test_rk4_of_a_small_species_mode_follows_its_own_diffusion(orc, name, grid, didx):
    """Time-integrated form of the same pin.  Around a uniform steady state
    (diffusion-reaction: u = v = -c^(1/3); Brusselator: (a, b / a)) a small
    perturbation eps * phi in species q evolves, up to O(eps), under the
    2 x 2 matrix J_k = J_react + lam_k diag(D_u, D_v), and RK4 multiplies it
    by the amplification matrix R(dt J_k) = sum_{j<=4} (dt J_k)^j / j! each
    step.  J_react is measured from the uniform mode (k = 0) of h(u), so
    diag(D) enters only through lam_k: the response of RK4 pins which
    coefficient diffuses which species."""
    cfg = W.config(name, **grid)
    p = orc.problem(cfg)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    if name == "diffreact2d":
        us = -cfg["param"][2] ** (1.0 / 3.0)
        base_vals = (us, us)
    else:
        base_vals = (cfg["param"][0], cfg["param"][1] / cfg["param"][0])
    base = np.concatenate([np.full(n, v) for v in base_vals])
    assert np.abs(orc.rhs(p, base)).max() < 1e-14
    D = np.array([cfg["param"][didx[0]], cfg["param"][didx[1]]])
    Jr = np.empty((2, 2))
    for q in (0, 1):
        r = _response(orc, p, base, q, np.ones(n))
        Jr[0, q], Jr[1, q] = r[0], r[n]
    phi, lam = _mode(cfg, 1)
    Jk = Jr + lam * np.diag(D)
    dt, steps, eps = 1e-2, 40, 1e-7
    Z = dt * Jk
    R = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    Rn = np.linalg.matrix_power(R, steps)
    # with the coefficients swapped the amplification differs by far more
    # than the tolerance below
    Zs = dt * (Jr + lam * np.diag(D[::-1]))
    Rs = np.linalg.matrix_power(np.eye(2) + Zs + Zs @ Zs / 2 + Zs @ Zs @ Zs / 6
                                + Zs @ Zs @ Zs @ Zs / 24, steps)
    tol = 1e-5 * np.abs(Rn).max()
    assert np.abs(Rs - Rn).max() > 100 * tol
    fb = orc.rk4(p, base, dt, steps)
    for q in (0, 1):
        pert = np.zeros_like(base)
        pert[q * n:(q + 1) * n] = eps * phi
        du = (orc.rk4(p, base + pert, dt, steps) - fb) / eps
        for j in (0, 1):
            got = du[j * n:(j + 1) * n]
            assert np.abs(got - Rn[j, q] * phi).max() < tol, (q, j)
