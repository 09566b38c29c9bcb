"""Pins for the oracle's shallow water in a box (Sec. 5.3 and its appendix:
a box whose walls the water rebounds from, and the bottom term -g h grad b).

* Method of images: a reflecting wall is a mirror.  The wall problem on an
  nx x ny box equals, bit for bit, the periodic problem on the 2nx x 2ny
  domain holding the state reflected across both walls (h, hv and b even,
  hu odd across x-walls; hu even, hv odd across y-walls), for the
  right-hand side and for F.  The periodic operator is pinned elsewhere, so
  a wrong ghost cell, sign or bottom difference at a wall fails here.
* Walls conserve mass: the sum of h is constant over many RK4 steps.
* The bottom term: water at rest over a linear bottom b = s x (or s y) has
  dh/dt = 0 and d(hu)/dt = -g h s (half that in a wall cell, where the
  bottom's neighbour across the wall is the cell itself).
* Still water over a flat bottom stays still; a solve with eps = 0
  reproduces the serial fine solution."""
import numpy as np
import pytest

import workloads as W


def _box(nx, ny, lx=2.0, ly=1.0, bc="neumann", bathymetry=None, **kw):
    c = dict(pde="swe2d", nx=nx, ny=ny, nz=1, lx=lx, ly=ly, lz=1.0, param=[9.81], t0=0.0,
             tN=0.02, N=2, nF=8, nG=2, M=8, m=2, lam=1e-7, tol=1e-6, seed=5, batch=1,
             ic="gauss_bump", bc=bc)
    if bathymetry is not None:
        c["bathymetry"] = bathymetry
    c.update(kw)
    return c


def _state(nx, ny, seed):
    rng = np.random.default_rng(seed)
    h = 1.0 + 0.5 * rng.random((ny, nx))
    hu = 0.3 * rng.standard_normal((ny, nx))
    hv = 0.3 * rng.standard_normal((ny, nx))
    return h, hu, hv


def _mirror(a, sx, sy):
    """Reflect an (ny, nx) field across x = L and y = L: (2ny, 2nx)."""
    ax = np.concatenate([a, sx * a[:, ::-1]], axis=1)
    return np.concatenate([ax, sy * ax[::-1, :]], axis=0)


def _flat(*fields):
    return np.concatenate([f.reshape(-1) for f in fields])


@pytest.mark.parametrize("nx,ny,with_b", [(8, 6, False), (9, 7, True), (16, 5, True)])
def test_wall_is_a_mirror(orc, nx, ny, with_b):
    h, hu, hv = _state(nx, ny, nx * ny)
    b = None
    if with_b:
        b = 0.2 * np.random.default_rng(3).random((ny, nx))
    pw = orc.problem(_box(nx, ny, bathymetry=b))
    pp = orc.problem(_box(2 * nx, 2 * ny, lx=4.0, ly=2.0, bc="periodic",
                          bathymetry=None if b is None else _mirror(b, 1, 1)))
    sw = _flat(h, hu, hv)
    sp = _flat(_mirror(h, 1, 1), _mirror(hu, -1, 1), _mirror(hv, 1, -1))
    n2 = 4 * nx * ny

    def restrict(v):
        return _flat(*[v[q * n2:(q + 1) * n2].reshape(2 * ny, 2 * nx)[:ny, :nx]
                       for q in range(3)])

    assert np.array_equal(orc.rhs(pw, sw), restrict(orc.rhs(pp, sp)))
    assert np.array_equal(orc.rk4(pw, sw, 1e-3, 12), restrict(orc.rk4(pp, sp, 1e-3, 12)))
    # the periodic operator on the box itself is different (the walls matter)
    pb = orc.problem(_box(nx, ny, bc="periodic", bathymetry=b))
    assert not np.array_equal(orc.rhs(pw, sw), orc.rhs(pb, sw))


def test_walls_conserve_mass(orc):
    nx, ny = 24, 12
    cfg = _box(nx, ny)
    p = orc.problem(cfg)
    h, hu, hv = _state(nx, ny, 1)
    s = _flat(h, hu, hv)
    out = orc.rk4(p, s, 2e-3, 200)
    n = nx * ny
    assert abs(out[:n].sum() - s[:n].sum()) <= 1e-12 * s[:n].sum()
    assert not np.allclose(out, s)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_bottom_slope_closed_form(orc, axis):
    nx, ny, lx, ly, g, slope, depth = 12, 10, 3.0, 2.0, 9.81, 0.05, 1.3
    x = (np.arange(nx) + 0.5) * (lx / nx)
    y = (np.arange(ny) + 0.5) * (ly / ny)
    X, Y = np.meshgrid(x, y)
    b = slope * (X if axis == "x" else Y)
    p = orc.problem(_box(nx, ny, lx=lx, ly=ly, bathymetry=b))
    n = nx * ny
    s = _flat(np.full((ny, nx), depth), np.zeros((ny, nx)), np.zeros((ny, nx)))
    r = orc.rhs(p, s)
    assert np.all(r[:n] == 0.0)
    q_on, q_off = (1, 2) if axis == "x" else (2, 1)
    assert np.all(r[q_off * n:(q_off + 1) * n] == 0.0)
    got = r[q_on * n:(q_on + 1) * n].reshape(ny, nx)
    want = np.full((ny, nx), -g * depth * slope)
    if axis == "x":
        want[:, 0] *= 0.5
        want[:, -1] *= 0.5
    else:
        want[0, :] *= 0.5
        want[-1, :] *= 0.5
    assert np.allclose(got, want, rtol=1e-12, atol=0)


def test_still_water_stays_still(orc):
    nx, ny = 10, 6
    p = orc.problem(_box(nx, ny))
    s = _flat(np.full((ny, nx), 2.0), np.zeros((ny, nx)), np.zeros((ny, nx)))
    assert np.all(orc.rhs(p, s) == 0.0)


def test_bathymetry_only_for_shallow_water(orc):
    cfg = W.config("diffreact2d", nx=8, ny=8, N=2, nF=2, nG=1)
    cfg["bathymetry"] = np.zeros((8, 8))
    rc, _, _, _ = orc.solve(orc.problem(cfg), W.initial_condition(cfg)[0])
    assert rc == 1  # ORC_EINVAL


def test_box_solve_tol0_is_serial_fine(orc):
    nx, ny = 12, 8
    b = 0.1 * np.random.default_rng(9).random((ny, nx))
    cfg = _box(nx, ny, bathymetry=b, N=4, nF=6, nG=2, tol=0.0, tN=0.05, ic="gauss_column")
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    rc, U, st, _ = orc.solve(p, u0)
    assert st.K == cfg["N"]
    assert np.array_equal(U, orc.serial_fine(p, u0))
