"""Pins for the oracle's Parareal driver (Alg. 1, Eq. 3, Eq. 5).

* tol = 0: no state ever passes the strict test of Eq. 5, only the exact
  leftmost slice advances, so K = N and every U_i equals the serial fine
  solution bit for bit (the K <= N remark of Sec. 2).
* G = F: the targets F - G vanish, the first sweep is already the serial
  fine solution and the iteration stops at K = 1.
* K <= N, L strictly increases, the dataset grows by N - L per iteration
  (Eq. 6 restricted to unconverged starts).
* converged error against serial F stays near tol (Table 3 reports 1e-8 to
  1e-11 for tol-converged runs).

The iterates for tol > 0 have no printed reference value: beyond these
invariants they are parity unpinned and the GPU is compared to this oracle.
"""
import numpy as np
import pytest

import workloads as W

SMALL = [
    ("burgers1d", dict(nx=32, N=6, nF=40, nG=2)),
    ("diffreact2d", dict(nx=8, ny=8, N=5, nF=20, nG=2, tN=0.5)),
    ("bruss2d", dict(nx=8, ny=8, N=5, nF=20, nG=2, tN=1.0)),
    ("bruss3d", dict(nx=4, ny=4, nz=4, N=4, nF=10, nG=2, tN=0.5, batch=1)),
    ("swe2d", dict(nx=8, ny=8, N=4, nF=20, nG=8)),
]


@pytest.mark.parametrize("corr", ["randnet", "parareal"])
@pytest.mark.parametrize("name,kw", SMALL)
def test_tol0_reproduces_serial_fine_bitwise(orc, name, kw, corr):
    cfg = W.config(name, tol=0.0, corr=corr, M=20, **kw)
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    rc, U, st, tr = orc.solve(p, u0, trace=True)
    assert rc == orc.ORC_OK
    assert st.K == cfg["N"] and st.converged
    assert list(tr["L_hist"]) == list(range(1, cfg["N"] + 1))
    assert np.array_equal(U, orc.serial_fine(p, u0))


@pytest.mark.parametrize("name,kw", SMALL[:3])
def test_G_equal_F_converges_at_first_iteration(orc, name, kw):
    cfg = W.config(name, gscheme="rk4", M=20, **kw)
    cfg["nG"] = cfg["nF"]
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    rc, U, st, _ = orc.solve(p, u0)
    assert rc == orc.ORC_OK and st.K == 1
    assert np.array_equal(U, orc.serial_fine(p, u0))


@pytest.mark.parametrize("name,kw", [
    ("burgers1d", dict()),
    ("diffreact2d", dict(nx=16, ny=16, N=12, nF=100)),
    ("bruss2d", dict(nx=16, ny=16, N=12, nF=200, nG=4, tN=2.0)),
])
def test_iteration_structure_and_accuracy(orc, name, kw):
    cfg = W.config(name, **kw)
    p = orc.problem(cfg)
    u0 = W.initial_condition(cfg)[0]
    rc, U, st, tr = orc.solve(p, u0, trace=True)
    N = cfg["N"]
    assert rc == orc.ORC_OK and st.converged and 1 <= st.K <= N
    Lh = [0] + list(tr["L_hist"])
    assert all(b > a for a, b in zip(Lh, Lh[1:])) and Lh[-1] == N
    assert st.pairs == sum(N - L for L in Lh[:-1])
    assert st.fine_cell_updates == sum(N - L for L in Lh[:-1]) * cfg["nF"] * p.nx * p.ny * p.nz * orc.lib().orc_ncomp(p)
    Us = orc.serial_fine(p, u0)
    err = np.abs(U[1:] - Us[1:]).max(axis=1)
    # Table 3 pattern: the converged error is at or below the tolerance
    assert err.mean() < cfg["tol"] and err.max() < 10 * cfg["tol"]
    # every neighbour index used refers to a pair stored at that time
    nn = tr["nn_idx"]
    assert nn.max() < st.pairs


def test_randnet_needs_fewer_iterations_than_parareal(orc):
    # Sec. 5: RandNet-Parareal converges in fewer iterations than Parareal.
    cfg = W.config("burgers1d")
    u0 = W.initial_condition(cfg)[0]
    K = {}
    for corr in ("randnet", "parareal"):
        rc, U, st, _ = orc.solve(orc.problem(cfg, corr=corr), u0)
        assert rc == orc.ORC_OK
        K[corr] = st.K
    assert K["randnet"] < K["parareal"]


def test_nonfinite_input_is_reported(orc):
    cfg = W.config("burgers1d", nx=16, N=4, nF=10, nG=2)
    u0 = W.initial_condition(cfg)[0]
    u0[3] = np.nan
    rc, *_ = orc.solve(orc.problem(cfg), u0)
    assert rc == orc.ORC_ENONFINITE


def test_max_iters_returns_not_converged(orc):
    cfg = W.config("burgers1d", max_iters=2, tol=1e-14)
    u0 = W.initial_condition(cfg)[0]
    rc, U, st, _ = orc.solve(orc.problem(cfg), u0)
    assert rc == orc.ORC_ENOTCONV and st.K == 2 and not st.converged
    assert np.all(np.isfinite(U))
