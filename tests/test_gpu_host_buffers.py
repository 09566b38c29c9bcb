"""rnp_solve with host buffers: u0 and U in host memory (pinned or pageable)
give exactly the U and the iteration counts of the same solve in device
memory.  The library copies the start states in and sends each member's
converged states out while later iterations run, the rest at the end;
every state of U is written (U starts as NaN), also for a solve that stops
at max_iters without converging."""
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


CASES = [
    ("diffreact2d", dict(nx=32, ny=32, N=16, nF=200, batch=2), "fp64"),
    ("diffreact2d", dict(nx=32, ny=32, N=16, nF=200, batch=3), "mixed"),
    ("bruss3d", dict(nx=10, ny=10, nz=10, N=8, nF=60, nG=3, tN=0.5, batch=2), "mixed"),
    ("burgers1d", dict(), "fp64"),
]


def solve_both(R, cfg, precision, pinned, check=True):
    import torch
    B = cfg.get("batch", 1)
    u0 = np.ascontiguousarray(W.initial_condition(cfg, batch=B))
    with R.Solver(R.problem(cfg, precision=precision)) as s:
        Ud, st_d = s.solve(torch.as_tensor(u0, device="cuda"), check=check)
        Ud = Ud.cpu().numpy()
        U_h = torch.full((B, s.N + 1, s.d), float("nan"), dtype=torch.float64)
        if pinned:
            # both buffers in pinned host memory
            u0_in = torch.as_tensor(u0).pin_memory()
            U_h = U_h.pin_memory()
        else:
            # start states on the device, the result into pageable memory
            u0_in = torch.as_tensor(u0, device="cuda")
        _, st_h = s.solve(u0_in, U=U_h, check=check)
    return Ud, st_d, U_h.numpy(), st_h


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("name,kw,precision", CASES)
def test_host_buffers_give_the_device_result(R, name, kw, precision, pinned):
    cfg = W.config(name, **kw)
    Ud, st_d, Uh, st_h = solve_both(R, cfg, precision, pinned)
    assert st_h["K_each"] == st_d["K_each"]
    assert st_h["converged"] == 1
    assert not np.isnan(Uh).any()
    assert np.array_equal(Uh, Ud)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_when_max_iters_stops_the_solve(R, pinned):
    cfg = W.config("diffreact2d", nx=32, ny=32, N=16, nF=200, batch=2, max_iters=2)
    Ud, st_d, Uh, st_h = solve_both(R, cfg, "fp64", pinned, check=False)
    assert max(st_d["K_each"]) == 2
    assert st_h["converged"] == st_d["converged"]
    assert st_h["K_each"] == st_d["K_each"]
    assert not np.isnan(Uh).any()
    assert np.array_equal(Uh, Ud)


def test_binding_accepts_host_tensors_only_where_the_call_does(R):
    import torch
    cfg = W.config("burgers1d")
    with R.Solver(R.problem(cfg, precision="fp64")) as s:
        with pytest.raises(TypeError):
            s.fine_batch(torch.zeros((1, 2, s.d), dtype=torch.float64))
