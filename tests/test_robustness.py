"""The robustness study (K over m, M and weight draws): host logic on the
CPU, and on the GPU a small grid whose every K equals the FP64 oracle's K
for the same weights, m and M."""
import numpy as np
import pytest

import workloads as W
from paper_2411_06225_gb300 import robustness as R


def test_grid_and_histograms():
    pts = R.grid([2, 4], [20, 100], R.weight_seeds(3))
    assert len(pts) == 12 and len(set(pts)) == 12
    assert {s for _, _, s in pts} == {7000, 7001, 7002}
    def outcome(m, M, s):
        if s == 7002 and m == 4 and M == 100:
            return "notconv"
        return "diverged" if (s == 7001 and m == 4 and M == 20) else "converged"
    res = [(m, M, s, 3 + (m == 4) + (M == 100), outcome(m, M, s)) for m, M, s in pts]
    h = R.histograms(res)
    assert h["solves"] == 12 and h["not_converged"] == 1 and h["diverged"] == 1
    assert h["K_hist_by_m"]["2"] == {"3": 3, "4": 3}
    assert h["K_hist_by_m"]["4"] == {"4": 2, "5": 2, "nc": 1, "div": 1}
    assert list(h["K_hist_by_m"]["4"]) == ["4", "5", "nc", "div"]
    assert h["K_hist_by_M"]["100"] == {"4": 3, "5": 2, "nc": 1}
    assert h["K_min"] == 3 and h["K_max"] == 5
    assert R._range("2:21:1") == list(range(2, 21)) and R._range("20,50") == [20, 50]


def test_system_sizes():
    assert W.dim(R.system_config("burgers")) == 128
    assert W.dim(R.system_config("diffreact")) == 722


def test_paper_burgers_setting_and_fine_solvers():
    # the paper's Burgers experiment: N = 128 on [0, 5.9], G = Euler x 4;
    # with RK8 the paper's 4e4 fine steps spread over the 128 slices
    b4, b8 = R.system_config("burgers"), R.system_config("burgers", "rk8")
    assert (b4["N"], b4["tN"], b4["nG"], b4["ic"]) == (128, 5.9, 4, "cos9")
    assert (b4["fscheme"], b4["nF"]) == ("rk4", 100)
    assert (b8["fscheme"], b8["nF"]) == ("rk8", 313) and 313 * 128 >= 40000
    with pytest.raises(ValueError):
        R.system_config("burgers", "rk5")


@pytest.mark.gpu
@pytest.mark.parametrize("system", ["burgers", "diffreact"])
def test_small_grid_matches_the_oracle(orc, system):
    import paper_2411_06225_gb300 as rnp
    rnp.build()
    rnp.lib()
    pts = R.grid([2, 8], [20, 100], R.weight_seeds(2))
    res = R.run(system, pts, precision="fp64", workers=4)
    cfg = R.system_config(system)
    u0 = W.initial_condition(cfg)[0]
    orc.set_threads(8)
    for (m, M, seed, K, outcome) in res:
        p = orc.problem(dict(cfg, m=m, M=M, seed=seed))
        rc, _, so, _ = orc.solve(p, u0)
        assert rc == 0 and outcome == "converged", (m, M, seed, rc, outcome)
        assert K == so.K, (m, M, seed, K, so.K)
