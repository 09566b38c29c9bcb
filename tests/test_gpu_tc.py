"""Random features on the tensor cores (tcgen05, BF16 operands, FP32
accumulation in tensor memory) against an FP64 evaluation of the same map on
the same BF16-rounded operands, and a RandNet-Parareal solve in that
precision against the FP64 oracle.

Bounds: features within 1e-4 of the largest feature magnitude (FP32
accumulation of d <= 32768 products); the solve within 1e-5 relative of the
FP64 oracle with K within 1.  With M > 128 neurons the rows take the CUDA-core
kernel of the sweep's single queries (also with few rows, and d = 1250 not a
multiple of the 1024-element chunks)."""
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


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def bf16(a):
    """Round-to-nearest-even to BF16 (8 significant bits) straight from the
    FP64 value: one rounding (a conversion through FP32 rounds twice)."""
    b = np.ascontiguousarray(a, np.float64).view(np.uint64)
    lsb = (b >> np.uint64(45)) & np.uint64(1)
    b = (b + np.uint64(0x00000FFFFFFFFFFF) + lsb) & ~np.uint64((1 << 45) - 1)
    return b.view(np.float64)


@pytest.mark.parametrize("nx,M,rows", [(64, 100, 64), (64, 100, 37), (128, 128, 64),
                                        (40, 150, 20), (25, 150, 3), (25, 150, 19)])
def test_feature_map_on_tensor_cores(R, nx, M, rows):
    cfg = W.config("diffreact2d", nx=nx, ny=nx, M=M)
    d = W.dim(cfg)
    rng = np.random.default_rng(nx + M + rows)
    U = rng.standard_normal((rows, d))
    c = np.array([[0.1, -0.2, 0.0]])
    r = np.array([[2.5, 3.0, 1.0]])
    with R.Solver(R.problem(cfg, precision="mixed_bf16")) as s:
        s.set_scaling(c, r)
        phi = s.features(dev(U)).cpu().numpy()
        A, z = s.weights()
        A, z = A.cpu().numpy(), z.cpu().numpy()
    n = d // 2
    S = np.concatenate([(U[:, :n] - c[0, 0]) / r[0, 0], (U[:, n:] - c[0, 1]) / r[0, 1]], axis=1)
    ref = np.maximum(bf16(S.astype(np.float32).astype(np.float64)) @ bf16(A).T + z, 0.0)
    exact = np.maximum(S @ A.T + z, 0.0)
    err = np.abs(phi - ref).max()
    assert err <= 1e-4 * np.abs(ref).max(), err
    # the BF16 rounding is visible against the unrounded FP64 map
    assert np.abs(phi - exact).max() > 10 * err


def test_solve_with_tensor_core_features_against_fp64_oracle(R, orc):
    cfg = W.config("diffreact2d", nx=32, ny=32, N=16, nF=200)
    u0 = W.initial_condition(cfg)
    with R.Solver(R.problem(cfg, precision="mixed_bf16")) as s:
        U, st = s.solve(dev(u0))
        U = U.cpu().numpy()[0]
    rc, Uo, so, _ = orc.solve(orc.problem(cfg), u0[0])
    e = np.abs(U - Uo).max() / np.abs(Uo).max()
    assert abs(st["K"] - so.K) <= 1 and e <= 1e-5, (st["K"], so.K, e)
