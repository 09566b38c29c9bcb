"""rnp_randnet_predict_noalloc, the prediction entry point that allocates no
device memory (for callers that cannot allocate when they predict), checked
through the C ABI against rnp_randnet_predict on two calls in a row, at the
tolerance of the other prediction tests (1e-10 relative).  This file is
collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-10


def test_noalloc_prediction_matches_the_context_prediction():
    import torch
    import paper_2411_06225_gb300 as rnp
    rnp.build()
    L = rnp.lib()
    cfg = W.config("diffreact2d", nx=40, ny=36, M=64, m=4)
    B, P, d = 1, 9, W.dim(cfg)
    rng = np.random.default_rng(21)
    Uin = rng.standard_normal((B, P, d))
    Y = rng.standard_normal((B, P, d))
    Uin[:, 3] = Uin[:, 1]
    Y[:, 3] = Y[:, 1]
    queries = [Uin[:, 2] + 1e-3 * rng.standard_normal((B, d)), Uin[:, 5] + 1e-2 * rng.standard_normal((B, d))]
    c = np.array([[0.25, -0.5, 0.0]])
    r = np.array([[2.0, 3.0, 1.0]])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    prob = rnp.problem(cfg, max_pairs=P + 4)
    with rnp.Solver(prob) as s:
        s.set_scaling(c, r)
        s.randnet_fit(dev(Uin), dev(Y))
        refs = [s.randnet_predict(dev(q)).cpu().numpy()[0] for q in queries]
        A, z = s.weights()
    n = d // 2
    Ut = dev(Uin[0])
    S = torch.cat([(Ut[:, :n] - c[0, 0]) / r[0, 0], (Ut[:, n:] - c[0, 1]) / r[0, 1]], dim=1).contiguous()
    Phi = torch.clamp(S @ A.T + z, min=0.0).contiguous()
    Yd = dev(Y[0])
    ch = (C.c_double * 3)(*c[0])
    rh = (C.c_double * 3)(*r[0])
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    p = C.c_void_p
    for q, ref in zip(queries, refs):      # two calls in a row, shared scratch
        out = torch.full((d,), float("nan"), dtype=torch.float64, device="cuda")
        qd = dev(q[0])
        rc = L.rnp_randnet_predict_noalloc(
            C.byref(prob), p(A.data_ptr()), p(z.data_ptr()), p(S.data_ptr()),
            p(Yd.data_ptr()), p(Phi.data_ptr()), P, ch, rh, p(qd.data_ptr()),
            p(out.data_ptr()), p(status.data_ptr()), p(stream.cuda_stream))
        assert rc == rnp.RNP_OK, L.rnp_last_error(None)
        torch.cuda.synchronize()
        assert int(status.item()) == rnp.RNP_OK
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= REL * np.abs(ref).max()
    # sizes beyond the fixed scratch are refused before any work
    rc = L.rnp_randnet_predict_noalloc(
        C.byref(prob), p(A.data_ptr()), p(z.data_ptr()), p(S.data_ptr()), p(Yd.data_ptr()),
        p(Phi.data_ptr()), 5000, ch, rh, p(qd.data_ptr()), p(out.data_ptr()), None,
        p(stream.cuda_stream))
    assert rc == rnp.RNP_EINVAL
    assert b"scratch" in L.rnp_last_error(None)
