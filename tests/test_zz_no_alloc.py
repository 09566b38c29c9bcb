"""rnp_randnet_predict_noalloc, the prediction entry point that allocates no
device memory (for callers that cannot allocate when they predict), checked
through the C ABI against rnp_randnet_predict on two calls in a row, at the
tolerance of the other prediction tests (1e-10 relative), for one-, two- and
three-species states; with no stored pair the prediction is 0.  A call
after the first leaves the device's free memory unchanged.  This file is
collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-10

CASES = [
    ("diffreact2d", dict(nx=40, ny=36), 9),
    ("burgers1d", dict(nx=96), 7),
    ("swe2d", dict(nx=24, ny=20), 6),
    ("diffreact2d", dict(nx=16, ny=8), 0),
]


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name,grid,P", CASES)
def test_noalloc_prediction_matches_the_context_prediction(name, grid, P):
    import torch
    import paper_2411_06225_gb300 as rnp
    rnp.build()
    L = rnp.lib()
    cfg = W.config(name, M=64, m=4, **grid)
    nc = W.ncomp(cfg)
    B, d = 1, W.dim(cfg)
    n = d // nc
    rng = np.random.default_rng(21 + P)
    Pd = max(P, 1)
    Uin = 1.0 + 0.3 * rng.standard_normal((B, Pd, d))
    Y = rng.standard_normal((B, Pd, d))
    if P > 3:
        Uin[:, 3] = Uin[:, 1]
        Y[:, 3] = Y[:, 1]
    queries = [Uin[:, min(2, Pd - 1)] + 1e-3 * rng.standard_normal((B, d)),
               Uin[:, min(5, Pd - 1)] + 1e-2 * rng.standard_normal((B, d))]
    c = np.array([[0.25, -0.5, 0.75]])
    r = np.array([[2.0, 3.0, 1.5]])
    c[0, nc:] = 0.0
    r[0, nc:] = 1.0
    prob = rnp.problem(cfg, max_pairs=P + 4)
    with rnp.Solver(prob) as s:
        s.set_scaling(c, r)
        if P > 0:
            s.randnet_fit(_dev(torch, Uin[:, :P]), _dev(torch, Y[:, :P]))
        refs = [s.randnet_predict(_dev(torch, q)).cpu().numpy()[0] for q in queries]
        A, z = s.weights()
    Ut = _dev(torch, Uin[0, :P])
    S = torch.cat([(Ut[:, q * n:(q + 1) * n] - c[0, q]) / r[0, q] for q in range(nc)],
                  dim=1).contiguous()
    Phi = torch.clamp(S @ A.T + z, min=0.0).contiguous()
    Yd = _dev(torch, Y[0, :P])
    ch = (C.c_double * 3)(*c[0])
    rh = (C.c_double * 3)(*r[0])
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    p = C.c_void_p
    ptr = (lambda t: p(t.data_ptr())) if P > 0 else (lambda t: None)
    outs = [torch.full((d,), float("nan"), dtype=torch.float64, device="cuda")
            for _ in queries]
    qds = [_dev(torch, q[0]) for q in queries]
    free = []
    for k, (qd, out, ref) in enumerate(zip(qds, outs, refs)):  # two calls, shared scratch
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        rc = L.rnp_randnet_predict_noalloc(
            C.byref(prob), p(A.data_ptr()), p(z.data_ptr()), ptr(S), ptr(Yd), ptr(Phi), P,
            ch, rh, p(qd.data_ptr()), p(out.data_ptr()), p(status.data_ptr()),
            p(stream.cuda_stream))
        assert rc == rnp.RNP_OK, L.rnp_last_error(None)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert int(status.item()) == rnp.RNP_OK
        got = out.cpu().numpy()
        if P == 0:
            assert np.all(ref == 0.0) and np.all(got == 0.0)
        else:
            assert np.abs(got - ref).max() <= REL * np.abs(ref).max()
    # the second call (after the first has loaded the module on this
    # device) allocates nothing
    assert free[2] == free[3]
    # sizes beyond the fixed scratch are refused before any work
    rc = L.rnp_randnet_predict_noalloc(
        C.byref(prob), p(A.data_ptr()), p(z.data_ptr()), p(A.data_ptr()), p(A.data_ptr()),
        p(A.data_ptr()), 5000, ch, rh, p(qds[0].data_ptr()), p(outs[0].data_ptr()), None,
        p(stream.cuda_stream))
    assert rc == rnp.RNP_EINVAL
    assert b"scratch" in L.rnp_last_error(None)
