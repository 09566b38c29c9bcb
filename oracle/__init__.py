"""ctypes binding of the FP64 CPU oracle (``rnp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the product package never
imports it.  It shares no code with the CUDA library.

Functions follow the paper (NeurIPS 2024, "Parallel-in-time solver for PDEs
with RandNet-Parareal"): Alg. 1 (generic Parareal), Alg. 3 (RandNet
training), Eq. 3 (update rule), Eq. 4 (classic correction), Eq. 5 (stopping
rule), Eq. HA (random network), Eq. ridgeless (readout), App. B (m nearest
neighbours).

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, invariants, brute force, library routines or published
test vectors.  The end-to-end iterates for tol > 0 have no value printed in
the paper; beyond the K = N exactness and G = F invariants they are
"parity unpinned" (see the test docstrings).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rnp_oracle.c")
_LIB = os.path.join(_HERE, "librnp_oracle.so")

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ENONFINITE, ORC_ENOTCONV = 0, 1, 2, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, FP64, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(_SRC[:-1] + "h"))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Problem(C.Structure):
    _fields_ = [
        ("pde", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
        ("param", C.c_double * 8), ("t0", C.c_double), ("tN", C.c_double),
        ("N", C.c_int), ("nF", C.c_int), ("nG", C.c_int), ("M", C.c_int),
        ("m", C.c_int), ("lam", C.c_double), ("seed", C.c_uint64),
        ("tol", C.c_double), ("max_iters", C.c_int), ("corr", C.c_int),
        ("scale_mode", C.c_int), ("gscheme", C.c_int), ("bc", C.c_int),
        ("fscheme", C.c_int), ("bathy", C.POINTER(C.c_double)),
    ]


class Stats(C.Structure):
    _fields_ = [("K", C.c_int), ("L", C.c_int), ("converged", C.c_int),
                ("pairs", C.c_long), ("fine_cell_updates", C.c_longlong),
                ("lambda_escalations", C.c_int)]


class Trace(C.Structure):
    _fields_ = [("L_hist", C.POINTER(C.c_int)), ("nn_idx", C.POINTER(C.c_long))]


_lib = None
_DP = C.POINTER(C.c_double)
_LP = C.POINTER(C.c_long)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        P = C.POINTER(Problem)
        sig = {
            "orc_ncomp": (C.c_int, [P]),
            "orc_dim": (C.c_long, [P]),
            "orc_set_threads": (None, [C.c_int]),
            "orc_rhs": (None, [P, _DP, _DP]),
            "orc_rk4": (None, [P, _DP, C.c_double, C.c_int]),
            "orc_euler": (None, [P, _DP, C.c_double, C.c_int]),
            "orc_rk8": (None, [P, _DP, C.c_double, C.c_int]),
            "orc_rk8_tableau": (None, [_DP, _DP, _DP]),
            "orc_fine": (None, [P, _DP, _DP]),
            "orc_coarse": (None, [P, _DP, _DP]),
            "orc_serial_fine": (None, [P, _DP, _DP]),
            "orc_splitmix64_next": (C.c_uint64, [C.POINTER(C.c_uint64)]),
            "orc_uniform": (C.c_double, [C.c_uint64, C.c_uint32, C.c_uint64]),
            "orc_weights": (None, [P, _DP, _DP]),
            "orc_scaling": (None, [P, _DP, C.c_int, _DP, _DP]),
            "orc_scale": (None, [P, _DP, _DP, _DP, _DP]),
            "orc_features": (None, [_DP, _DP, C.c_int, C.c_long, _DP, _DP]),
            "orc_nn": (C.c_int, [_DP, C.c_long, C.c_long, _DP, C.c_int, _LP, _DP]),
            "orc_cholesky_solve": (C.c_int, [_DP, C.c_int, _DP, _DP]),
            "orc_ridge_dual": (C.c_int, [_DP, C.c_int, C.c_int, _DP, C.c_double, _DP]),
            "orc_ridge_primal": (C.c_int, [_DP, _DP, C.c_int, C.c_int, C.c_long,
                                           _DP, C.c_double, _DP]),
            "orc_predict": (C.c_int, [P, _DP, _DP, _DP, C.c_long, _DP, _DP, _DP,
                                      _DP, _DP, _DP, _LP]),
            "orc_solve": (C.c_int, [P, _DP, _DP, C.POINTER(Stats), C.POINTER(Trace)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def problem(cfg: dict, **kw) -> Problem:
    """Oracle problem struct from a workload dict (see ``workloads``)."""
    from workloads import PDE_IDS
    c = dict(cfg)
    c.update(kw)
    p = Problem()
    p.pde = PDE_IDS[c["pde"]]
    p.nx, p.ny, p.nz = c["nx"], c["ny"], c["nz"]
    p.lx, p.ly, p.lz = c["lx"], c["ly"], c["lz"]
    for i, v in enumerate(c["param"]):
        p.param[i] = v
    p.t0, p.tN = c["t0"], c["tN"]
    p.N, p.nF, p.nG = c["N"], c["nF"], c["nG"]
    p.M, p.m, p.lam = c["M"], c["m"], c["lam"]
    p.seed = c["seed"]
    p.tol = c["tol"]
    p.max_iters = c.get("max_iters", c["N"])
    p.corr = {"randnet": 0, "parareal": 1}[c.get("corr", "randnet")]
    p.scale_mode = {"minmax": 0, "none": 1}[c.get("scale", "minmax")]
    p.gscheme = {"euler": 0, "rk4": 1}[c.get("gscheme", "euler")]
    p.bc = {"periodic": 0, "neumann": 1}[c.get("bc", "periodic")]
    p.fscheme = {"rk4": 0, "rk8": 1}[c.get("fscheme", "rk4")]
    b = c.get("bathymetry")
    if b is not None:
        b = np.ascontiguousarray(b, np.float64).reshape(-1)
        assert b.size == c["nx"] * c["ny"] * c["nz"]
        p._bathy = b                      # keeps the array alive with p
        p.bathy = b.ctypes.data_as(_DP)
    return p


def set_threads(n: int) -> None:
    lib().orc_set_threads(n)


def dim(p: Problem) -> int:
    return lib().orc_dim(C.byref(p))


def rhs(p: Problem, u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float64)
    out = np.empty_like(u)
    lib().orc_rhs(C.byref(p), _dp(u), _dp(out))
    return out


def rk4(p: Problem, u: np.ndarray, dt: float, n: int) -> np.ndarray:
    v = np.array(u, np.float64, copy=True)
    lib().orc_rk4(C.byref(p), _dp(v), dt, n)
    return v


def rk8(p: Problem, u: np.ndarray, dt: float, n: int) -> np.ndarray:
    v = np.array(u, np.float64, copy=True)
    lib().orc_rk8(C.byref(p), _dp(v), dt, n)
    return v


def rk8_tableau():
    """(A, b, c) of the oracle's RK8 as an 11 x 11 strictly lower-triangular
    matrix and two vectors."""
    a, b, c = np.zeros(55), np.zeros(11), np.zeros(11)
    lib().orc_rk8_tableau(_dp(a), _dp(b), _dp(c))
    A = np.zeros((11, 11))
    for s in range(1, 11):
        A[s, :s] = a[s * (s - 1) // 2: s * (s - 1) // 2 + s]
    return A, b, c


def euler(p: Problem, u: np.ndarray, dt: float, n: int) -> np.ndarray:
    v = np.array(u, np.float64, copy=True)
    lib().orc_euler(C.byref(p), _dp(v), dt, n)
    return v


def fine(p: Problem, u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float64)
    out = np.empty_like(u)
    lib().orc_fine(C.byref(p), _dp(u), _dp(out))
    return out


def coarse(p: Problem, u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float64)
    out = np.empty_like(u)
    lib().orc_coarse(C.byref(p), _dp(u), _dp(out))
    return out


def serial_fine(p: Problem, u0: np.ndarray) -> np.ndarray:
    u0 = np.ascontiguousarray(u0, np.float64)
    U = np.empty((p.N + 1, u0.size), np.float64)
    lib().orc_serial_fine(C.byref(p), _dp(u0), _dp(U))
    return U


def splitmix64_seq(seed: int, n: int) -> list[int]:
    s = C.c_uint64(seed)
    return [lib().orc_splitmix64_next(C.byref(s)) for _ in range(n)]


def uniform(seed: int, stream: int, idx: int) -> float:
    return lib().orc_uniform(seed, stream, idx)


def weights(p: Problem) -> tuple[np.ndarray, np.ndarray]:
    d = dim(p)
    A = np.empty((p.M, d), np.float64)
    z = np.empty(p.M, np.float64)
    lib().orc_weights(C.byref(p), _dp(A), _dp(z))
    return A, z


def scaling(p: Problem, U: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    U = np.ascontiguousarray(U, np.float64)
    c = np.empty(3, np.float64)
    r = np.empty(3, np.float64)
    lib().orc_scaling(C.byref(p), _dp(U), U.shape[0], _dp(c), _dp(r))
    return c, r


def scale(p: Problem, c, r, u) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float64)
    s = np.empty_like(u)
    lib().orc_scale(C.byref(p), _dp(np.ascontiguousarray(c, np.float64)),
                    _dp(np.ascontiguousarray(r, np.float64)), _dp(u), _dp(s))
    return s


def features(A: np.ndarray, zeta: np.ndarray, s: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, np.float64)
    M, d = A.shape
    phi = np.empty(M, np.float64)
    lib().orc_features(_dp(A), _dp(np.ascontiguousarray(zeta, np.float64)), M, d,
                       _dp(np.ascontiguousarray(s, np.float64)), _dp(phi))
    return phi


def nn(S: np.ndarray, q: np.ndarray, m: int):
    S = np.ascontiguousarray(S, np.float64)
    P, d = S.shape
    idx = np.zeros(max(m, 1), np.int64)
    dist = np.zeros(max(m, 1), np.float64)
    me = lib().orc_nn(_dp(S), P, d, _dp(np.ascontiguousarray(q, np.float64)), m,
                      idx.ctypes.data_as(_LP), _dp(dist))
    return idx[:me].copy(), dist[:me].copy()


def cholesky_solve(K: np.ndarray, b: np.ndarray):
    K = np.ascontiguousarray(K, np.float64)
    x = np.zeros(K.shape[0], np.float64)
    rc = lib().orc_cholesky_solve(_dp(K), K.shape[0],
                                  _dp(np.ascontiguousarray(b, np.float64)), _dp(x))
    return rc, x


def ridge_dual(X: np.ndarray, phiq: np.ndarray, lam: float):
    X = np.ascontiguousarray(X, np.float64)
    m, M = X.shape
    alpha = np.zeros(m, np.float64)
    esc = lib().orc_ridge_dual(_dp(X), m, M, _dp(np.ascontiguousarray(phiq, np.float64)),
                               lam, _dp(alpha))
    return esc, alpha


def ridge_primal(X: np.ndarray, Y: np.ndarray, phiq: np.ndarray, lam: float):
    X = np.ascontiguousarray(X, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    m, M = X.shape
    d = Y.shape[1]
    pred = np.zeros(d, np.float64)
    rc = lib().orc_ridge_primal(_dp(X), _dp(Y), m, M, d,
                                _dp(np.ascontiguousarray(phiq, np.float64)), lam,
                                _dp(pred))
    return rc, pred


def predict(p: Problem, S, Y, Phi, A, zeta, c, r, u):
    S = np.ascontiguousarray(S, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    Phi = np.ascontiguousarray(Phi, np.float64)
    out = np.zeros(dim(p), np.float64)
    nn_out = np.full(max(p.m, 1), -1, np.int64)
    rc = lib().orc_predict(C.byref(p), _dp(S), _dp(Y), _dp(Phi), S.shape[0],
                           _dp(np.ascontiguousarray(A, np.float64)),
                           _dp(np.ascontiguousarray(zeta, np.float64)),
                           _dp(np.ascontiguousarray(c, np.float64)),
                           _dp(np.ascontiguousarray(r, np.float64)),
                           _dp(np.ascontiguousarray(u, np.float64)), _dp(out),
                           nn_out.ctypes.data_as(_LP))
    return rc, out, nn_out


def solve(p: Problem, u0: np.ndarray, trace: bool = False):
    """Alg. 1; returns (status, U [N+1, d], Stats, trace dict or None)."""
    u0 = np.ascontiguousarray(u0, np.float64)
    d = dim(p)
    U = np.zeros((p.N + 1, d), np.float64)
    st = Stats()
    tr = None
    trp = None
    if trace:
        Lh = np.full(p.N, -1, np.int32)
        nn_idx = np.full(p.N * (p.N + 1) * p.m, -1, np.int64)
        tr = Trace(Lh.ctypes.data_as(C.POINTER(C.c_int)),
                   nn_idx.ctypes.data_as(_LP))
        trp = C.byref(tr)
    rc = lib().orc_solve(C.byref(p), _dp(u0), _dp(U), C.byref(st), trp)
    tdict = None
    if trace:
        tdict = dict(L_hist=Lh[: st.K].copy(),
                     nn_idx=nn_idx.reshape(p.N, p.N + 1, p.m)[: st.K].copy())
    return rc, U, st, tdict
