"""RandNet-Parareal on GB300 -- Python binding of librnp (``include/rnp.h``).

The binding only marshals arguments: every step of the method runs in the
CUDA kernels of ``librnp.so``.  PyTorch provides device memory and the
stream.  There is no CPU fallback: if the library is not built, or there is
no CUDA device, every call raises.

>>> import paper_2411_06225_gb300 as rnp, workloads as W
>>> cfg = W.config("burgers1d")
>>> s = rnp.Solver(rnp.problem(cfg, precision="fp64"))
>>> U, st = s.solve(torch.as_tensor(W.initial_condition(cfg), device="cuda"))
"""
from __future__ import annotations

import ctypes as C
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librnp.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "rnp.h")

RNP_OK, RNP_EINVAL, RNP_ENOMEM, RNP_ECUDA = 0, 1, 2, 3
RNP_ENONFINITE, RNP_ENOTCONV, RNP_ETIMEOUT, RNP_EBUSY = 4, 5, 6, 7
STATUS_NAMES = {0: "RNP_OK", 1: "RNP_EINVAL", 2: "RNP_ENOMEM", 3: "RNP_ECUDA",
                4: "RNP_ENONFINITE", 5: "RNP_ENOTCONV", 6: "RNP_ETIMEOUT",
                7: "RNP_EBUSY"}
PDE = {"burgers1d": 0, "diffreact2d": 1, "bruss2d": 2, "bruss3d": 3, "swe2d": 4,
       "heat": 5, "advect1d": 6}
MAX_BATCH = 64
MAX_M = 32
RNP_MEMBER_FREE, RNP_MEMBER_ACTIVE, RNP_MEMBER_CONVERGED, RNP_MEMBER_NOTCONV = 0, 1, 2, 3


class RnpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Problem(C.Structure):
    """Mirror of ``rnp_problem``."""
    _fields_ = [
        ("pde", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
        ("param", C.c_double * 8), ("t0", C.c_double), ("tN", C.c_double),
        ("N", C.c_int), ("nF", C.c_int), ("nG", C.c_int), ("M", C.c_int),
        ("m", C.c_int), ("lam", C.c_double), ("seed", C.c_uint64),
        ("tol", C.c_double), ("max_iters", C.c_int), ("corr", C.c_int),
        ("scale_mode", C.c_int), ("gscheme", C.c_int), ("precision", C.c_int),
        ("exec_", C.c_int), ("batch", C.c_int), ("cluster", C.c_int),
        ("threads", C.c_int), ("max_pairs", C.c_longlong), ("autotune", C.c_int),
        ("bc", C.c_int), ("fscheme", C.c_int), ("bathymetry", C.POINTER(C.c_double)),
    ]


class Stats(C.Structure):
    """Mirror of ``rnp_stats``."""
    _fields_ = [
        ("K", C.c_int), ("L", C.c_int), ("converged", C.c_int),
        ("pairs", C.c_longlong), ("fine_cell_updates", C.c_longlong),
        ("lambda_escalations", C.c_int), ("t_fine_ms", C.c_double),
        ("t_sweep_ms", C.c_double), ("t_fit_ms", C.c_double),
        ("t_total_ms", C.c_double), ("kernel_launches", C.c_longlong),
        ("K_each", C.c_int * MAX_BATCH),
    ]

    def as_dict(self, batch: int = 1) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "K_each"}
        d["K_each"] = list(self.K_each[:batch])
        return d


def problem(cfg: dict, precision: str = "fp64", exec: str = "fused", **kw) -> Problem:
    """Build an ``rnp_problem`` from a workload dict (see ``workloads``)."""
    c = dict(cfg)
    c.update(kw)
    p = Problem()
    p.pde = PDE[c["pde"]]
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
    p.precision = {"fp64": 0, "mixed": 1, "mixed_bf16": 2}[precision]
    p.exec_ = {"fused": 0, "plain": 1}[exec]
    p.batch = c.get("batch", 1)
    p.cluster = c.get("cluster", 0)
    p.threads = c.get("threads", 0)
    p.max_pairs = c.get("max_pairs", 0)
    p.autotune = int(c.get("autotune", 0))
    p.bc = {"periodic": 0, "neumann": 1}[c.get("bc", "periodic")]
    p.fscheme = {"rk4": 0, "rk8": 1}[c.get("fscheme", "rk4")]
    b = c.get("bathymetry")
    if b is not None:
        import numpy as np
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        if b.size != c["nx"] * c["ny"] * c["nz"]:
            raise ValueError("bathymetry needs one value per cell")
        p._bathymetry = b                 # alive as long as the struct
        p.bathymetry = b.ctypes.data_as(C.POINTER(C.c_double))
    return p


_lib = None


def build(force: bool = False) -> str:
    """Compile librnp.so with nvcc for sm_103a (see builder.py)."""
    from .builder import build as _build
    return _build(force=force)


def exported_symbols() -> list[str]:
    """Function names declared in include/rnp.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rnp_[a-z_0-9]+)\s*\(", src)))


def lib() -> C.CDLL:
    """Load librnp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2411_06225_gb300.build() "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, dp = C.c_void_p, C.c_void_p
    sig = {
        "rnp_create": (C.c_int, [C.POINTER(Problem), vp, C.POINTER(vp)]),
        "rnp_destroy": (C.c_int, [vp]),
        "rnp_fine_batch": (C.c_int, [vp, dp, C.c_int, dp]),
        "rnp_coarse_sweep": (C.c_int, [vp, C.c_int, dp, dp]),
        "rnp_randnet_fit": (C.c_int, [vp, dp, dp, C.c_int]),
        "rnp_randnet_predict": (C.c_int, [vp, dp, dp]),
        "rnp_solve": (C.c_int, [vp, dp, dp, C.POINTER(Stats)]),
        "rnp_last_error": (C.c_char_p, [vp]),
        "rnp_get_weights": (C.c_int, [vp, dp, dp]),
        "rnp_set_scaling": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "rnp_get_scaling": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "rnp_reset": (C.c_int, [vp]),
        "rnp_get_pairs": (C.c_int, [vp, C.POINTER(C.c_longlong)]),
        "rnp_dim": (C.c_longlong, [C.POINTER(Problem)]),
        "rnp_stencil_config": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int)]),
        "rnp_member_start": (C.c_int, [vp, C.c_int, dp]),
        "rnp_features": (C.c_int, [vp, dp, C.c_int, dp]),
        "rnp_iterate": (C.c_int, [vp, C.POINTER(C.c_int)]),
        "rnp_member_status": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int)]),
        "rnp_member_result": (C.c_int, [vp, C.c_int, dp]),
        "rnp_randnet_predict_noalloc": (C.c_int, [
            C.POINTER(Problem), dp, dp, dp, dp, dp, C.c_int, C.POINTER(C.c_double),
            C.POINTER(C.c_double), dp, dp, dp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def dim(p: Problem) -> int:
    return lib().rnp_dim(C.byref(p))


def _ptr(t, dtype=None, shape=None, name="tensor", host_ok=False):
    """Address of a contiguous FP64 tensor: a CUDA tensor, or also a CPU
    tensor (host memory, pinned or not) where the call takes host memory."""
    import torch
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or (host_ok and t.device.type == "cpu")):
        raise TypeError(f"{name} must be a CUDA tensor" + (" or a CPU tensor" if host_ok else ""))
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


class Solver:
    """One RandNet-Parareal context (``rnp_ctx``) bound to a CUDA stream."""

    def __init__(self, prob: Problem, stream=None):
        import torch
        self.p = prob
        self.B = prob.batch
        self.N = prob.N
        self.M = prob.M
        self.d = dim(prob)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        self._ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            st = lib().rnp_create(C.byref(prob), C.c_void_p(self.stream.cuda_stream),
                                  C.byref(self._ctx))
        if st != RNP_OK:
            raise RnpError(st, lib().rnp_last_error(None).decode())

    def _check(self, st: int):
        if st != RNP_OK:
            raise RnpError(st, lib().rnp_last_error(self._ctx).decode())

    def close(self):
        if self._ctx:
            lib().rnp_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _empty(self, *shape):
        import torch
        return torch.empty(*shape, dtype=torch.float64, device=self.device)

    # --- the six calls of the method --------------------------------------
    def fine_batch(self, U_in, out=None):
        n = U_in.shape[1]
        out = self._empty(self.B, n, self.d) if out is None else out
        self._check(lib().rnp_fine_batch(self._ctx, _ptr(U_in, shape=(self.B, n, self.d)),
                                         n, _ptr(out, shape=(self.B, n, self.d))))
        return out

    def coarse_sweep(self, first: int, U_first, U=None):
        U = self._empty(self.B, self.N + 1, self.d) if U is None else U
        self._check(lib().rnp_coarse_sweep(self._ctx, first,
                                           _ptr(U_first, shape=(self.B, self.d)),
                                           _ptr(U, shape=(self.B, self.N + 1, self.d))))
        return U

    def randnet_fit(self, Uin, Y):
        P = Uin.shape[1]
        self._check(lib().rnp_randnet_fit(self._ctx, _ptr(Uin, shape=(self.B, P, self.d)),
                                          _ptr(Y, shape=(self.B, P, self.d)), P))

    def randnet_predict(self, q, out=None):
        out = self._empty(self.B, self.d) if out is None else out
        self._check(lib().rnp_randnet_predict(self._ctx, _ptr(q, shape=(self.B, self.d)),
                                              _ptr(out, shape=(self.B, self.d))))
        return out

    def solve(self, u0, U=None, check: bool = True):
        """Returns (U [B, N+1, d], stats dict).  u0 and U may be CUDA or CPU
        tensors (host memory: the library copies in and out, the output
        while later iterations run); U defaults to a new CUDA tensor.  With
        check=False an RNP_ENOTCONV result is returned instead of raised."""
        U = self._empty(self.B, self.N + 1, self.d) if U is None else U
        st = Stats()
        rc = lib().rnp_solve(self._ctx, _ptr(u0, shape=(self.B, self.d), host_ok=True),
                             _ptr(U, shape=(self.B, self.N + 1, self.d), host_ok=True),
                             C.byref(st))
        if rc == RNP_ENOTCONV and not check:
            return U, st.as_dict(self.B)
        self._check(rc)
        return U, st.as_dict(self.B)

    # --- Alg. 1 one iteration at a time (continuous batching) ---------------
    def member_start(self, member: int, u0):
        self._check(lib().rnp_member_start(self._ctx, member, _ptr(u0, shape=(self.d,))))

    def iterate(self) -> int:
        n = C.c_int(0)
        self._check(lib().rnp_iterate(self._ctx, C.byref(n)))
        return n.value

    def member_status(self, member: int) -> dict:
        st, K, L = C.c_int(), C.c_int(), C.c_int()
        self._check(lib().rnp_member_status(self._ctx, member, C.byref(st), C.byref(K),
                                            C.byref(L)))
        return dict(state=st.value, K=K.value, L=L.value)

    def member_result(self, member: int, U=None, check: bool = True):
        U = self._empty(self.N + 1, self.d) if U is None else U
        rc = lib().rnp_member_result(self._ctx, member, _ptr(U, shape=(self.N + 1, self.d)))
        if not (rc == RNP_ENOTCONV and not check):
            self._check(rc)
        return U

    # --- inspection ------------------------------------------------------
    def features(self, U):
        """Random features ReLU(A s(U) + zeta) of R states U [R, d]."""
        R = U.shape[0]
        phi = self._empty(R, self.M)
        self._check(lib().rnp_features(self._ctx, _ptr(U, shape=(R, self.d)), R, _ptr(phi)))
        return phi

    def weights(self):
        A = self._empty(self.M, self.d)
        z = self._empty(self.M)
        self._check(lib().rnp_get_weights(self._ctx, _ptr(A), _ptr(z)))
        return A, z

    def set_scaling(self, c, r):
        import numpy as np
        c = np.ascontiguousarray(c, np.float64).reshape(self.B, 3)
        r = np.ascontiguousarray(r, np.float64).reshape(self.B, 3)
        self._check(lib().rnp_set_scaling(
            self._ctx, c.ctypes.data_as(C.POINTER(C.c_double)),
            r.ctypes.data_as(C.POINTER(C.c_double))))

    def scaling(self):
        import numpy as np
        c = np.zeros((self.B, 3))
        r = np.zeros((self.B, 3))
        self._check(lib().rnp_get_scaling(
            self._ctx, c.ctypes.data_as(C.POINTER(C.c_double)),
            r.ctypes.data_as(C.POINTER(C.c_double))))
        return c, r

    def reset(self):
        self._check(lib().rnp_reset(self._ctx))

    def stencil_config(self, which: str = "fine") -> dict:
        out = (C.c_int * 6)()
        self._check(lib().rnp_stencil_config(self._ctx, {"fine": 0, "coarse": 1}[which], out))
        return dict(cluster=out[0], threads=out[1], px=out[2], rs=out[3], tuned=bool(out[4]),
                    tm=bool(out[5]))

    def pairs(self):
        out = (C.c_longlong * self.B)()
        self._check(lib().rnp_get_pairs(self._ctx, out))
        return list(out)
