"""The C-ABI boundary without a GPU: librnp.so builds for sm_103a, loads,
exports every function include/rnp.h declares, and the Python mirrors of
rnp_problem / rnp_stats have the C layout (checked against gcc's offsetof
on the real header).  No compute call is made here."""
import ctypes as C
import os
import subprocess

import pytest

import paper_2411_06225_gb300 as rnp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    rnp.build()
    return rnp.lib()


def test_every_declared_symbol_is_exported(built):
    names = rnp.exported_symbols()
    assert {"rnp_create", "rnp_destroy", "rnp_fine_batch", "rnp_coarse_sweep",
            "rnp_randnet_fit", "rnp_randnet_predict", "rnp_solve",
            "rnp_last_error"} <= set(names)
    for n in names:
        assert hasattr(built, n), n


def _c_layout(struct, fields):
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "rnp.h"',
           'int main(void) {', f'  printf("%zu\\n", sizeof({struct}));']
    for f in fields:
        src.append(f'  printf("%zu\\n", offsetof({struct}, {f}));')
    src += ['  return 0;', '}']
    exe = os.path.join(ROOT, "paper_2411_06225_gb300", "_build", f"layout_{struct}")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run(["gcc", "-x", "c", "-", "-I", os.path.join(ROOT, "include"), "-o", exe],
                   input="\n".join(src).encode(), check=True)
    out = subprocess.run([exe], check=True, capture_output=True).stdout.decode().split()
    return [int(x) for x in out]


@pytest.mark.parametrize("cname,pystruct,cfields", [
    ("rnp_problem", rnp.Problem, None),
    ("rnp_stats", rnp.Stats, None),
])
def test_struct_layout_matches_header(cname, pystruct, cfields):
    py_fields = [f for f, _ in pystruct._fields_]
    c_fields = [("exec" if f == "exec_" else "lambda" if f == "lam" else f) for f in py_fields]
    got = _c_layout(cname, c_fields)
    assert got[0] == C.sizeof(pystruct)
    for f, off in zip(py_fields, got[1:]):
        assert getattr(pystruct, f).offset == off, f


def test_create_rejects_bad_problem_without_touching_a_gpu(built):
    # validation happens before any CUDA call
    p = rnp.Problem()
    p.pde = 99
    ctx = C.c_void_p()
    assert built.rnp_create(C.byref(p), None, C.byref(ctx)) == rnp.RNP_EINVAL
    assert b"pde" in built.rnp_last_error(None)
    import workloads as W
    p = rnp.problem(W.config("burgers1d"), m=64)
    assert built.rnp_create(C.byref(p), None, C.byref(ctx)) == rnp.RNP_EINVAL
    assert rnp.dim(rnp.problem(W.config("bruss3d"))) == 2 * 40**3


def test_create_refuses_unsupported_solver_options_without_a_gpu(built):
    import numpy as np
    import workloads as W
    ctx = C.c_void_p()
    # the eighth-order fine solver runs in FP64 only
    p = rnp.problem(W.config("burgers1d", fscheme="rk8"), precision="mixed")
    assert built.rnp_create(C.byref(p), None, C.byref(ctx)) == rnp.RNP_EINVAL
    assert b"RK8" in built.rnp_last_error(None)
    # an unknown fine integrator
    p = rnp.problem(W.config("burgers1d"))
    p.fscheme = 7
    assert built.rnp_create(C.byref(p), None, C.byref(ctx)) == rnp.RNP_EINVAL
    assert b"fscheme" in built.rnp_last_error(None)
    # a bottom profile belongs to shallow water only
    cfg = W.config("diffreact2d", nx=8, ny=8)
    cfg["bathymetry"] = np.zeros((8, 8))
    p = rnp.problem(cfg)
    assert built.rnp_create(C.byref(p), None, C.byref(ctx)) == rnp.RNP_EINVAL
    assert b"bathymetry" in built.rnp_last_error(None)
    with pytest.raises(ValueError):
        rnp.problem(dict(W.config("swe_box"), bathymetry=np.zeros(7)))


def test_serving_pools_separate_bottoms_and_solvers():
    import numpy as np
    import workloads as W
    from paper_2411_06225_gb300.serve import class_key
    base = W.config("swe_box", nx=20, ny=10)
    b1 = dict(base, bathymetry=np.zeros((10, 20)))
    b2 = dict(base, bathymetry=np.full((10, 20), 0.1))
    assert class_key(b1) == class_key(dict(base, bathymetry=np.zeros((10, 20))))
    assert class_key(b1) != class_key(b2) != class_key(base)
    assert class_key(base) != class_key(dict(base, bc="periodic"))
    assert class_key(base) != class_key(dict(base, fscheme="rk8"))
