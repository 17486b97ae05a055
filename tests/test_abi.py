"""The C ABI library loads and exports every function its headers declare.

Runs without a GPU: it only loads liblamino.so and looks the symbols up."""
import ctypes
import os
import re

import pytest

from paper_2511_01893_b300 import build, lamino

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def so():
    build.build()
    return ctypes.CDLL(lamino.LIB_PATH)


def test_headers_declare_the_boundary():
    names = _declared()
    for n in ["lam_plan_create", "lam_forward", "lam_adjoint", "tv_grad", "tv_div", "admm_step", "reconstruct",
              "lam_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(so):
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert missing == []


def test_checked_library_exports_every_declared_symbol():
    path = build.build(checked=True)
    lib = ctypes.CDLL(path)
    assert [n for n in _declared() if not hasattr(lib, n)] == []
    assert lib.lam_bounds_checked() == 1


def test_plain_library_has_no_index_checks(so):
    assert so.lam_bounds_checked() == 0
    # the self-test refuses on the host before any launch
    assert so.lamx_bounds_selftest(None, 70, None) == -6


def test_binding_signatures_cover_exports(so):
    lib = lamino.lib()
    for n in _declared():
        assert getattr(lib, n).restype is not None


def test_host_side_argument_errors_need_no_gpu(so):
    # argument checks happen before any CUDA call
    lib = lamino.lib()
    h = ctypes.c_void_p()
    th = (ctypes.c_double * 4)(0, 1, 2, 3)
    assert lib.lam_plan_create(ctypes.byref(h), 12, 16, 16, 16, 4, th, 0.5, 2, 4, 0) == -6   # n not a multiple of 8
    assert b"multiple of 8" in lib.lam_last_error()
    assert lib.lam_plan_create(ctypes.byref(h), 16, 14, 16, 16, 4, th, 0.5, 2, 4, 0) == -6   # nz = 2 * 7
    assert b"2^a 3^b 5^c" in lib.lam_last_error()
    assert lib.lam_plan_create(ctypes.byref(h), 16, 16, 15, 16, 4, th, 0.5, 2, 4, 0) == -6   # odd det_h
    assert b"even" in lib.lam_last_error()
    assert lib.lam_plan_create(ctypes.byref(h), 16, 16, 16, 16, 4, th, 2.0, 2, 4, 0) == -1   # phi >= pi/2
    assert lib.lam_plan_create(ctypes.byref(h), 16, 16, 16, 16, 4, th, 0.5, 3, 4, 0) == -6   # oversample
    assert lib.lam_plan_create(ctypes.byref(h), 16, 16, 16, 16, 4, None, 0.5, 2, 4, 0) == -1
    assert lib.lam_forward(None, None, None, None, None) == -1
