"""The C ABI: the library loads (no GPU needed to load it), exports every
function that include/lbpwfa.h declares, and the binding refuses to run
without it.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbpwfa_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2309_04872_gb300 import build
    return build.build()


def test_header_declares_the_core_calls():
    d = _declared()
    for name in ("lbpwfa_create", "lbpwfa_step", "lbpwfa_moments", "lbpwfa_fields",
                 "lbpwfa_destroy", "lbpwfa_status_string"):
        assert name in d


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2309_04872_gb300 import lbpwfa
    assert set(lbpwfa.EXPORTED) == _declared()


def test_status_strings(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.lbpwfa_status_string.restype = ctypes.c_char_p
    assert lib.lbpwfa_status_string(0) == b"ok"
    assert lib.lbpwfa_status_string(-1) == b"invalid argument"
    assert lib.lbpwfa_status_string(12345) == b"unknown status"


def test_invalid_parameters_rejected_before_any_device_work(lib_path):
    """Validation runs on the host before the first CUDA call, so it can be
    exercised without a GPU."""
    from paper_2309_04872_gb300 import lbpwfa
    lib = lbpwfa.load_library()
    base = dict(dim=2, n=(16, 8), dx=0.05, courant=0.1, tau=0.53, closure="lec", dv=3, mu=1e-2,
                alpha=0.1, sigma_z=1.0, sigma_r=0.5, z0=1.0)
    bad = [dict(tau=0.5), dict(courant=0.8), dict(n=(2, 8)), dict(dim=4, n=(8, 8, 8)), dict(dv=2),
           dict(mu=-1e-3), dict(sigma_z=0.0), dict(sigma_r=-1.0), dict(dx=0.0), dict(closure=5),
           dict(geometry=2), dict(geometry="axisymmetric", dim=3, n=(8, 8, 8)),
           dict(geometry="axisymmetric", boundary="periodic"), dict(record_tape=-1), dict(checkpoint_every=-5),
           dict(n=(16, 4 * 65535 + 1)), dict(dim=3, n=(8, 8, 4 * 65535 + 1)), dict(dim=3, n=(8, 4 * 65535 + 1, 8))]
    for b in bad:
        p, keep = lbpwfa.make_params({**base, **b})
        h = ctypes.c_void_p()
        assert lib.lbpwfa_create(ctypes.byref(p), ctypes.byref(h)) == -1, b
        assert not h.value
    # axisymmetric runs take the plain or the persistent kernel (variants 0, 1, 3)
    for v in (2, 4):
        p, keep = lbpwfa.make_params({**base, "geometry": "axisymmetric"}, variant=v)
        h = ctypes.c_void_p()
        assert lib.lbpwfa_create(ctypes.byref(p), ctypes.byref(h)) == -1
    p, keep = lbpwfa.make_params(base, precision=7)
    h = ctypes.c_void_p()
    assert lib.lbpwfa_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert lib.lbpwfa_create(None, ctypes.byref(h)) == -1
    assert lib.lbpwfa_step(None, 1) == -1
    assert lib.lbpwfa_autotune(None, None) == -1
    # the diagnostics check their handle and arguments on the host
    fp = lbpwfa.FitParams()
    out = (ctypes.c_double * 5)()
    assert lib.lbpwfa_line_fit(None, ctypes.byref(fp), out) == -1
    lo = (ctypes.c_int * 3)(0, 0, 0)
    hi = (ctypes.c_int * 3)(1, 1, 1)
    assert lib.lbpwfa_gauss_residual(None, lo, hi, out) == -1


def test_device_memory_cap_refuses_before_any_device_work(lib_path):
    """A cap below the state's size returns OOM from lbpwfa_create before
    the first CUDA call (so no GPU is needed); no handle is returned."""
    from paper_2309_04872_gb300 import lbpwfa
    lib = lbpwfa.load_library()
    base = dict(dim=2, n=(64, 32), dx=0.05, courant=0.1, tau=0.53, closure="warmc", dv=3, mu=1e-2,
                alpha=0.1, sigma_z=1.0, sigma_r=0.5, z0=1.0)
    for prec in ("fp64", "fp32", "fp16s"):
        for cap in (1, 4096, 64 * 32 * 72 * 2):
            p, keep = lbpwfa.make_params({**base, "device_bytes_cap": cap}, precision=prec)
            h = ctypes.c_void_p()
            assert lib.lbpwfa_create(ctypes.byref(p), ctypes.byref(h)) == -2, (prec, cap)
            assert not h.value
    assert lib.lbpwfa_set_wait_limit(None, 0) == -1
