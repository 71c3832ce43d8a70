"""The C ABI library without a GPU: it builds, loads, exports every entry
point that include/fv.h declares, and its host-side argument checks reject
bad calls before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1812_07977_gb300 import fv
from paper_1812_07977_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return fv.load_library()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "fv.h")).read()
    return sorted(set(re.findall(r"^FV_API\s+[\w\s\*]+?\b(fv_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_symbols():
    assert _declared_symbols() == sorted(fv.ABI_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_only_the_abi_is_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", fv.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert exported == sorted(fv.ABI_SYMBOLS)


def test_status_strings(lib):
    for s, name in enumerate(["FV_OK", "FV_ERR_INVALID_ARG", "FV_ERR_OOM", "FV_ERR_CUDA",
                              "FV_ERR_NONPHYSICAL", "FV_ERR_TIMEOUT", "FV_ERR_BAD_HANDLE"]):
        assert lib.fv_status_string(s).decode() == name
    assert lib.fv_status_string(99).decode() == "FV_ERR_UNKNOWN"


def _desc(**kw):
    d = fv.MeshDesc()
    d.nx, d.ny, d.nz = kw.get("n", (8, 8, 8))
    d.lx = d.ly = d.lz = kw.get("l", 1.0)
    d.gamma = kw.get("gamma", 1.4)
    d.theta = kw.get("theta", 2.0)
    for a in range(3):
        d.bc[a] = kw.get("bc", 0)
    d.precision = kw.get("precision", 0)
    return d


@pytest.mark.parametrize("bad", [dict(n=(0, 8, 8)), dict(n=(8, -1, 8)), dict(l=0.0),
                                 dict(l=float("inf")), dict(gamma=1.0), dict(gamma=float("nan")),
                                 dict(theta=-0.5), dict(theta=2.5), dict(bc=7),
                                 dict(precision=9), dict(n=(4096, 4096, 4096))])
def test_create_rejects_bad_descriptions(lib, bad):
    h = ctypes.c_void_p()
    d = _desc(**bad)
    st = lib.fv_create_mesh(ctypes.byref(d), None, ctypes.byref(h))
    assert st == fv.ERR_INVALID_ARG
    assert h.value is None
    assert lib.fv_last_error().decode()


def test_create_rejects_null_arguments(lib):
    assert lib.fv_create_mesh(None, None, None) == fv.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.fv_create_mesh(None, None, ctypes.byref(h)) == fv.ERR_INVALID_ARG


def test_calls_on_bad_handles(lib):
    bogus = ctypes.c_void_p(0x1234)
    dt = ctypes.c_double()
    assert lib.fv_step(bogus, 0.1) == fv.ERR_BAD_HANDLE
    assert lib.fv_step(None, 0.1) == fv.ERR_BAD_HANDLE
    assert lib.fv_reduce_dt(bogus, 0.4, ctypes.byref(dt)) == fv.ERR_BAD_HANDLE
    assert lib.fv_destroy_mesh(bogus) == fv.ERR_BAD_HANDLE
    assert lib.fv_destroy_mesh(None) == fv.OK
    assert "not live" in lib.fv_last_error().decode()


def _enum_values(name):
    text = open(os.path.join(ROOT, "include", "fv.h")).read()
    body = re.search(r"typedef enum\s*\{([^}]*)\}\s*" + name + r"\s*;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return {k: int(v) for k, v in re.findall(r"(\w+)\s*=\s*(\d+)", body)}


def test_precision_enum_keeps_the_boundary_values():
    """FV_PREC_FP64 = 0 and FV_PREC_FP32_BULK = 1 as the boundary first fixed
    them; later arithmetic variants take new values, and the binding's names
    map onto the header's numbers."""
    v = _enum_values("fv_precision")
    assert v["FV_PREC_FP64"] == 0 and v["FV_PREC_FP32_BULK"] == 1
    assert v["FV_PREC_FP64_FMA"] == 2
    assert len(set(v.values())) == len(v)
    for name, num in fv.PRECISION.items():
        assert v["FV_PREC_" + name.upper()] == num


def test_status_and_bc_enum_values():
    s = _enum_values("fv_status")
    assert [s[k] for k in ("FV_OK", "FV_ERR_INVALID_ARG", "FV_ERR_OOM", "FV_ERR_CUDA",
                           "FV_ERR_NONPHYSICAL", "FV_ERR_TIMEOUT",
                           "FV_ERR_BAD_HANDLE")] == list(range(7))
    b = _enum_values("fv_bc")
    assert b == {"FV_BC_OUTFLOW": 0, "FV_BC_PERIODIC": 1}
    assert fv.BC == {"outflow": 0, "periodic": 1}


def test_tuning_keys_match_the_header():
    """The binding's tuning-key names map onto fv_tuning_key's numbers, one
    name per key."""
    v = _enum_values("fv_tuning_key")
    assert len(set(v.values())) == len(v) == len(fv.TUNING_KEYS)
    for name, num in fv.TUNING_KEYS.items():
        assert v["FV_TUNE_" + name.upper()] == num
