"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/crv.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "crv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(crv_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1511_05578_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["crv_plan_create", "crv_plan_destroy", "crv_plan_info", "crv_sht_fwd", "crv_sht_inv",
              "crv_analysis", "crv_synthesis", "crv_analysis_lm", "crv_synthesis_lm", "crv_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (crv_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_resolves(libpath):
    import paper_1511_05578_gb300 as crv
    h = crv.load()
    for n in _declared():
        assert hasattr(h, n)
    assert crv.crv_status_string(crv.CRV_EINVAL) == "CRV_EINVAL"
    assert crv.crv_launch_count() >= 0


def test_plan_create_rejects_bad_arguments_without_gpu(libpath):
    """Argument validation happens before any device call."""
    import paper_1511_05578_gb300 as crv
    h = crv.load()
    out = ctypes.c_void_p()
    assert h.crv_plan_create(ctypes.byref(out), 1, 2.0, 0, 0, 0, 0, 1, None) == crv.CRV_EINVAL
    assert h.crv_plan_create(ctypes.byref(out), 64, 1.0, 0, 0, 0, 0, 1, None) == crv.CRV_EINVAL
    assert h.crv_plan_create(ctypes.byref(out), 64, 2.0, 0, 2, 0, crv.CRV_F_REAL, 1, None) == crv.CRV_EINVAL
    assert h.crv_plan_create(ctypes.byref(out), 64, 2.0, 0, 3, 0, 0, 1, None) == crv.CRV_EINVAL  # 2^0 < 3
    assert h.crv_plan_create(ctypes.byref(out), 64, 2.0, 9, 0, 0, 0, 1, None) == crv.CRV_EINVAL  # J0 > J = 6
    assert h.crv_plan_create(ctypes.byref(out), 64, 2.0, 0, 0, 7, 0, 1, None) == crv.CRV_EINVAL
    assert h.crv_plan_create(ctypes.byref(out), 64, 2.0, 0, 0, 0, 0, 0, None) == crv.CRV_EINVAL
    # the FP64 tensor-core contractions are a form of the plain rotated path only
    for bad in (crv.CRV_F_FP64_TC | crv.CRV_F_MIXED, crv.CRV_F_FP64_TC | crv.CRV_F_UNROTATED, 128):
        assert h.crv_plan_create(ctypes.byref(out), 16, 2.0, 0, 0, 0, bad, 1, None) == crv.CRV_EINVAL
    assert out.value is None
    assert "must" in crv.crv_last_error() or crv.crv_last_error() != ""
