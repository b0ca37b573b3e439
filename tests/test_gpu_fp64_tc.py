"""FP64 tensor-core contractions (CRV_F_FP64_TC): parity with the FP64 oracle at the plain
path's bar (1e-10 relative L2 per scale, the element-wise error max|GPU - oracle| /
max|oracle| beside it), in one pass and in many passes over m' (a small A buffer), with the
7-bit digits of real signals and the 6-bit digits that complex signals above L = 512 use
(forced here at a small L); and agreement with the CUDA-core FP64 path at L = 256. A wrong
slice weight, exponent or level would show at 1e-7 or worse, far above these bars."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(__file__))

import paper_1511_05578_gb300 as crv  # noqa: E402
from gpu_util import W_from_device, flm_to_device, map_from_device, max_rel, rel_l2  # noqa: E402
from paper_1511_05578_gb300 import inputs  # noqa: E402
from test_gpu_parity import _analysis_parity  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TC = crv.CRV_F_FP64_TC


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def test_fp64_tc_real_L64():
    """1 real spin-0 map, L=64, lambda=2, J0=2 (seed 0), 7-bit digits, one pass."""
    e = _analysis_parity(64, 2.0, 2, 0, True, crv.CRV_F_REAL | TC, 1e-10)
    assert e["roundtrip"] < 1e-12


@pytest.mark.parametrize("L,lam,J0,s", [(24, 2.0, 2, 2), (33, 2.0, 1, 0), (9, 3.0, 0, 1), (2, 2.0, 1, 0)])
def test_fp64_tc_complex(L, lam, J0, s):
    e = _analysis_parity(L, lam, J0, s, False, TC, 1e-10, seed=7, power=3.0 if s else 2.0)
    assert e["roundtrip"] < 1e-12


def test_fp64_tc_many_passes(monkeypatch):
    """A 1 MB A buffer: the engine runs one pass per m' or two (L=64 real, odd lambda)."""
    monkeypatch.setenv("CRV_FP64_TC_A_GB", "0.001")
    e = _analysis_parity(64, 1.7, 1, 0, True, crv.CRV_F_REAL | TC, 1e-10, seed=5)
    assert e["roundtrip"] < 1e-12


def test_fp64_tc_six_bit_digits(monkeypatch):
    """The 6-bit digits (spin 2, complex, L=40), also over several passes."""
    monkeypatch.setenv("CRV_FP64_TC_BITS", "6")
    monkeypatch.setenv("CRV_FP64_TC_A_GB", "0.002")
    e = _analysis_parity(40, 2.0, 2, 2, False, TC, 1e-10, seed=9, power=3.0)
    assert e["roundtrip"] < 1e-12


def test_fp64_tc_matches_cuda_core_path_L256():
    """The same real map (L=256, lambda=2, J0=2, seed 11) through the CUDA-core FP64 plan and the
    tensor-core FP64 plan: W per scale within 1e-11 (relative L2 and element-wise), round trips
    both within 1e-12."""
    L = 256
    f = inputs.flm_gaussian(L, 11, 0, True, 2.0)
    pa = crv.Plan(L, 2.0, 2, 0, crv.CRV_F_REAL)
    pb = crv.Plan(L, 2.0, 2, 0, crv.CRV_F_REAL | TC)
    fmap = pa.map_tensor(1)
    crv.crv_sht_inv(pa.handle, flm_to_device(f), fmap, 1)
    outs = []
    for p in (pa, pb):
        W, Wphi = p.W_tensors(1), p.Wphi_tensor(1)
        crv.crv_analysis(p.handle, fmap, W, Wphi, 1)
        out = p.map_tensor(1)
        crv.crv_synthesis(p.handle, W, Wphi, out, 1)
        crv.crv_plan_check(p.handle)
        outs.append((W, out))
    ref_map = map_from_device(fmap, True)
    for j in range(2, pa.J + 1):
        a, b = W_from_device(outs[0][0], j, True), W_from_device(outs[1][0], j, True)
        assert rel_l2(b, a) < 1e-11 and max_rel(b, a) < 1e-11, j
    for _, out in outs:
        assert rel_l2(map_from_device(out, True), ref_map) < 1e-12
    pa.close()
    pb.close()

