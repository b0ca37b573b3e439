"""Parity at the benchmark's full sizes, in the configuration bench.py times.

At L = 512 (plain FP64) and L = 1024 (mixed precision, FP32 W) the oracle cannot
evaluate every SO(3) ring, so sampled rings of every scale are compared one by one
(the oracle evaluates Eq. wav_analysis_harmonic directly per ring). Synthesis is
checked per scale through a property that holds at any size: synthesising scale j
alone returns f_lm kappa^(j)(l)^2 (Sum_n |zeta_ln|^2 = 1; kappa from the oracle),
and the full round trip reproduces the input map.
"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))

import oracle as O  # noqa: E402
import paper_1511_05578_gb300 as crv  # noqa: E402
from gpu_util import map_from_device, map_to_device, rel_l2  # noqa: E402
from paper_1511_05578_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _full_case(L, lam, J0, flags, seed, ring_tol, scale_tol, rt_tol, rings_per_scale):
    f = inputs.flm_gaussian(L, seed, real=True)
    fmap = O.sht_inverse(f, L, 0).real
    flm_o = O.sht_forward(fmap, L, 0)          # oracle coefficients of the input map
    p = crv.Plan(L, lam, J0, 0, flags)
    W = p.W_tensors(1)
    Wphi = p.Wphi_tensor(1)
    crv.crv_analysis(p.handle, map_to_device(fmap, True), W, Wphi, 1)
    crv.crv_plan_check(p.handle)
    report = {}
    for j in range(J0, p.J + 1):
        Lb = p.Lj[j]
        rings = sorted({0, Lb // 2, Lb - 1} if rings_per_scale >= 3 else {Lb // 3, Lb - 1})
        if Lb <= 64:
            rings = list(range(Lb))
        ref = O.analysis_rings(flm_o, lam, j, 0, L, rings=rings).real
        got = W[j][0].cpu().numpy().astype(np.float64)[rings]
        report[j] = rel_l2(got, ref)
    Wp_ref = O.scaling_map(flm_o, lam, J0, L).real
    report["phi"] = rel_l2(map_from_device(Wphi, True), Wp_ref)
    bad = {k: v for k, v in report.items() if not v < ring_tol}
    assert not bad, (bad, report)
    # per-scale synthesis: scale j alone -> f_lm kappa_j(l)^2
    l = np.floor(np.sqrt(np.arange(L * L))).astype(int)
    flm = p.flm_tensor(1)
    zeros = p.W_tensors(1)
    scale_err = {}
    for j in range(J0, p.J + 1):
        Wj = [zeros[k] if k != j else W[k] for k in range(p.J + 1)]
        crv.crv_synthesis_lm(p.handle, Wj, None, flm, 1)
        want = flm_o * O.kappa(lam, j, L)[l] ** 2
        scale_err[j] = rel_l2(flm[0].cpu().numpy(), want)
    bad = {k: v for k, v in scale_err.items() if not v < scale_tol}
    assert not bad, (bad, scale_err)
    out = p.map_tensor(1)
    crv.crv_synthesis(p.handle, W, Wphi, out, 1)
    crv.crv_plan_check(p.handle)
    rt = rel_l2(map_from_device(out, True), fmap)
    assert rt < rt_tol, rt
    p.close()
    print(f"\nL={L} flags={flags}: ring rel-L2 {report}\nper-scale synthesis rel-L2 {scale_err}\nround trip {rt:.2e}")


def test_L512_fp64_sampled_rings_and_reconstruction():
    """1 real spin-0 map, L=512, lambda=2, J0=2, plain FP64 (seed 1000)."""
    _full_case(512, 2.0, 2, crv.CRV_F_REAL, 1000, 1e-10, 1e-10, 1e-12, 3)


def test_L1024_mixed_sampled_rings_and_reconstruction():
    """The benchmark's map shape: L=1024, lambda=2, J0=2, split-FP32 contraction,
    FP32 DFTs and W (seed 2000): 1e-5 relative L2 per ring, per scale and round trip."""
    _full_case(1024, 2.0, 2, crv.CRV_F_REAL | crv.CRV_F_MIXED | crv.CRV_F_W_FP32, 2000, 1e-5, 1e-5, 1e-5, 2)
