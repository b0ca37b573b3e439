"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the same
seeded inputs. Tolerances: FP64 path 1e-10 relative L2 per scale (the bar for the
plain path); mixed path 1e-5 relative L2 per scale. Beside every relative L2 the
element-wise error max|GPU - oracle| / max|oracle| of the same scale is held to the
same bar, so that one wrong (m, n) column or ring cannot hide in a scale's norm."""
import numpy as np
import sys, os
sys.path.insert(0, os.path.dirname(__file__))
import pytest

import oracle as O
import paper_1511_05578_gb300 as crv
from gpu_util import (W_from_device, W_to_device, case, flm_to_device, map_from_device, map_to_device, max_rel,
                      rel_l2)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("L", [8, 64, 300])
def test_delta_tables_match_risbo(L):
    p = crv.Plan(L, 2.0, 0, 0, crv.CRV_F_REAL)
    for l in sorted({0, 1, 2, L // 3, L - 1}):
        D = O.delta_matrix(l)[l:, l:]  # m', n >= 0 quadrant
        got = p.delta(l)
        assert np.abs(got - D).max() < 1e-14 + 2e-16 * l, l
    p.close()


def test_delta_tables_large_l():
    L = 1024
    p = crv.Plan(L, 2.0, 2, 0, crv.CRV_F_REAL)
    for l in [700, 1023]:
        D = O.delta_matrix(l)[l:, l:]
        assert np.abs(p.delta(l) - D).max() < 2e-13, l
    p.close()


@pytest.mark.parametrize("lam,J0,s,L", [(2.0, 2, 0, 64), (2.0, 1, 2, 32), (1.7, 1, -1, 20), (3.0, 0, 1, 40)])
def test_plan_kernels_match_oracle(lam, J0, s, L):
    p = crv.Plan(L, lam, J0, s, 0)
    assert p.J == O.J_max(lam, L) and p.L_phi == O.L_phi(lam, J0, L)
    assert np.abs(p.scaling() - O.phi_scaling(lam, J0, L)).max() < 1e-13
    for j in range(J0, p.J + 1):
        assert p.Lj[j] == O.band_limit(lam, j, L)
        # two evaluations of the same closed form; rounding grows ~linearly in l
        assert np.abs(p.kernel(j) - O.psi(lam, j, s, p.Lj[j])).max() < 1e-13 + 1e-14 * p.Lj[j], j
    p.close()


@pytest.mark.parametrize("L,s,real", [(2, 0, True), (7, 0, False), (64, 0, True), (33, 2, False), (17, -1, False)])
def test_sht_matches_oracle(L, s, real):
    f, fmap = case(L, 2.0, 0, s, real, seed=100 + L)
    p = crv.Plan(L, 2.0, 0 if s == 0 else 2, s, crv.CRV_F_REAL if real else 0)
    m = map_to_device(fmap, real)
    flm = p.flm_tensor(1)
    crv.crv_sht_fwd(p.handle, m, flm, 1)
    got = flm[0].cpu().numpy()
    ref = O.sht_forward(fmap, L, s)
    assert np.abs(got - ref).max() < 1e-13
    out = p.map_tensor(1)
    crv.crv_sht_inv(p.handle, flm_to_device(f), out, 1)
    assert np.abs(map_from_device(out, real) - (O.sht_inverse(f, L, s).real if real else O.sht_inverse(f, L, s))).max() < 1e-13
    p.close()


def _analysis_parity(L, lam, J0, s, real, flags, tol, seed=0, power=2.0, unrot=False):
    f, fmap = case(L, lam, J0, s, real, seed, power)
    flm_o, W_o, Wphi_o = O.analysis(fmap, lam, J0, s, L, unrotated=unrot)
    p = crv.Plan(L, lam, J0, s, flags | (crv.CRV_F_UNROTATED if unrot else 0))
    W = p.W_tensors(1)
    Wphi = p.Wphi_tensor(1)
    crv.crv_analysis(p.handle, map_to_device(fmap, real), W, Wphi, 1)
    torch.cuda.synchronize()
    errs = {}
    for j in range(J0, p.J + 1):
        ref = W_o[j].real if real else W_o[j]
        got = W_from_device(W, j, real)
        errs[j] = rel_l2(got, ref)
        errs[f"{j}/max"] = max_rel(got, ref)
    got = map_from_device(Wphi, real)
    ref = Wphi_o.real if real else Wphi_o
    errs["phi"] = rel_l2(got, ref)
    errs["phi/max"] = max_rel(got, ref)
    # synthesis of the oracle's coefficients
    Wd = W_to_device(p, W_o)
    Wphid = map_to_device(Wphi_o.real if real else Wphi_o, real)
    flm = p.flm_tensor(1)
    crv.crv_synthesis_lm(p.handle, Wd, Wphid, flm, 1)
    f_ref = O.synthesis_flm(W_o, Wphi_o, lam, J0, s, L, unrotated=unrot)
    errs["synthesis"] = rel_l2(flm[0].cpu().numpy(), f_ref)
    errs["synthesis/max"] = max_rel(flm[0].cpu().numpy(), f_ref)
    # round trip through the GPU alone
    out = p.map_tensor(1)
    crv.crv_synthesis(p.handle, W, Wphi, out, 1)
    errs["roundtrip"] = rel_l2(map_from_device(out, real), fmap)
    errs["roundtrip/max"] = max_rel(map_from_device(out, real), fmap)
    p.close()
    bad = {k: v for k, v in errs.items() if not v < tol}
    assert not bad, (bad, errs)
    return errs


def test_analysis_synthesis_fp64_L64_real():
    """Workload: 1 real spin-0 map, L=64, lambda=2, J0=2, Gaussian f_lm C_l=(l+1)^-2, seed 0."""
    e = _analysis_parity(64, 2.0, 2, 0, True, crv.CRV_F_REAL, 1e-10)
    assert e["roundtrip"] < 1e-12


@pytest.mark.parametrize("L,lam,J0,s", [(24, 2.0, 2, 2), (20, 1.7, 1, -1), (33, 2.0, 1, 0), (9, 3.0, 0, 1)])
def test_analysis_synthesis_fp64_complex(L, lam, J0, s):
    e = _analysis_parity(L, lam, J0, s, False, 0, 1e-10, seed=7, power=3.0 if s else 2.0)
    assert e["roundtrip"] < 1e-12


def test_analysis_synthesis_tiny_and_degenerate():
    # L = 2: one scale j = 1 with L_j = 2; J0 = J
    _analysis_parity(2, 2.0, 1, 0, True, crv.CRV_F_REAL, 1e-12)
    _analysis_parity(3, 2.0, 2, 0, False, 0, 1e-12)


def test_analysis_synthesis_fp64_real_odd_L():
    """Real spin-0 map with odd band limits (L=33): the last (m, m+1) column pair of the beta
    transforms has no partner, and the n >= 0 half of the ring transforms is uneven."""
    e = _analysis_parity(33, 2.0, 2, 0, True, crv.CRV_F_REAL, 1e-10, seed=3)
    assert e["roundtrip"] < 1e-12


def test_mixed_precision_real_odd_L_lambda():
    """Mixed precision, real spin 0, L=45, lambda=1.7, J0=1: odd and non-power-of-two band
    limits through the tensor-core tables and the paired beta kernels."""
    e = _analysis_parity(45, 1.7, 1, 0, True, crv.CRV_F_REAL | crv.CRV_F_MIXED, 1e-5, seed=4)
    assert e["roundtrip"] < 1e-5


def test_mixed_precision_L64():
    e = _analysis_parity(64, 2.0, 2, 0, True, crv.CRV_F_REAL | crv.CRV_F_MIXED, 1e-5)
    assert e["roundtrip"] < 1e-5


def test_mixed_precision_w_fp32_spin2():
    _analysis_parity(32, 2.0, 1, 2, False, crv.CRV_F_MIXED | crv.CRV_F_W_FP32, 1e-5)


def test_batch_matches_single():
    L, lam, J0 = 32, 2.0, 2
    p = crv.Plan(L, lam, J0, 0, crv.CRV_F_REAL, max_batch=3)
    maps = [case(L, lam, J0, 0, True, seed=s)[1] for s in (1, 2, 3)]
    mb = torch.tensor(np.stack(maps), device="cuda")
    Wb = p.W_tensors(3)
    crv.crv_analysis(p.handle, mb, Wb, None, 3)
    for b in range(3):
        W1 = p.W_tensors(1)
        crv.crv_analysis(p.handle, map_to_device(maps[b], True), W1, None, 1)
        for j in range(J0, p.J + 1):
            assert torch.equal(Wb[j][b], W1[j][0])
    with pytest.raises(crv.CrvError):
        crv.crv_analysis(p.handle, mb, Wb, None, 4)  # B > max_batch
    crv.crv_analysis(p.handle, mb, Wb, None, 0)  # empty batch is a no-op
    p.close()


# ---- unrotated curvelets (CRV_F_UNROTATED): the paper's O(L^3 log L) path --------------

@pytest.mark.parametrize("lam,J0,s,L", [(2.0, 2, 0, 64), (2.0, 1, 2, 32), (1.7, 1, -1, 20)])
def test_unrotated_plan_kernels_match_oracle(lam, J0, s, L):
    p = crv.Plan(L, lam, J0, s, crv.CRV_F_UNROTATED)
    for j in range(J0, p.J + 1):
        assert np.abs(p.kernel(j) - O.psi(lam, j, s, p.Lj[j], unrotated=True)).max() < 1e-13 + 1e-14 * p.Lj[j], j
    p.close()


@pytest.mark.parametrize("L,lam,J0,s,real", [(64, 2.0, 2, 0, True), (33, 2.0, 2, 0, True), (24, 2.0, 2, 2, False),
                                             (20, 1.7, 1, -1, False), (9, 3.0, 0, 1, False), (2, 2.0, 1, 0, True)])
def test_unrotated_fp64(L, lam, J0, s, real):
    """W~ on the SO(3) grid against the oracle (1e-10 per scale), synthesis of the oracle's W~,
    and the GPU round trip."""
    e = _analysis_parity(L, lam, J0, s, real, crv.CRV_F_REAL if real else 0, 1e-10, seed=11, power=3.0 if s else 2.0,
                         unrot=True)
    assert e["roundtrip"] < 1e-12


@pytest.mark.parametrize("L,lam,J0,s,real", [(64, 2.0, 2, 0, True), (45, 1.7, 1, 0, True), (32, 2.0, 1, 2, False)])
def test_unrotated_mixed(L, lam, J0, s, real):
    flags = crv.CRV_F_MIXED | crv.CRV_F_W_FP32 | (crv.CRV_F_REAL if real else 0)
    e = _analysis_parity(L, lam, J0, s, real, flags, 1e-5, seed=12, power=3.0 if s else 2.0, unrot=True)
    assert e["roundtrip"] < 1e-5
