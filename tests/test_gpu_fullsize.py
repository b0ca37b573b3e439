"""Parity at the benchmark's full sizes, in the configuration bench.py times.

At L = 512 (plain FP64) and L = 1024 (mixed precision, FP32 W) the oracle cannot
evaluate every SO(3) ring, so sampled rings of every scale are compared one by one
(the oracle evaluates Eq. wav_analysis_harmonic directly per ring). Synthesis is
checked per scale through a property that holds at any size: synthesising scale j
alone returns f_lm kappa^(j)(l)^2 (Sum_n |zeta_ln|^2 = 1; kappa from the oracle),
and the full round trip reproduces the input map. Every relative L2 has the
element-wise error max|GPU - oracle| / max|oracle| of the same set beside it, held to
the same bar. Ring b = 0, next to the pole where d^l(beta) is most extreme, is in
every sampled set.
"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))

import oracle as O  # noqa: E402
import paper_1511_05578_gb300 as crv  # noqa: E402
from gpu_util import W_from_device, map_from_device, map_to_device, max_rel, rel_l2  # noqa: E402
from paper_1511_05578_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _full_case(L, lam, J0, flags, seed, ring_tol, scale_tol, rt_tol, rings_per_scale, spin=0, synth_scales=None):
    unrot = bool(flags & crv.CRV_F_UNROTATED)
    real = bool(flags & crv.CRV_F_REAL)
    f = inputs.flm_gaussian(L, seed, spin, real, 3.0 if spin else 2.0)
    fmap = O.sht_inverse(f, L, spin)
    if real:
        fmap = fmap.real
    flm_o = O.sht_forward(fmap, L, spin)       # oracle coefficients of the input map
    p = crv.Plan(L, lam, J0, spin, flags)
    W = p.W_tensors(1)
    Wphi = p.Wphi_tensor(1)
    crv.crv_analysis(p.handle, map_to_device(fmap, real), W, Wphi, 1)
    crv.crv_plan_check(p.handle)
    report = {}
    for j in range(J0, p.J + 1):
        Lb = p.Lj[j]
        rings = sorted({0, Lb // 2, Lb - 1} if rings_per_scale >= 3 else {0, Lb // 3, Lb - 1})
        if Lb <= 64:
            rings = list(range(Lb))
        ref = O.analysis_rings(flm_o, lam, j, spin, L, rings=rings, unrotated=unrot)
        ref = ref.real if real else ref
        got = W_from_device(W, j, real)[rings]
        report[j] = rel_l2(got, ref)
        report[f"{j}/max"] = max_rel(got, ref)
        for i, b in enumerate(rings):  # each sampled ring on its own
            report[f"{j}/ring{b}"] = rel_l2(got[i], ref[i])
    Wp_ref = O.scaling_map(flm_o, lam, J0, L)
    Wp_ref = Wp_ref.real if real else Wp_ref
    report["phi"] = rel_l2(map_from_device(Wphi, real), Wp_ref)
    report["phi/max"] = max_rel(map_from_device(Wphi, real), Wp_ref)
    bad = {k: v for k, v in report.items() if not v < ring_tol}
    assert not bad, (bad, report)
    # per-scale synthesis: scale j alone -> f_lm kappa_j(l)^2
    l = np.floor(np.sqrt(np.arange(L * L))).astype(int)
    flm = p.flm_tensor(1)
    # the other scales read as zero: one zero buffer of the largest scale's size serves them all
    zero = torch.zeros(max(W[k].numel() for k in range(J0, p.J + 1)), dtype=W[p.J].dtype, device="cuda")
    scale_err = {}
    for j in (synth_scales if synth_scales is not None else range(J0, p.J + 1)):
        Wj = [W[k] if (k == j or W[k] is None) else zero[: W[k].numel()].view(W[k].shape) for k in range(p.J + 1)]
        crv.crv_synthesis_lm(p.handle, Wj, None, flm, 1)
        want = flm_o * O.kappa(lam, j, L)[l] ** 2
        got = flm[0].cpu().numpy()
        scale_err[j] = rel_l2(got, want)
        scale_err[f"{j}/max"] = max_rel(got, want)
    del zero
    bad = {k: v for k, v in scale_err.items() if not v < scale_tol}
    assert not bad, (bad, scale_err)
    out = p.map_tensor(1)
    crv.crv_synthesis(p.handle, W, Wphi, out, 1)
    crv.crv_plan_check(p.handle)
    rt = rel_l2(map_from_device(out, real), fmap)
    rt_max = max_rel(map_from_device(out, real), fmap)
    assert rt < rt_tol and rt_max < rt_tol, (rt, rt_max)
    p.close()
    print(f"\nL={L} spin={spin} flags={flags}: ring rel-L2 {report}\nper-scale synthesis rel-L2 {scale_err}\nround trip {rt:.2e}")


def test_L512_fp64_sampled_rings_and_reconstruction():
    """1 real spin-0 map, L=512, lambda=2, J0=2, plain FP64 (seed 1000)."""
    _full_case(512, 2.0, 2, crv.CRV_F_REAL, 1000, 1e-10, 1e-10, 1e-12, 3)


def test_L1024_fp64_sampled_rings_and_reconstruction():
    """Plain FP64 at the benchmark's map shape: 1 real spin-0 map, L=1024, lambda=2, J0=2
    (seed 2000). Rings 0, L_j/3 and L_j - 1 of every scale against the oracle at 1e-10
    (relative L2 per ring and per scale, element-wise per scale); synthesis of the lowest
    and the two top scales alone against f_lm kappa_j(l)^2 at 1e-10; round trip 1e-12."""
    _full_case(1024, 2.0, 2, crv.CRV_F_REAL, 2000, 1e-10, 1e-10, 1e-12, 2, synth_scales=[2, 9, 10])


def test_L1024_fp64_tc_sampled_rings_and_reconstruction():
    """Plain FP64 with the contractions on the tensor cores (CRV_F_FP64_TC, 7-bit digits) at
    the benchmark's map shape (L=1024, lambda=2, J0=2, seed 2000): the plain path's bars,
    1e-10 per ring and per scale, 1e-12 round trip."""
    _full_case(1024, 2.0, 2, crv.CRV_F_REAL | crv.CRV_F_FP64_TC, 2000, 1e-10, 1e-10, 1e-12, 2,
               synth_scales=[2, 9, 10])


def test_L1024_mixed_sampled_rings_and_reconstruction():
    """The benchmark's map shape: L=1024, lambda=2, J0=2, split-FP32 contraction,
    FP32 DFTs and W (seed 2000): 1e-5 relative L2 per ring, per scale and round trip."""
    _full_case(1024, 2.0, 2, crv.CRV_F_REAL | crv.CRV_F_MIXED | crv.CRV_F_W_FP32, 2000, 1e-5, 1e-5, 1e-5, 2)


def test_L1024_mixed_spin2_sampled_rings_and_reconstruction():
    """A complex spin-2 map at L=1024 (lambda=2, J0=2; f_lm Gaussian with C_l=(l+1)^-3, seed
    3000), mixed precision: the complex-signal ring and beta kernels at P = 4096 (all m, all n),
    1e-5 relative L2 per sampled ring, per scale and round trip (~175 GB on the device)."""
    _full_case(1024, 2.0, 2, crv.CRV_F_MIXED | crv.CRV_F_W_FP32, 3000, 1e-5, 1e-5, 1e-5, 2, spin=2)


def test_L1024_mixed_unrotated_sampled_rings_and_reconstruction():
    """The benchmark's map shape with the unrotated curvelets (CRV_F_UNROTATED: the paper's
    single-term l = |n| contraction, every n in the planes), mixed precision (seed 2000):
    1e-5 relative L2 per sampled ring, per scale (synthesis of scale j alone gives
    f_lm kappa^(j)(l)^2, Sum_n |zeta~_ln|^2 = 1) and round trip."""
    _full_case(1024, 2.0, 2, crv.CRV_F_REAL | crv.CRV_F_MIXED | crv.CRV_F_W_FP32 | crv.CRV_F_UNROTATED, 2000,
               1e-5, 1e-5, 1e-5, 2)
