"""Guard regions (CRV_F_GUARD) as the memory check of the library's kernels, in place of a
memory checker: every device buffer of a plan is followed by a guard region of a known
pattern, and every caller buffer here is followed by a sentinel tail. Each path (mixed with
map workers, plain FP64 complex spin 2, FP64 on tensor cores over many passes, unrotated
with the rotation of Wigner coefficients, and the full-size L = 1024 mixed and L = 520 FP64
kernels) runs its calls and must leave every guard and every tail intact. The check itself is
tested by changing guard bytes from the host (inside the allocation)."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))

import paper_1511_05578_gb300 as crv  # noqa: E402
from paper_1511_05578_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
PAD = 4096  # sentinel elements after each caller buffer
SENT = 12345.5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


class Guarded:
    """Device buffers with a sentinel tail of PAD elements each."""

    def __init__(self):
        self.bufs = []

    def new(self, shape, dtype):
        n = int(np.prod(shape))
        full = torch.full((n + PAD,), SENT, dtype=dtype, device="cuda")
        self.bufs.append((full, n))
        return full[:n].view(shape)

    def like(self, t):
        return None if t is None else self.new(tuple(t.shape), t.dtype)

    def intact(self):
        return all(bool((full[n:] == SENT).all()) for full, n in self.bufs)


def _round_trip(L, lam, J0, s, flags, B=1, max_batch=1, rotate=False):
    real = bool(flags & crv.CRV_F_REAL)
    p = crv.Plan(L, lam, J0, s, flags | crv.CRV_F_GUARD, max_batch=max_batch)
    assert crv.crv_plan_guard_count(p.handle) > 0
    g = Guarded()
    flm = g.like(p.flm_tensor(B))
    for b in range(B):
        flm[b].copy_(torch.from_numpy(inputs.flm_gaussian(L, 100 + b, s, real, 3.0 if s else 2.0)))
    fmap, out, flm2 = g.like(p.map_tensor(B)), g.like(p.map_tensor(B)), g.like(p.flm_tensor(B))
    W = [g.like(w) for w in p.W_tensors(B)]
    Wphi = g.like(p.Wphi_tensor(B))
    crv.crv_sht_inv(p.handle, flm, fmap, B)
    crv.crv_sht_fwd(p.handle, fmap, flm2, B)
    crv.crv_analysis(p.handle, fmap, W, Wphi, B)
    crv.crv_synthesis(p.handle, W, Wphi, out, B)
    crv.crv_analysis_lm(p.handle, flm, W, Wphi, B)
    crv.crv_synthesis_lm(p.handle, W, Wphi, flm2, B)
    if rotate:
        for j in (J0, p.J):
            wt = g.like(p.wigner_edge_tensor(j, B))
            wt.copy_(torch.randn(wt.shape, dtype=wt.dtype, device="cuda"))
            w = g.like(p.wigner_tensor(j, B))
            crv.crv_rotate_wigner(p.handle, j, wt, w, B)
            crv.crv_rotate_wigner_adjoint(p.handle, j, w, wt, B)
    crv.crv_plan_check(p.handle)
    st, nbad = crv.crv_plan_check_guards(p.handle)
    rt = float(torch.linalg.vector_norm(out - fmap) / torch.linalg.vector_norm(fmap))
    ok_tails = g.intact()
    p.close()
    assert st == crv.CRV_OK and nbad == 0, crv.crv_last_error()
    assert ok_tails, "a caller buffer was written past its end"
    return rt


@pytest.mark.parametrize("name,L,lam,J0,s,flags,B,max_batch,tol", [
    ("mixed real, four maps on workers", 64, 2.0, 2, 0, crv.CRV_F_REAL | crv.CRV_F_MIXED | crv.CRV_F_W_FP32, 4, 4, 1e-5),
    ("plain FP64, complex spin 2", 33, 2.0, 1, 2, 0, 1, 1, 1e-12),
    ("plain FP64, odd lambda", 45, 1.7, 1, -1, 0, 1, 1, 1e-12),
])
def test_guards_intact(name, L, lam, J0, s, flags, B, max_batch, tol):
    assert _round_trip(L, lam, J0, s, flags, B, max_batch) < tol, name


def test_guards_intact_fp64_tensor_cores_many_passes(monkeypatch):
    monkeypatch.setenv("CRV_FP64_TC_A_GB", "0.001")
    assert _round_trip(40, 2.0, 2, 0, crv.CRV_F_REAL | crv.CRV_F_FP64_TC) < 1e-12


def test_guards_intact_unrotated_and_rotation():
    assert _round_trip(48, 2.0, 2, 0, crv.CRV_F_REAL | crv.CRV_F_MIXED | crv.CRV_F_UNROTATED, rotate=True) < 1e-5


def test_guards_intact_full_size():
    """The benchmark's kernels (L = 1024 mixed, P = 4096 FFTs, tensor-core tables) and the
    FP64 ones at L = 520."""
    assert _round_trip(1024, 2.0, 2, 0, crv.CRV_F_REAL | crv.CRV_F_MIXED | crv.CRV_F_W_FP32) < 1e-5
    assert _round_trip(520, 2.0, 2, 0, crv.CRV_F_REAL) < 1e-12


def test_guard_check_finds_a_changed_byte():
    p = crv.Plan(16, 2.0, 0, 0, crv.CRV_F_REAL | crv.CRV_F_GUARD)
    n = crv.crv_plan_guard_count(p.handle)
    assert crv.crv_plan_check_guards(p.handle) == (crv.CRV_OK, 0)
    crv.crv_debug_poke_guard(p.handle, 0)
    crv.crv_debug_poke_guard(p.handle, n - 1)
    st, nbad = crv.crv_plan_check_guards(p.handle)
    assert st == crv.CRV_EGUARD and nbad == 2
    assert "guard 0" in crv.crv_last_error()
    p.close()
    q = crv.Plan(16, 2.0, 0, 0, crv.CRV_F_REAL)
    assert crv.crv_plan_guard_count(q.handle) == 0
    with pytest.raises(crv.CrvError):
        crv.crv_plan_check_guards(q.handle)
    q.close()
