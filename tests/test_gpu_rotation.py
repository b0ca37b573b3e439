"""Rotation of Wigner coefficients on the GPU (crv_rotate_wigner and its adjoint, Sec. III-A-1,
Eqs. curvelet_Wigner, curvelet_Wigner_inverse, rotateWigner) against the FP64 oracle: random
coefficients supported on |m|, |n| <= l, element-wise to 1e-13 of the largest entry, for spins
0, 2, -1 and several lambda, band limits (odd and even) and scales; batches; argument errors."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))

import oracle as O  # noqa: E402
import paper_1511_05578_gb300 as crv  # noqa: E402
from gpu_util import max_rel  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _random_edge(rng, Lj):
    N = 2 * Lj - 1
    wt = np.zeros((2, Lj, N), dtype=np.complex128)
    for l in range(Lj):
        ms = slice(Lj - 1 - l, Lj + l)
        wt[0][l, ms] = rng.normal(size=2 * l + 1) + 1j * rng.normal(size=2 * l + 1)
        if l > 0:
            wt[1][l, ms] = rng.normal(size=2 * l + 1) + 1j * rng.normal(size=2 * l + 1)
    return wt


def _random_dense(rng, Lj):
    N = 2 * Lj - 1
    w = np.zeros((Lj, N, N), dtype=np.complex128)
    for l in range(Lj):
        ms = slice(Lj - 1 - l, Lj + l)
        w[l, ms, ms] = rng.normal(size=(2 * l + 1, 2 * l + 1)) + 1j * rng.normal(size=(2 * l + 1, 2 * l + 1))
    return w


@pytest.mark.parametrize("L,lam,J0,s", [(64, 2.0, 2, 0), (33, 2.0, 1, 2), (20, 1.7, 1, -1), (45, 3.0, 1, 1)])
def test_rotation_matches_oracle(L, lam, J0, s):
    rng = np.random.default_rng(L)
    p = crv.Plan(L, lam, J0, s, crv.CRV_F_REAL if s == 0 else 0)
    for j in range(J0, p.J + 1):
        Lj = p.Lj[j]
        wt = _random_edge(rng, Lj)
        dwt = p.wigner_edge_tensor(j, 1)
        dwt.copy_(torch.from_numpy(wt[None]))
        dw = p.wigner_tensor(j, 1)
        dw.fill_(float("nan"))
        crv.crv_rotate_wigner(p.handle, j, dwt, dw, 1)
        want = O.rotate_wigner(wt, lam, j, s, Lj)
        got = dw[0].cpu().numpy()
        assert max_rel(got, want) < 1e-13, (j, max_rel(got, want))
        w = _random_dense(rng, Lj)
        dw.copy_(torch.from_numpy(w[None]))
        dwt.fill_(float("nan"))
        crv.crv_rotate_wigner_adjoint(p.handle, j, dw, dwt, 1)
        want = O.rotate_wigner_adjoint(w, lam, j, s, Lj)
        got = dwt[0].cpu().numpy()
        assert max_rel(got, want) < 1e-13, (j, max_rel(got, want))
    p.close()


def test_rotation_batch_roundtrip_and_errors():
    L, lam, J0, s = 48, 2.0, 2, 2
    rng = np.random.default_rng(7)
    p = crv.Plan(L, lam, J0, s, 0, max_batch=2)
    j = p.J
    Lj = p.Lj[j]
    wt = np.stack([_random_edge(rng, Lj) for _ in range(2)])
    dwt = p.wigner_edge_tensor(j, 2)
    dwt.copy_(torch.from_numpy(wt))
    dw = p.wigner_tensor(j, 2)
    crv.crv_rotate_wigner(p.handle, j, dwt, dw, 2)
    back = p.wigner_edge_tensor(j, 2)
    crv.crv_rotate_wigner_adjoint(p.handle, j, dw, back, 2)
    assert max_rel(back.cpu().numpy(), wt) < 1e-13       # the adjoint inverts the rotation
    for b in range(2):
        assert max_rel(dw[b].cpu().numpy(), O.rotate_wigner(wt[b], lam, j, s, Lj)) < 1e-13
    with pytest.raises(crv.CrvError):
        crv.crv_rotate_wigner(p.handle, J0 - 1, dwt, dw, 1)   # scale below J0
    with pytest.raises(crv.CrvError):
        crv.crv_rotate_wigner(p.handle, j, dwt, dw, 3)        # B > max_batch
    crv.crv_rotate_wigner(p.handle, j, dwt, dw, 0)            # empty batch is a no-op
    p.close()
