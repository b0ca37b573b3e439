"""Pins of the oracle's rotation of Wigner coefficients (Sec. III-A-1: Eqs. curvelet_Wigner,
curvelet_Wigner_inverse, rotateWigner) against things other than itself:

  - the Wigner coefficients of the unrotated coefficients W~_j on the grid (the forward
    quadrature, pinned by brute force), rotated, equal those of the rotated W_j on the grid
    (pinned by brute-force evaluation of Eq. wav_analysis_harmonic): rotation in harmonic
    space is the composition W(rho) = W~(rho rho*) on the grid;
  - the closed forms (8 pi^2/(2l+1)) f_lm psi~_ln and (8 pi^2/(2l+1)) f_lm psi_ln
    (Eq. wav_harmonic_coeff) map onto each other;
  - the adjoint inverts the rotation (orthogonality of d^l);
  - a planted transposition of d^l (d_nk for d_kn) is caught.
"""
import numpy as np
import pytest

import oracle as O
from paper_1511_05578_gb300 import inputs as I


def _sparse_part(coef, Lj):
    """[2][Lj][2Lj-1]: the n = +l and n = -l columns of dense coefficients."""
    N = 2 * Lj - 1
    wt = np.zeros((2, Lj, N), dtype=np.complex128)
    for l in range(Lj):
        wt[0][l] = coef[l, :, Lj - 1 + l]
        if l > 0:
            wt[1][l] = coef[l, :, Lj - 1 - l]
    return wt


@pytest.mark.parametrize("lam,s,L,real", [(2.0, 0, 8, True), (2.0, 2, 12, False), (1.7, -1, 10, False),
                                          (3.0, 1, 9, False)])
def test_rotating_grid_coefficients(lam, s, L, real):
    f = I.flm_gaussian(L, 21 + L, spin=s, real=real, power=3.0 if s else 2.0)
    for j in sorted({O.J_max(lam, L), O.J_max(lam, L) - 1}):
        if lam ** j < abs(s):
            continue
        Lj = O.band_limit(lam, j, L)
        Wt = O.analysis_rings(f, lam, j, s, L, unrotated=True)
        W = O.analysis_rings(f, lam, j, s, L)
        ct = O.wigner_forward_coeffs(Wt, Lj)
        c = O.wigner_forward_coeffs(W, Lj)
        got = O.rotate_wigner(_sparse_part(ct, Lj), lam, j, s, Lj)
        assert np.abs(got - c).max() < 1e-12 * np.abs(c).max(), j
        back = O.rotate_wigner_adjoint(c, lam, j, s, Lj)
        assert np.abs(back - _sparse_part(ct, Lj)).max() < 1e-12 * np.abs(c).max(), j


@pytest.mark.parametrize("lam,s,L", [(2.0, 0, 24), (2.0, 2, 20), (1.7, -1, 18)])
def test_closed_forms_map_onto_each_other(lam, s, L):
    f = I.flm_gaussian(L, 5, spin=s, real=(s == 0), power=3.0 if s else 2.0)
    j = O.J_max(lam, L)
    Lj = O.band_limit(lam, j, L)
    N = 2 * Lj - 1
    pt = O.psi(lam, j, s, Lj, unrotated=True)
    pr = O.psi(lam, j, s, Lj)
    want = np.zeros((Lj, N, N), dtype=np.complex128)
    ct = np.zeros((Lj, N, N), dtype=np.complex128)
    for l in range(Lj):
        for m in range(-l, l + 1):
            a = 8 * np.pi ** 2 / (2 * l + 1) * f[l * l + l + m]
            ct[l, m + Lj - 1] = a * pt[l]
            want[l, m + Lj - 1] = a * pr[l]
    got = O.rotate_wigner(_sparse_part(ct, Lj), lam, j, s, Lj)
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_adjoint_inverts_rotation_on_random_coefficients():
    lam, s, Lj, j = 2.0, 2, 16, 3
    rng = np.random.default_rng(3)
    N = 2 * Lj - 1
    wt = np.zeros((2, Lj, N), dtype=np.complex128)
    for l in range(Lj):
        ms = slice(Lj - 1 - l, Lj + l)
        wt[0][l, ms] = rng.normal(size=2 * l + 1) + 1j * rng.normal(size=2 * l + 1)
        if l > 0:
            wt[1][l, ms] = rng.normal(size=2 * l + 1) + 1j * rng.normal(size=2 * l + 1)
    w = O.rotate_wigner(wt, lam, j, s, Lj)
    assert np.abs(O.rotate_wigner_adjoint(w, lam, j, s, Lj) - wt).max() < 1e-13
    # entries outside |m|, |k| <= l are zero
    for l in range(Lj):
        blk = w[l].copy()
        blk[Lj - 1 - l: Lj + l, Lj - 1 - l: Lj + l] = 0
        assert np.abs(blk).max() == 0.0


def test_planted_transposed_rotation_is_caught():
    lam, s, L = 2.0, 2, 12
    f = I.flm_gaussian(L, 4, spin=s, power=3.0)
    j = O.J_max(lam, L)
    Lj = O.band_limit(lam, j, L)
    ct = O.wigner_forward_coeffs(O.analysis_rings(f, lam, j, s, L, unrotated=True), Lj)
    c = O.wigner_forward_coeffs(O.analysis_rings(f, lam, j, s, L), Lj)
    O.MUTATION["rotation_transposed"] = True
    try:
        bad = O.rotate_wigner(_sparse_part(ct, Lj), lam, j, s, Lj)
    finally:
        O.MUTATION["rotation_transposed"] = False
    assert np.abs(bad - c).max() > 1e-3 * np.abs(c).max()
