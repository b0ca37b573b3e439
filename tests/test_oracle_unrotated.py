"""Pins of the oracle's unrotated curvelet coefficients W~ (Sec. III-A-1) against things other
than itself: the rotation convention of the Wigner matrices (D(rho rho*) = D(rho) D(rho*) with the
factorial-sum d), the geometric relation W(rho) = W~(rho rho*) of Eq. (rotateWigner) between the
pinned rotated coefficients and a brute-force sum at the composed rotation, brute force on the
grid, the |n| = l sparsity of Eq. (curvelet_Wigner_property), exact reconstruction and the
single-scale closed form of synthesis."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1511_05578_gb300 import inputs as I


@pytest.mark.parametrize("s", [0, 2, -1])
def test_unrotated_zeta_support_and_normalisation(s):
    Lj = 16
    z = O.zeta_unrotated(s, Lj)
    n = np.arange(-(Lj - 1), Lj)
    for l in range(Lj):
        if l < abs(s):
            assert not z[l].any()
            continue
        assert np.all(z[l][np.abs(n) != l] == 0.0)  # |n| = l only (Sec. II-B)
        if l > 0:
            assert abs(np.sum(z[l] ** 2) - 1.0) < 1e-15  # Eq. directionality_normalisation
            assert z[l, Lj - 1 - l] == (-1) ** l * z[l, Lj - 1 + l]


def _D(l, a, b, g):
    m = np.arange(-l, l + 1)
    d = np.array([[O.wigner_d_factsum(l, mm, nn, b) for nn in m] for mm in m])
    return np.exp(-1j * m * a)[:, None] * d * np.exp(-1j * m * g)[None, :]


def test_euler_composition_matches_wigner_matrices():
    """The Euler angles of R(rho) R(rho*) give D^l(rho rho*) = D^l(rho) D^l(rho*) for l <= 3:
    euler_matrix/euler_angles follow the convention of the oracle's D."""
    rng = np.random.default_rng(5)
    for _ in range(6):
        r1 = (rng.uniform(0, 2 * np.pi), rng.uniform(0.1, 3.0), rng.uniform(0, 2 * np.pi))
        r2 = (0.0, rng.uniform(0.1, 3.0), 0.0)
        rc = O.euler_angles(O.euler_matrix(*r1) @ O.euler_matrix(*r2))
        for l in range(1, 4):
            assert np.abs(_D(l, *rc) - _D(l, *r1) @ _D(l, *r2)).max() < 1e-13


@pytest.mark.parametrize("lam,J0,s,L,real", [(2.0, 0, 0, 5, True), (2.0, 1, 2, 6, False), (1.6, 1, -1, 5, False)])
def test_rotated_equals_unrotated_at_composed_rotation(lam, J0, s, L, real):
    """Eq. (rotateWigner): W(rho) = W~(rho rho*), rho* = (0, vartheta^j, 0), vartheta^j =
    arccos(-s/lam^j). W from the (brute-force-pinned) grid analysis, W~ by the direct sum at the
    off-grid composed rotation."""
    f = I.flm_gaussian(L, 31, spin=s, real=real)
    rng = np.random.default_rng(L + 7 * abs(s))
    for j in range(J0, O.J_max(lam, L) + 1):
        Lj = O.band_limit(lam, j, L)
        N = 2 * Lj - 1
        W = O.analysis_rings(f, lam, j, s, L)
        pst = O.psi(lam, j, s, Lj, unrotated=True)
        th = math.acos(-s / lam ** j)
        for _ in range(4):
            a, b, g = (int(x) for x in (rng.integers(N), rng.integers(Lj), rng.integers(N)))
            rho = (2 * np.pi * a / N, np.pi * (2 * b + 1) / N, 2 * np.pi * g / N)
            rc = O.euler_angles(O.euler_matrix(*rho) @ O.euler_matrix(0.0, th, 0.0))
            got = O.analysis_point(f, pst, Lj, *rc)
            assert abs(got - W[b, a, g]) < 1e-13 * max(1.0, abs(W[b, a, g]))


def _brute_W(flm, psi_j, Lj, b):
    N = 2 * Lj - 1
    ang = 2 * np.pi * np.arange(N) / N
    beta = np.pi * (2 * b + 1) / N
    out = np.zeros((N, N), dtype=np.complex128)
    for l in range(Lj):
        for m in range(-l, l + 1):
            for n in (-l, l) if l else (0,):
                c = flm[l * l + l + m] * psi_j[l, n + Lj - 1] * O.wigner_d_factsum(l, m, n, beta)
                if c != 0:
                    out += c * np.exp(1j * m * ang)[:, None] * np.exp(1j * n * ang)[None, :]
    return out


@pytest.mark.parametrize("lam,J0,s,L,real", [(2.0, 0, 0, 6, True), (2.0, 1, 2, 5, False)])
def test_unrotated_grid_against_brute_force(lam, J0, s, L, real):
    f = I.flm_gaussian(L, 41, spin=s, real=real)
    mp = O.sht_inverse(f, L, s)
    _, W, _ = O.analysis(mp, lam, J0, s, L, unrotated=True)
    for j in W:
        Lj = O.band_limit(lam, j, L)
        ps = O.psi(lam, j, s, Lj, unrotated=True)
        for b in range(Lj):
            assert np.abs(W[j][b] - _brute_W(f, ps, Lj, b)).max() < 1e-13
            if real:
                assert np.abs(W[j][b].imag).max() < 1e-14


def test_unrotated_wigner_coefficients_sparse():
    """Eq. (curvelet_Wigner_property): the Wigner coefficients of W~_j recovered by the forward
    quadrature are (8pi^2/(2l+1)) f_lm psi~_ln, zero unless |n| = l."""
    L, lam, s = 12, 2.0, 0
    f = I.flm_gaussian(L, 9, real=True)
    j = O.J_max(lam, L)
    Lj = O.band_limit(lam, j, L)
    W = O.analysis_rings(f, lam, j, s, L, unrotated=True)
    coef = O.wigner_forward_coeffs(W, Lj)
    ps = O.psi(lam, j, s, Lj, unrotated=True)
    want = np.zeros_like(coef)
    for l in range(Lj):
        for m in range(-l, l + 1):
            for n in range(-l, l + 1):
                want[l, m + Lj - 1, n + Lj - 1] = 8 * np.pi ** 2 / (2 * l + 1) * f[l * l + l + m] * ps[l, n + Lj - 1]
    assert np.abs(coef - want).max() < 1e-12 * np.abs(want).max()
    n = np.arange(-(Lj - 1), Lj)
    for l in range(Lj):
        assert np.abs(coef[l][:, np.abs(n) != l]).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("lam,J0,s,L,real", [(2.0, 1, 0, 8, True), (2.0, 2, 0, 16, True), (2.0, 2, 2, 12, False),
                                             (1.7, 1, -1, 10, False), (3.0, 0, 1, 9, False)])
def test_unrotated_exact_reconstruction_and_single_scale(lam, J0, s, L, real):
    f = I.flm_gaussian(L, 5 + L, spin=s, real=real)
    mp = O.sht_inverse(f, L, s)
    flm, W, Wphi = O.analysis(mp, lam, J0, s, L, unrotated=True)
    fr = O.synthesis_flm(W, Wphi, lam, J0, s, L, unrotated=True)
    assert np.abs(fr - f).max() < 1e-13
    mr = O.synthesis(W, Wphi, lam, J0, s, L, unrotated=True)
    assert np.abs(mr - mp).max() < 1e-13
    # scale j alone gives f_lm kappa^(j)(l)^2 (Sum_n |zeta~_ln|^2 = 1 for l >= 1)
    l = np.floor(np.sqrt(np.arange(L * L))).astype(int)
    for j in W:
        g = O.synthesis_flm({j: W[j]}, None, lam, J0, s, L, unrotated=True)
        assert np.abs(g - f * O.kappa(lam, j, L)[l] ** 2).max() < 1e-13


def test_planted_wrong_sign_of_zeta_is_caught():
    """A zeta~_{l,-l} without its (-1)^l breaks Eq. (rotateWigner) for the odd-l content."""
    L, lam, s = 5, 2.0, 0
    f = I.flm_gaussian(L, 31, real=True)
    j = O.J_max(lam, L) - 1  # support l = 3, 4: one odd l
    Lj = O.band_limit(lam, j, L)
    assert np.abs(O.psi(lam, j, s, Lj, unrotated=True)[3]).max() > 0.1
    N = 2 * Lj - 1
    W = O.analysis_rings(f, lam, j, s, L)
    bad = np.abs(O.psi(lam, j, s, Lj, unrotated=True))
    rho = (2 * np.pi * 2 / N, np.pi * 3 / N, 2 * np.pi * 5 / N)
    rc = O.euler_angles(O.euler_matrix(*rho) @ O.euler_matrix(0.0, math.pi / 2, 0.0))
    assert abs(O.analysis_point(f, bad, Lj, *rc) - W[1, 2, 5]) > 1e-6
