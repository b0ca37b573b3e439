"""Pins of the oracle's curvelet construction, analysis and synthesis against
things other than itself: scipy quadrature of k_lambda, the admissibility
identity (Eq. admissibility), the literal rotation of the directional component
with the factorial-sum d (Eq. wigner_sum_reln), brute-force evaluation of Eq.
(wav_analysis_harmonic) at every SO(3) grid point for tiny L, brute-force Wigner
coefficients, exact reconstruction, the single-scale closed form of synthesis,
Parseval, and planted mistakes."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1511_05578_gb300 import inputs as I


def _k_scipy(lam, t):
    integrate = pytest.importorskip("scipy.integrate")

    def s(x):
        return math.exp(-1.0 / (1.0 - x * x)) if -1 < x < 1 else 0.0

    def g(x):
        v = s(2 * lam / (lam - 1) * (x - 1 / lam) - 1)
        return v * v / x
    if t < 1 / lam:
        return 1.0
    if t >= 1:
        return 0.0
    num = integrate.quad(g, t, 1, epsabs=1e-16, epsrel=1e-13, limit=400)[0]
    den = integrate.quad(g, 1 / lam, 1, epsabs=1e-16, epsrel=1e-13, limit=400)[0]
    return num / den


@pytest.mark.parametrize("lam", [2.0, 1.5, 3.0])
def test_k_lambda_against_scipy(lam):
    for t in np.linspace(1 / lam - 0.05, 1.02, 23):
        assert abs(O.k_lambda(lam, t) - _k_scipy(lam, t)) < 1e-12


@pytest.mark.parametrize("lam,J0,L", [(2.0, 2, 64), (2.0, 0, 33), (1.5, 1, 40), (3.0, 1, 100), (2.0, 3, 1024)])
def test_kernel_support_peak_and_admissibility(lam, J0, L):
    J = O.J_max(lam, L)
    assert lam ** J >= L * (1 - 1e-12) and (J == 0 or lam ** (J - 1) < L)
    tot = O.phi_scaling(lam, J0, L) ** 2
    l = np.arange(L)
    for j in range(J0, J + 1):
        k = O.kappa(lam, j, L)
        inside = (l > lam ** (j - 1)) & (l < lam ** (j + 1))
        assert np.all(k[~inside] == 0.0)
        # strictly positive on the open support (Sec. II-B: the bump vanishes only at its ends)
        assert np.all(k[inside] > 0.0)
        Lj = O.band_limit(lam, j, L)
        assert np.all(k[Lj:] == 0.0)
        pk = lam ** j
        if abs(pk - round(pk)) < 1e-12 and round(pk) < L:
            assert abs(k[int(round(pk))] - 1.0) < 1e-15  # peak of unity at l = lam^j
        tot = tot + k ** 2
    # Eq. (admissibility), with Sum_n |zeta_ln|^2 = 1 folded in
    assert np.abs(tot - 1.0).max() < 1e-14


@pytest.mark.parametrize("s", [0, 2, -1])
def test_zeta_normalised_and_rotated(s):
    lam, L = 2.0, 24
    for j in range(3, 6):
        Lj = O.band_limit(lam, j, L)
        z = O.zeta(lam, j, s, Lj)
        for l in range(max(1, abs(s)), Lj):
            assert abs(np.sum(z[l] ** 2) - 1.0) < 1e-14  # Eq. directionality_normalisation
        # literal rotation sum_n d^l_kn(vartheta) zeta~_ln with the factorial sum
        th = math.acos(-s / lam ** j)
        for l in range(max(1, abs(s)), min(Lj, 12)):
            for k in range(-l, l + 1):
                want = (O.wigner_d_factsum(l, k, l, th) + (-1) ** l * O.wigner_d_factsum(l, k, -l, th)) / math.sqrt(2)
                assert abs(z[l, k + Lj - 1] - want) < 1e-14
        if s == 0:
            for l in range(1, Lj):
                D = O.delta_matrix(l)
                k = np.arange(-l, l + 1)
                want = np.where(k % 2 == 0, math.sqrt(2) * D[:, 2 * l], 0.0)
                assert np.abs(z[l, Lj - 1 - l: Lj + l] - want).max() < 1e-14


def _brute_W(flm, psi_j, Lj, b):
    """Eq. (wav_analysis_harmonic) at every (alpha_a, gamma_g) of ring b, with
    D^{l*}_mn(rho) = e^{i m a} d^l_mn(b) e^{i n g} and d from the factorial sum."""
    N = 2 * Lj - 1
    a = 2 * np.pi * np.arange(N) / N
    beta = np.pi * (2 * b + 1) / N
    W = np.zeros((N, N), dtype=np.complex128)
    for l in range(Lj):
        for m in range(-l, l + 1):
            for n in range(-l, l + 1):
                c = flm[l * l + l + m] * psi_j[l, n + Lj - 1] * O.wigner_d_factsum(l, m, n, beta)
                if c != 0:
                    W += c * np.exp(1j * m * a)[:, None] * np.exp(1j * n * a)[None, :]
    return W


@pytest.mark.parametrize("lam,J0,s,L,real", [(2.0, 0, 0, 5, True), (2.0, 1, 2, 6, False), (1.6, 1, -1, 5, False)])
def test_analysis_against_brute_force(lam, J0, s, L, real):
    f = I.flm_gaussian(L, 21, spin=s, real=real)
    mp = O.sht_inverse(f, L, s)
    flm, W, Wphi = O.analysis(mp, lam, J0, s, L)
    assert np.abs(flm - f).max() < 1e-14
    for j in W:
        Lj = O.band_limit(lam, j, L)
        ps = O.psi(lam, j, s, Lj)
        for b in range(Lj):
            assert np.abs(W[j][b] - _brute_W(f, ps, Lj, b)).max() < 1e-13
            if real:
                assert np.abs(W[j][b].imag).max() < 1e-14
    # scaling map: inverse spin-0 SHT of sqrt(k(l/lam^J0)) f_lm (Eq. analysis_scaling_harmonic)
    Lp = O.L_phi(lam, J0, L)
    th, ph = O.mw_theta(Lp), O.mw_phi(Lp)
    want = np.zeros((Lp, 2 * Lp - 1), dtype=np.complex128)
    for l in range(min(Lp, L)):
        for m in range(-l, l + 1):
            y = math.sqrt((2 * l + 1) / (4 * math.pi)) * np.array([O.wigner_d_factsum(l, m, 0, t) for t in th])
            want += math.sqrt(O.k_lambda(lam, l / lam ** J0)) * f[l * l + l + m] * y[:, None] * np.exp(1j * m * ph)[None, :]
    assert np.abs(Wphi - want).max() < 1e-14


def test_analysis_ring_methods_agree():
    """Risbo-at-beta and l-recurrence evaluations of the same rings agree (to the
    l-recurrence's rounding growth near the pole ring, ~1e-13 at L = 96)."""
    L, lam = 96, 2.0
    f = I.flm_gaussian(L, 1, real=True)
    for j in [5, 6]:
        a = O.analysis_rings(f, lam, j, 0, L, rings=[0, 17, O.band_limit(lam, j, L) - 1])
        b = O.analysis_rings(f, lam, j, 0, L, rings=[0, 17, O.band_limit(lam, j, L) - 1], method="lrec")
        assert np.abs(a - b).max() < 5e-13


def test_alpha_shift_covariance():
    """f_lm -> f_lm e^{-i m alpha_k} rotates the map by alpha_k about z, which
    shifts every W_j by k samples in alpha (Eq. wav_analysis_harmonic)."""
    L, lam, J0, s = 12, 2.0, 1, 0
    f = I.flm_gaussian(L, 4, real=True)
    J = O.J_max(lam, L)
    j = J
    Lj = O.band_limit(lam, j, L)
    N = 2 * Lj - 1
    k = 3
    l = np.floor(np.sqrt(np.arange(L * L))).astype(int)
    m = np.arange(L * L) - l * l - l
    g = f * np.exp(-1j * m * 2 * np.pi * k / N)
    Wf = O.analysis_rings(f, lam, j, s, L)
    Wg = O.analysis_rings(g, lam, j, s, L)
    assert np.abs(Wg - np.roll(Wf, k, axis=1)).max() < 1e-14


def _wigner_brute_grid(coef, Lj):
    """W on the grid from dense Wigner coefficients coef[l][m][n] by the direct
    inverse sum W = sum (2l+1)/(8 pi^2) W^l_mn D^{l*}_mn (factorial-sum d)."""
    N = 2 * Lj - 1
    a = 2 * np.pi * np.arange(N) / N
    W = np.zeros((Lj, N, N), dtype=np.complex128)
    for b in range(Lj):
        beta = np.pi * (2 * b + 1) / N
        for l in range(Lj):
            for m in range(-l, l + 1):
                for n in range(-l, l + 1):
                    c = coef[l, m + Lj - 1, n + Lj - 1]
                    if c != 0:
                        W[b] += (2 * l + 1) / (8 * np.pi ** 2) * c * O.wigner_d_factsum(l, m, n, beta) * \
                            np.exp(1j * m * a)[:, None] * np.exp(1j * n * a)[None, :]
    return W


def test_forward_wigner_recovers_brute_force_coefficients():
    """The forward Wigner quadrature (Eqs. Fmn..flml, general n) inverts the
    direct inverse sum for arbitrary band-limited coefficients."""
    Lj = 4
    N = 2 * Lj - 1
    rng = np.random.default_rng(0)
    coef = np.zeros((Lj, N, N), dtype=np.complex128)
    for l in range(Lj):
        for m in range(-l, l + 1):
            for n in range(-l, l + 1):
                coef[l, m + Lj - 1, n + Lj - 1] = rng.normal() + 1j * rng.normal()
    W = _wigner_brute_grid(coef, Lj)
    got = O.wigner_forward_coeffs(W, Lj)
    assert np.abs(got - coef).max() < 1e-12


@pytest.mark.parametrize("lam,J0,s,L,real", [(2.0, 1, 0, 8, True), (2.0, 2, 0, 16, True), (2.0, 2, 2, 12, False),
                                             (1.7, 1, -1, 10, False), (2.0, 2, 0, 33, True), (3.0, 0, 1, 9, False)])
def test_exact_reconstruction(lam, J0, s, L, real):
    f = I.flm_gaussian(L, 3 + L, spin=s, real=real)
    mp = O.sht_inverse(f, L, s)
    flm, W, Wphi = O.analysis(mp, lam, J0, s, L)
    fr = O.synthesis_flm(W, Wphi, lam, J0, s, L)
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) < 1e-13
    assert np.abs(fr - f).max() < 1e-13
    mr = O.synthesis(W, Wphi, lam, J0, s, L)
    assert np.abs(mr - mp).max() < 1e-13


def test_single_scale_closed_form_and_parseval():
    """Synthesis of one scale alone gives f_lm kappa^(j)(l)^2 (Sum_n |zeta_ln|^2 = 1),
    scaling alone gives f_lm k(l/lam^J0); Parseval in harmonic space."""
    lam, J0, s, L = 2.0, 1, 2, 12
    f = I.flm_gaussian(L, 8, spin=s)
    W, Wphi = O.analysis_from_flm(f, lam, J0, s, L)
    l = np.floor(np.sqrt(np.arange(L * L))).astype(int)
    energy = np.sum(np.abs(O.phi_scaling(lam, J0, L)[l] * f) ** 2)
    for j in W:
        part = O.synthesis_flm({j: W[j]}, None, lam, J0, s, L)
        want = f * O.kappa(lam, j, L)[l] ** 2
        want[: s * s] = 0
        assert np.abs(part - want).max() < 1e-14
        Lj = O.band_limit(lam, j, L)
        coef = O.wigner_forward_coeffs(W[j], Lj)
        ll = np.arange(Lj)[:, None, None]
        energy += np.sum((2 * ll + 1) / (8 * np.pi ** 2) * np.abs(coef) ** 2)
    part = O.synthesis_flm({}, Wphi, lam, J0, s, L)
    want = f * O.phi_scaling(lam, J0, L)[l] ** 2
    want[: s * s] = 0
    assert np.abs(part - want).max() < 1e-14
    assert abs(energy - np.sum(np.abs(f) ** 2)) < 1e-13 * np.sum(np.abs(f) ** 2)


def test_north_pole_centring_spin0():
    """Rotated to the North pole (Sec. II-B): the spatial curvelet's largest
    magnitude at the finest scale lies at the pole ring (beta closest to 0)."""
    lam, L = 2.0, 32
    j = O.J_max(lam, L) - 1
    Lj = O.band_limit(lam, j, L)
    ps = O.psi(lam, j, 0, Lj)
    c = np.zeros(Lj * Lj, dtype=np.complex128)
    for l in range(Lj):
        for m in range(-l, l + 1):
            c[l * l + l + m] = ps[l, m + Lj - 1]
    mp = np.abs(O.sht_inverse(c, Lj, 0))
    t, _ = np.unravel_index(np.argmax(mp), mp.shape)
    assert t == 0


@pytest.mark.parametrize("mut", ["ext_sign", "half_phase", "weight_sign"])
def test_planted_mistakes_break_reconstruction(mut):
    lam, J0, s, L = 2.0, 1, 1, 8
    f = I.flm_gaussian(L, 2, spin=s)
    W, Wphi = O.analysis_from_flm(f, lam, J0, s, L)
    O.MUTATION[mut] = True
    try:
        fr = O.synthesis_flm(W, Wphi, lam, J0, s, L)
    finally:
        O.MUTATION[mut] = False
    assert np.abs(fr - f).max() > 1e-3
