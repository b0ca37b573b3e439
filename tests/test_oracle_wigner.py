"""Pins of the oracle's Wigner functions, Delta matrices and quadrature weights
against things other than themselves: hand-evaluated closed forms of Eq.
(wigner_sum_reln), the factorial sum itself (for the two recursions), exact
integer arithmetic, orthogonality, the Delta factorisation identity and
numerical integration (scipy)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _betas():
    return [1e-3, 0.37, 1.1, math.pi / 2, 2.5, math.pi - 1e-3]


def test_factsum_matches_closed_forms_l_le_2():
    """Eq. (wigner_sum_reln) against the l <= 2 closed forms (golden table),
    plus the symmetries used to fill the rest of each matrix."""
    data = json.load(open(os.path.join(GOLD, "wigner_d_l2.json")))
    for beta in _betas():
        env = {"c": math.cos(beta), "s": math.sin(beta), "sqrt": math.sqrt}
        for e in data["entries"]:
            l, m, n = e["l"], e["m"], e["n"]
            want = eval(e["expr"], {}, env)
            for (mm, nn, sgn) in [(m, n, 1), (-m, -n, (-1) ** (m + n)), (n, m, (-1) ** (m - n))]:
                got = O.wigner_d_factsum(l, mm, nn, beta)
                assert abs(got - sgn * want) < 1e-15, (l, mm, nn, beta, got, sgn * want)


@pytest.mark.parametrize("beta", _betas())
def test_lrec_matches_factsum(beta):
    """Three-term l-recurrence vs the factorial sum for l <= 14, all m, n. (The
    recurrence's rounding error grows near the poles, ~1e-14 here at beta=1e-3.)"""
    L = 15
    err = 0.0
    for m in range(-(L - 1), L):
        for n in range(-(L - 1), L):
            d = O.wigner_d_lrec(L, m, n, beta=beta)
            for l in range(L):
                err = max(err, abs(d[l] - O.wigner_d_factsum(l, m, n, beta)))
    assert err < 5e-14


def test_lrec_on_grid_endpoints():
    """At beta = pi (the last MW colatitude) d^l_mn = (-1)^{l+m} delta_{m,-n}
    (Eq. wigner_sum_reln with cos(beta/2) = 0: only the term with
    m + n + 2k = 0 survives)."""
    L = 9
    sh, ch = O.half_angles(L, L - 1)
    assert ch == 0.0
    for m in range(-(L - 1), L):
        for n in range(-(L - 1), L):
            d = O.wigner_d_lrec(L, m, n, sh=float(sh), ch=float(ch))
            for l in range(max(abs(m), abs(n)), L):
                want = (-1) ** (l + m) if m == -n else 0.0
                assert abs(d[l] - want) < 1e-14, (l, m, n, d[l])


@pytest.mark.parametrize("beta", [0.37, 2.5])
def test_risbo_matches_factsum(beta):
    for l in range(0, 13):
        M = O.risbo_matrix(l, beta=beta)
        for m in range(-l, l + 1):
            for n in range(-l, l + 1):
                assert abs(M[m + l, n + l] - O.wigner_d_factsum(l, m, n, beta)) < 5e-15


def test_delta_edge_column_exact():
    """Delta^l_{m,l} = 2^-l sqrt(C(2l, l+m)) from Eq. (wigner_sum_reln) at beta =
    pi/2 (one surviving term), compared in exact rational arithmetic."""
    for l in [1, 7, 40, 120]:
        D = O.delta_matrix(l)
        for m in range(-l, l + 1):
            exact = Fraction(math.comb(2 * l, l + m), 4 ** l)
            want = math.sqrt(exact.numerator) / math.sqrt(exact.denominator)
            assert abs(D[m + l, 2 * l] - want) <= 1e-13 * abs(want) + 1e-300  # Risbo: a few ulp per step


@pytest.mark.parametrize("l", [30, 200, 500])
def test_delta_orthogonal_and_symmetric(l):
    D = O.delta_matrix(l)
    assert np.abs(D.T @ D - np.eye(2 * l + 1)).max() < 1e-14 + 4e-16 * l  # grows ~linearly in l
    k = np.arange(-l, l + 1)
    # Delta^l_{m,-n} = (-1)^{l+m} Delta^l_{mn}; Delta^l_{-m,n} = (-1)^{l+n} Delta^l_{mn};
    # Delta^l_{nm} = (-1)^{m-n} Delta^l_{mn}
    sm = np.where((l + k) % 2 == 0, 1.0, -1.0)
    assert np.abs(D[:, ::-1] - sm[:, None] * D).max() < 1e-14
    assert np.abs(D[::-1, :] - sm[None, :] * D).max() < 1e-14
    smn = np.where((k[None, :] - k[:, None]) % 2 == 0, 1.0, -1.0)
    assert np.abs(D.T - smn * D).max() < 1e-14


@pytest.mark.parametrize("l", [5, 21, 64])
def test_delta_factorisation_identity(l):
    """d^l_mn(beta) = i^{n-m} sum_{m'} Delta^l_{m'm} Delta^l_{m'n} e^{i m' beta}
    (Sec. III-A-2): Risbo's Delta at pi/2 against the l-recurrence at beta."""
    D = O.delta_matrix(l)
    k = np.arange(-l, l + 1)
    rng = np.random.default_rng(l)
    for beta in rng.uniform(0.05, math.pi - 0.05, size=3):
        e = np.exp(1j * k * beta)
        for m in range(-l, l + 1, max(1, l // 7)):
            for n in range(-l, l + 1, max(1, l // 5)):
                d = O.wigner_d_lrec(l + 1, m, n, beta=float(beta))[l]
                val = (1j) ** (n - m) * np.sum(D[:, m + l] * D[:, n + l] * e)
                assert abs(val.imag) < 1e-13 and abs(val.real - d) < 1e-13, (l, m, n)


def test_lrec_large_l_against_factorisation():
    """At l = 700 (where naive seeds underflow double precision near the poles)
    the recurrence still matches the factorisation through Risbo's Delta; Risbo
    run directly at beta matches both."""
    l = 700
    D = O.delta_matrix(l)
    k = np.arange(-l, l + 1)
    for beta in [0.004, 1.3, 3.1]:
        e = np.exp(1j * k * beta)
        for (m, n) in [(0, 0), (700, -3), (-650, 640), (10, 699), (350, -351)]:
            d = O.wigner_d_lrec(l + 1, m, n, beta=beta)[l]
            val = ((1j) ** (n - m) * np.sum(D[:, m + l] * D[:, n + l] * e)).real
            assert abs(val - d) < 1e-11, (m, n, beta, val, d)
        R = O.risbo_matrix(l, beta=beta)
        for (m, n) in [(0, 0), (700, -3), (-650, 640), (10, 699), (350, -351), (5, 5)]:
            val = ((1j) ** (n - m) * np.sum(D[:, m + l] * D[:, n + l] * e)).real
            assert abs(val - R[m + l, n + l]) < 5e-13, (m, n, beta)


def test_quadrature_weights_against_integration():
    """w(p) = int_0^pi sin(b) e^{i p b} db (Eq. gmnmp) against scipy quad."""
    integrate = pytest.importorskip("scipy.integrate")
    for p in range(-9, 10):
        re = integrate.quad(lambda b: math.sin(b) * math.cos(p * b), 0, math.pi, epsabs=1e-14)[0]
        im = integrate.quad(lambda b: math.sin(b) * math.sin(p * b), 0, math.pi, epsabs=1e-14)[0]
        w = complex(O.quad_weight(np.array([p]))[0])
        assert abs(w - complex(re, im)) < 1e-13, (p, w, re, im)


def test_weights_reproduce_integral_of_band_limited_function():
    """The extension-and-weights quadrature of Sec. III-A-2 integrates
    sin(b) times a trigonometric polynomial of degree < L over [0, pi] exactly."""
    L = 11
    rng = np.random.default_rng(3)
    c = rng.normal(size=2 * L - 1) + 1j * rng.normal(size=2 * L - 1)
    k = np.arange(-(L - 1), L)
    exact = np.sum(c * O.quad_weight(k))
    integrate = pytest.importorskip("scipy.integrate")
    fr = lambda b: (np.sum(c * np.exp(1j * k * b)) * math.sin(b)).real
    fi = lambda b: (np.sum(c * np.exp(1j * k * b)) * math.sin(b)).imag
    num = integrate.quad(fr, 0, math.pi, epsabs=1e-13, limit=200)[0] + 1j * integrate.quad(fi, 0, math.pi, epsabs=1e-13, limit=200)[0]
    assert abs(exact - num) < 1e-12
