"""Pins of the oracle's spin spherical harmonic transform on the MW grid:
low-l closed forms (golden), scipy's spherical harmonics, the conjugate-symmetry
relation of the spin harmonics, and forward o inverse = identity (the inverse is
the direct sum of Eq. spin_sphericalHarmonics; the forward is the
extension-and-weights quadrature, so any slip in the forward fails it)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1511_05578_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_low_l_harmonics_closed_form():
    data = json.load(open(os.path.join(GOLD, "sht_low_l.json")))
    L = 5
    th, ph = O.mw_theta(L), O.mw_phi(L)
    T, P = np.meshgrid(th, ph, indexing="ij")
    for e in data["entries"]:
        f = np.zeros(L * L, dtype=np.complex128)
        f[e["l"] ** 2 + e["l"] + e["m"]] = 1.0
        got = O.sht_inverse(f, L, 0)
        want = eval(e["expr"], {"sqrt": np.sqrt, "cos": np.cos, "sin": np.sin, "exp": np.exp, "pi": np.pi},
                    {"theta": T, "phi": P})
        assert np.abs(got - want).max() < 1e-15


def test_spin0_against_scipy():
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    L = 7
    th, ph = O.mw_theta(L), O.mw_phi(L)
    T, P = np.meshgrid(th, ph, indexing="ij")
    f = I.flm_gaussian(L, 11, spin=0, real=False)
    want = np.zeros_like(T, dtype=np.complex128)
    for l in range(L):
        for m in range(-l, l + 1):
            want += f[l * l + l + m] * special.sph_harm_y(l, m, T, P)
    assert np.abs(O.sht_inverse(f, L, 0) - want).max() < 1e-13


@pytest.mark.parametrize("s", [1, 2, -3])
def test_spin_conjugate_symmetry(s):
    """sY*_lm = (-1)^{s+m} (-s)Y_{l,-m} (footnote to Eq. spin_sphericalHarmonics)."""
    L = 6
    for l in range(abs(s), L):
        for m in range(-l, l + 1):
            f = np.zeros(L * L, dtype=np.complex128)
            f[l * l + l + m] = 1.0
            g = np.zeros(L * L, dtype=np.complex128)
            g[l * l + l - m] = 1.0
            a = np.conj(O.sht_inverse(f, L, s))
            b = (-1) ** (s + m) * O.sht_inverse(g, L, -s)
            assert np.abs(a - b).max() < 1e-14


@pytest.mark.parametrize("L,s,real", [(1, 0, True), (2, 0, False), (8, 0, True), (9, -1, False),
                                      (16, 2, False), (33, 3, False), (64, 0, True)])
def test_forward_inverts_inverse(L, s, real):
    f = I.flm_gaussian(L, 7 + L, spin=s, real=real)
    mp = O.sht_inverse(f, L, s)
    if real:
        assert np.abs(mp.imag).max() < 1e-14
    f2 = O.sht_forward(mp, L, s)
    assert np.abs(f2 - f).max() < 5e-15 * max(1, L / 8)


def test_forward_orthonormal_quadrature():
    """The quadrature recovers a single harmonic exactly (orthonormality of the
    sY_lm under the exact MW quadrature)."""
    L = 10
    for (l, m, s) in [(0, 0, 0), (4, -3, 0), (9, 9, 1), (5, 2, -2), (9, -8, 4)]:
        f = np.zeros(L * L, dtype=np.complex128)
        f[l * l + l + m] = 1.0
        g = O.sht_forward(O.sht_inverse(f, L, s), L, s)
        assert np.abs(g - f).max() < 1e-14


@pytest.mark.parametrize("mut", ["ext_sign", "half_phase", "weight_sign"])
def test_planted_mistakes_are_caught(mut):
    """A deliberate slip planted in the oracle's quadrature (wrong extension sign,
    missing half-sample phase, sign slip in the even-p weights) breaks forward o inverse."""
    L, s = 12, 1
    f = I.flm_gaussian(L, 5, spin=s)
    mp = O.sht_inverse(f, L, s)
    O.MUTATION[mut] = True
    try:
        f2 = O.sht_forward(mp, L, s)
    finally:
        O.MUTATION[mut] = False
    assert np.abs(f2 - f).max() > 1e-3


def test_odd_weights_cancel():
    """The p = +-1 weights never contribute: the extended integrand has parity
    (-1)^{m+s} in beta, so their terms cancel in pairs over +-m'. (A fact the CUDA
    path relies on; pinned here on the oracle.)"""
    L, s = 12, 1
    f = I.flm_gaussian(L, 5, spin=s)
    mp = O.sht_inverse(f, L, s)
    w1 = O.quad_weight(np.array([1, -1]))
    assert abs(w1[0]) > 1
    orig = O.curvelet.quad_weight

    def no_odd(p):
        w = orig(p)
        w[np.abs(np.asarray(p)) == 1] = 0.0
        return w
    O.curvelet.quad_weight = no_odd
    try:
        f2 = O.sht_forward(mp, L, s)
    finally:
        O.curvelet.quad_weight = orig
    assert np.abs(f2 - f).max() < 1e-14
