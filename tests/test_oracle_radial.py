"""Pins of the radial kernel reading (Sec. II-B: s, s_lambda, k_lambda, kappa_lambda)
against properties the paper's definitions fix, so that a misread affine map in
s_lambda, a wrong bump or a wrong weight in the k_lambda integral fails here even
though admissibility (which telescopes for any k) and the unit peak would still hold:

  - s(t) = exp(-1/(1-t^2)) on (-1, 1) and s_lambda(t) = s(2 lam/(lam-1) (t - 1/lam) - 1):
    zero outside [1/lam, 1], positive inside, symmetric about the centre
    (1 + 1/lam)/2 where it equals s(0) = e^-1, and s_lambda(t) = exp(-4/3) where the
    argument is -1/2 or 1/2 (t = 1/lam + (1 - 1/lam)/4 and its mirror);
  - k_lambda(t) = 1 up to 1/lam, 0 from 1 on, strictly decreasing in between;
  - k_lambda is the normalised integral of s_lambda(t)^2 / t, so its derivative is
    -s_lambda(t)^2 / (t C) with one constant C for every t (central differences);
  - kappa^(j)(l) > 0 for every integer l strictly inside (lam^(j-1), lam^(j+1)).
"""
import math

import numpy as np
import pytest

import oracle as O

LAMS = [2.0, 1.5, 3.0, 2.7]


@pytest.mark.parametrize("lam", LAMS)
def test_s_lambda_support_centre_symmetry(lam):
    a, b = 1.0 / lam, 1.0
    c = 0.5 * (a + b)
    # zero on and outside the ends of [1/lam, 1]
    for t in [a - 0.3, a - 1e-9, a, b, b + 1e-9, b + 0.5, 0.0]:
        assert O.s_lambda(lam, t) == 0.0, t
    # positive strictly inside
    inside = a + (b - a) * np.linspace(0.002, 0.998, 301)
    assert np.all(O.s_lambda(lam, inside) > 0.0)
    # centre value s(0) = e^-1
    assert abs(O.s_lambda(lam, c) - math.exp(-1.0)) < 1e-16
    # the argument is -1/2 and +1/2 a quarter of the support from either end: exp(-4/3)
    q = (b - a) / 4
    assert abs(O.s_lambda(lam, a + q) - math.exp(-4.0 / 3.0)) < 1e-15
    assert abs(O.s_lambda(lam, b - q) - math.exp(-4.0 / 3.0)) < 1e-15
    # symmetric about the centre
    u = (b - a) / 2 * np.linspace(0.01, 0.99, 57)
    assert np.abs(O.s_lambda(lam, c + u) - O.s_lambda(lam, c - u)).max() < 1e-15
    # largest at the centre
    assert O.s_lambda(lam, inside).max() <= math.exp(-1.0) + 1e-16


@pytest.mark.parametrize("lam", LAMS)
def test_k_lambda_ends_and_strictly_decreasing(lam):
    a = 1.0 / lam
    for t in [0.0, a / 2, a - 1e-12, a]:
        assert O.k_lambda(lam, t) == 1.0
    for t in [1.0, 1.0 + 1e-12, 2.0]:
        assert O.k_lambda(lam, t) == 0.0
    t = a + (1 - a) * np.linspace(0.01, 0.99, 199)
    k = O.k_lambda(lam, t)
    # non-increasing everywhere, strictly where 1 - k and k are resolved in double
    assert np.all(np.diff(k) <= 0.0)
    mid = (k > 1e-10) & (k < 1 - 1e-10)
    assert mid.sum() > 150 and np.all(np.diff(k[mid]) < 0.0)
    # k(t_i) - k(t_i+1) as one integral: positive for every step, down to the ends
    h = O.lib()
    gaps = [h.orc_k_diff(lam, float(t[i]), float(t[i + 1])) for i in range(len(t) - 1)]
    assert np.all(np.array(gaps) > 0.0)
    assert np.all((k > 0.0) & (k <= 1.0 + 4e-16))
    # continuous at both ends
    assert O.k_lambda(lam, a + 1e-6 * (1 - a)) > 1 - 1e-12
    assert O.k_lambda(lam, 1 - 1e-6 * (1 - a)) < 1e-12


@pytest.mark.parametrize("lam", LAMS)
def test_k_lambda_derivative_is_s_lambda_squared_over_t(lam):
    """-k'(t) t / s_lambda(t)^2 is one constant over the support (Richardson-extrapolated
    central differences); a weight other than 1/t, or s_lambda not squared, makes it vary."""
    a = 1.0 / lam
    ts = a + (1 - a) * np.linspace(0.15, 0.85, 15)
    ratios = []
    for t in ts:
        def d(h):
            return (O.k_lambda(lam, t - h) - O.k_lambda(lam, t + h)) / (2 * h)
        h = 1e-3 * (1 - a)
        deriv = (4 * d(h / 2) - d(h)) / 3
        ratios.append(deriv * t / O.s_lambda(lam, t) ** 2)
    ratios = np.array(ratios)
    assert np.all(ratios > 0)
    assert (ratios.max() - ratios.min()) / ratios.mean() < 1e-6, ratios


@pytest.mark.parametrize("lam,L", [(2.0, 2048), (1.5, 120), (3.0, 400), (2.7, 300)])
def test_kappa_positive_on_open_support(lam, L):
    l = np.arange(L)
    for j in range(0, O.J_max(lam, L) + 1):
        k = O.kappa(lam, j, L)
        inside = (l > lam ** (j - 1) * (1 + 1e-12)) & (l < lam ** (j + 1) * (1 - 1e-12))
        assert np.all(k[inside] > 0.0), (j, l[inside][k[inside] <= 0.0])
        assert np.all(k[~inside] == 0.0)
