"""Host logic of bench.py's algorithmic work model (no GPU): the contraction's term count over
the kernel's support, checked against a brute-force count of the (l, m, n, m' >= 0) terms with
a nonzero product, and the support start against the radial kernel of the oracle."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import bench  # noqa: E402
import oracle as O  # noqa: E402


def _brute(Lb, lmin, real, spin):
    n = 0
    for l in range(lmin, Lb):
        for m in range(-l, l + 1):
            if real and m < 0:
                continue
            for k in range(-l, l + 1):
                if spin == 0 and k % 2:
                    continue
                n += l + 1  # m' = 0..l
    return n


@pytest.mark.parametrize("Lb,lmin", [(1, 0), (2, 1), (9, 3), (12, 5), (17, 9), (16, 16)])
@pytest.mark.parametrize("real,spin", [(True, 0), (False, 0), (False, 2)])
def test_contraction_terms_match_brute_force(Lb, lmin, real, spin):
    assert bench.contraction_terms(Lb, lmin, real, spin) == _brute(Lb, lmin, real, spin)


@pytest.mark.parametrize("lam,J0,L", [(2.0, 2, 64), (1.5, 2, 40), (3.0, 1, 60)])
def test_support_start_is_first_nonzero_kappa(lam, J0, L):
    J = O.J_max(lam, L)
    for j in range(J0, J + 1):
        k = O.kappa(lam, j, L)
        nz = np.nonzero(k > 0)[0]
        first = int(nz[0]) if len(nz) else L
        assert min(bench.support_start(lam, j), L) == first, (lam, j)


def test_top_scales_at_the_benchmark_size():
    # L = 1024, lambda = 2: scale 10 from l = 513, scale 9 from 257 (kappa^(j) > 0 iff
    # 2^(j-1) < l < 2^(j+1)); the support cuts the top scale's terms by about (513/1024)^4
    assert bench.support_start(2.0, 10) == 513 and bench.support_start(2.0, 9) == 257
    full, sup = bench.contraction_terms(1024, 0), bench.contraction_terms(1024, 513)
    assert 0.92 < sup / full < 0.95
