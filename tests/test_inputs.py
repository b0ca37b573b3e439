"""The seeded input generator: determinism, the published splitmix64 values,
real-signal symmetry and the requested spectrum."""
import numpy as np

from paper_1511_05578_gb300 import inputs as I


def test_splitmix64_reference_values():
    # splitmix64 from state 0: the first outputs of the published generator
    z = I.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_deterministic_and_seed_dependent():
    a = I.flm_gaussian(32, 5)
    b = I.flm_gaussian(32, 5)
    c = I.flm_gaussian(32, 6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_real_symmetry_and_spin_zeros():
    L = 40
    f = I.flm_gaussian(L, 1, real=True)
    for l in range(L):
        assert f[l * l + l].imag == 0
        for m in range(1, l + 1):
            assert f[l * l + l - m] == (-1) ** m * np.conj(f[l * l + l + m])
    g = I.flm_gaussian(L, 1, spin=2)
    assert np.all(g[:4] == 0) and np.all(g[4:] != 0)


def test_spectrum():
    L = 400
    f = I.flm_gaussian(L, 9, power=2.0)
    l = np.floor(np.sqrt(np.arange(L * L))).astype(int)
    cl = np.bincount(l, weights=np.abs(f) ** 2) / (2 * np.arange(L) + 1)
    ratio = cl[50:] * (np.arange(50, L) + 1.0) ** 2
    assert abs(ratio.mean() - 1.0) < 0.02
