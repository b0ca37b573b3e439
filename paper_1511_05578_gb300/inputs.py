"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle runs.

This module holds none of the transform's arithmetic: it only draws harmonic
coefficients f_lm with a prescribed angular power spectrum from a counter-based
generator (splitmix64 -> Box-Muller), so the CUDA path and the oracle can be fed
bit-identical inputs.

Workload recipe (the paper's Sec. III-C protocol draws Re/Im uniform in [-1,1];
the default here is the Gaussian spectrum C_l = (l+1)^-p):
  * for l >= |s|: Re f_lm, Im f_lm ~ N(0, C_l / 2) independently;
  * real spin-0 signals: f_l0 real ~ N(0, C_l), f_{l,-m} = (-1)^m conj(f_lm);
  * f_lm = 0 for l < |s|.
Coefficients are stored at index l*l + l + m.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Output of splitmix64 for stream `seed` at the given counters (uint64 array):
    state = seed + (counter + 1) * golden, then the standard finaliser."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian_pairs(seed: int, idx: np.ndarray):
    """Two independent N(0,1) draws per index (Box-Muller on counters 2i, 2i+1)."""
    u1 = uniform01(seed, 2 * idx)
    u2 = uniform01(seed, 2 * idx + 1)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    return r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)


def flm_gaussian(L: int, seed: int, spin: int = 0, real: bool = False, power: float = 2.0,
                 dist: str = "gaussian") -> np.ndarray:
    """Band-limited harmonic coefficients f_lm (complex128, length L*L)."""
    idx = np.arange(L * L, dtype=np.int64)
    l = np.floor(np.sqrt(idx)).astype(np.int64)
    m = idx - l * l - l
    if dist == "gaussian":
        a, b = gaussian_pairs(seed, idx)
        cl = (l + 1.0) ** (-power)
        f = (a + 1j * b) * np.sqrt(cl / 2.0)
    elif dist == "uniform":
        f = (2 * uniform01(seed, 2 * idx) - 1) + 1j * (2 * uniform01(seed, 2 * idx + 1) - 1)
    else:
        raise ValueError(dist)
    f[l < abs(spin)] = 0.0
    if real:
        if spin != 0:
            raise ValueError("real signals are spin 0")
        m0 = m == 0
        f[m0] = f[m0].real * (np.sqrt(2.0) if dist == "gaussian" else 1.0)
        neg = m < 0
        pos_idx = l[neg] * l[neg] + l[neg] - m[neg]
        sign = np.where((m[neg] % 2) == 0, 1.0, -1.0)
        f[neg] = sign * np.conj(f[pos_idx])
    return f


def seed_for(config: int, map_index: int) -> int:
    """Seed of map `map_index` of workload `config` (1000*config + map)."""
    return 1000 * int(config) + int(map_index)
