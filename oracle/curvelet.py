"""numpy layer of the FP64 oracle: grids, spin SHT, curvelet kernels, analysis and
synthesis, in the order and notation of arXiv:1511.05578 Sec. II-III.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). numpy.fft serves as the library
DFT step; everything else is written out from the paper. Arrays over an azimuthal
index m (or n, m') are kept in centred order, position m + L - 1 for |m| < L;
harmonic coefficients f_lm sit at l*l + l + m.
"""
import ctypes
import math

import numpy as np

from . import build as _build

__all__ = [
    "lib", "mw_theta", "mw_phi", "half_angles", "wigner_d_factsum", "wigner_d_lrec",
    "risbo_matrix", "delta_matrix", "quad_weight", "sht_inverse", "sht_forward",
    "s_lambda", "k_lambda", "J_max", "band_limit", "L_phi", "kappa", "phi_scaling", "zeta", "zeta_unrotated", "psi",
    "euler_matrix", "euler_angles", "analysis_point", "analysis_rings", "analysis_from_flm", "analysis", "scaling_map", "wigner_forward_Y",
    "wigner_forward_coeffs", "synthesis_flm", "synthesis", "rotate_wigner", "rotate_wigner_adjoint", "MUTATION",
]

# Deliberate-mistake switches, used only by tests that check the pins catch them.
MUTATION = {"ext_sign": False, "half_phase": False, "weight_sign": False, "rotation_transposed": False}

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        h = ctypes.CDLL(_build.build())
        h.orc_d_factsum.restype = ctypes.c_double
        h.orc_d_factsum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        h.orc_d_lrec.restype = None
        h.orc_d_lrec.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        h.orc_risbo_matrix.restype = None
        h.orc_risbo_matrix.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        h.orc_sht_fwd_contract.restype = None
        h.orc_sht_fwd_contract.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
        h.orc_wigner_fwd_contract.restype = None
        h.orc_wigner_fwd_contract.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
        h.orc_analysis_ring.restype = None
        h.orc_analysis_ring.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
        h.orc_analysis_ring_lrec.restype = None
        h.orc_analysis_ring_lrec.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
        h.orc_sht_inv_rings.restype = None
        h.orc_sht_inv_rings.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp]
        h.orc_d_edge.restype = ctypes.c_double
        h.orc_d_edge.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        h.orc_d_edge_row.restype = None
        h.orc_d_edge_row.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        h.orc_k_diff.restype = ctypes.c_double
        h.orc_k_diff.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        h.orc_k_lambda.restype = ctypes.c_double
        h.orc_k_lambda.argtypes = [ctypes.c_double, ctypes.c_double]
        h.orc_s_lambda.restype = ctypes.c_double
        h.orc_s_lambda.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib = h
    return _lib


def _p(a):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


# --------------------------------------------------------------------------
# Sampling (Sec. III-A-2, Eqs. nodes_alpha, nodes_beta, nodes_gamma; the MW
# sphere grid uses the same colatitude rule)
# --------------------------------------------------------------------------
def mw_theta(L):
    return np.pi * (2 * np.arange(L) + 1) / (2 * L - 1)


def mw_phi(L):
    return 2 * np.pi * np.arange(2 * L - 1) / (2 * L - 1)


def half_angles(L, idx):
    """(sin, cos) of beta_b / 2 for beta_b = pi (2b+1)/(2L-1); exact at b = L-1 (beta = pi)."""
    b = np.asarray(idx, dtype=np.float64)
    sh = np.sin(np.pi * (2 * b + 1) / (2 * (2 * L - 1)))
    ch = np.sin(np.pi * (L - 1 - b) / (2 * L - 1))
    return sh, ch


# --------------------------------------------------------------------------
# Wigner functions (Sec. II-A)
# --------------------------------------------------------------------------
def wigner_d_factsum(l, m, n, beta):
    """d^l_mn(beta) by the explicit factorial sum, Eq. (wigner_sum_reln). Small l only."""
    return lib().orc_d_factsum(int(l), int(m), int(n), float(beta))


def wigner_d_lrec(L, m, n, beta=None, sh=None, ch=None):
    """d^l_mn(beta) for l = 0..L-1 by the three-term l-recurrence (see orc.c)."""
    if sh is None:
        sh, ch = math.sin(beta / 2), math.cos(beta / 2)
    out = np.zeros(L)
    lib().orc_d_lrec(int(L), int(m), int(n), float(sh), float(ch), _p(out))
    return out


def risbo_matrix(l, beta=None, sh=None, ch=None):
    """Full d^l(beta) matrix [m+l, n+l] by Risbo's half-integer recursion."""
    if sh is None:
        sh, ch = math.sin(beta / 2), math.cos(beta / 2)
    out = np.zeros((2 * l + 1, 2 * l + 1))
    lib().orc_risbo_matrix(int(l), float(sh), float(ch), _p(out))
    return out


def delta_matrix(l):
    """Delta^l_mn = d^l_mn(pi/2) (Sec. III-A-2, after Eq. flml) as [m+l, n+l]."""
    s = math.sqrt(0.5)
    return risbo_matrix(l, sh=s, ch=s)


def quad_weight(p):
    """w(p) = int_0^pi sin(b) e^{i p b} db (Eq. gmnmp), evaluated in closed form."""
    p = np.asarray(p)
    w = np.zeros(p.shape, dtype=np.complex128)
    even = (p % 2) == 0
    w[even] = 2.0 / (1.0 - p[even].astype(np.float64) ** 2)
    w[p == 1] = 0.5j * np.pi
    w[p == -1] = -0.5j * np.pi
    if MUTATION["weight_sign"]:
        w[even & (p != 0)] *= -1.0
    return w


def _weight_matrix(L):
    """Wmat[m'' + L-1, m' + L-1] = w(m'' - m') for |m''|, |m'| < L."""
    idx = np.arange(-(L - 1), L)
    return quad_weight(idx[:, None] - idx[None, :])


def _ext_sign(k):
    s = np.where(np.asarray(k) % 2 == 0, 1.0, -1.0)
    return -s if MUTATION["ext_sign"] else s


# --------------------------------------------------------------------------
# Spin spherical harmonic transform on the MW grid
# --------------------------------------------------------------------------
def sht_inverse(flm, L, s):
    """f(theta_t, phi_p) = sum_lm f_lm sY_lm(theta_t, phi_p), with sY_lm from
    Eq. (spin_sphericalHarmonics) summed directly (d^l_{m,-s} by l-recurrence).
    Returns the complex map [L][2L-1]."""
    N = 2 * L - 1
    flm = np.ascontiguousarray(flm[: L * L], dtype=np.complex128)
    sh, ch = half_angles(L, np.arange(L))
    g = np.zeros((L, N), dtype=np.complex128)
    lib().orc_sht_inv_rings(L, int(s), _p(flm.view(np.float64)), L, _p(sh), _p(ch), _p(g.view(np.float64)))
    # sum over m of g_m e^{i m phi_p}: an inverse DFT of length 2L-1
    return N * np.fft.ifft(np.fft.ifftshift(g, axes=1), axis=1)


def _theta_quadrature(Fm, L, sgn_idx):
    """Shared steps of the exact quadrature over colatitude (Eqs. TildaFmn, Fmnmp,
    gmnmp): given F[t, ...] on t < L, extend to t in [L, 2L-2] with sign
    (-1)^{sgn_idx}, take the DFT over the 2L-1 samples (half-sample phase of
    beta_b), and apply the weights w. Returns G[..., m'] centred over m'."""
    N = 2 * L - 1
    Fbar = np.empty((N,) + Fm.shape[1:], dtype=np.complex128)
    Fbar[:L] = Fm
    Fbar[L:] = _ext_sign(sgn_idx) * Fm[L - 2::-1] if L > 1 else Fm[:0]
    Fk = np.fft.fftshift(np.fft.fft(Fbar, axis=0), axes=0) / N  # over m'' centred
    mpp = np.arange(-(L - 1), L)
    if not MUTATION["half_phase"]:
        Fk = Fk * np.exp(-1j * np.pi * mpp / N).reshape((N,) + (1,) * (Fk.ndim - 1))
    Fk = np.moveaxis(Fk, 0, -1)  # [..., m'']
    return Fk @ _weight_matrix(L)  # sum_{m''} F_{m''} w(m'' - m')


def sht_forward(fmap, L, s):
    """f_lm of a band-limited spin-s map on the MW grid by the exact quadrature:
    DFT over phi, extension over theta with (-1)^{m+s}, DFT over theta, weights,
    then Eq. (flml)-like Delta contraction with n = -s (orc_sht_fwd_contract)."""
    N = 2 * L - 1
    fmap = np.asarray(fmap, dtype=np.complex128).reshape(L, N)
    F = np.fft.fftshift(np.fft.fft(fmap, axis=1), axes=1) / N  # F[t, m]
    m = np.arange(-(L - 1), L)
    G = 2 * np.pi * _theta_quadrature(F, L, (m + s)[None, :])  # [m, m']
    G = np.ascontiguousarray(G)
    flm = np.zeros(L * L, dtype=np.complex128)
    lib().orc_sht_fwd_contract(L, int(s), _p(G.view(np.float64)), _p(flm.view(np.float64)))
    return flm


# --------------------------------------------------------------------------
# Curvelet construction (Sec. II-B)
# --------------------------------------------------------------------------
def s_lambda(lam, t):
    """s_lambda(t) = s(2 lam/(lam-1) (t - 1/lam) - 1) with s(t) = exp(-1/(1-t^2)) on
    (-1, 1) and 0 elsewhere (Sec. II-B): the bump whose square, weighted by 1/t,
    k_lambda integrates."""
    h = lib()
    t = np.asarray(t, dtype=np.float64)
    return np.vectorize(lambda x: h.orc_s_lambda(float(lam), float(x)), otypes=[np.float64])(t)


def k_lambda(lam, t):
    """k_lambda(t) (Sec. II-B): normalised integral of s_lambda^2(t')/t' from t to 1."""
    h = lib()
    t = np.asarray(t, dtype=np.float64)
    return np.vectorize(lambda x: h.orc_k_lambda(float(lam), float(x)), otypes=[np.float64])(t)


def J_max(lam, L):
    """Largest analysis scale: the smallest J with lam^J >= L (reading: the paper
    leaves J open; this J makes the admissibility sum telescope to 1 for all l < L)."""
    J = 0
    while lam ** J < L * (1 - 1e-14):
        J += 1
    return J


def _ceil_pow(lam, e):
    v = lam ** e
    r = round(v)
    return int(r) if abs(v - r) < 1e-9 * max(1.0, v) else int(math.ceil(v))


def band_limit(lam, j, L):
    """Band limit L_j = min(L, ceil(lam^(j+1))) of scale j (Sec. III-A-3)."""
    return min(L, _ceil_pow(lam, j + 1))


def L_phi(lam, J0, L=None):
    """Band limit of the scaling map: ceil(lam^J0), capped at the signal's band limit
    L (Phi_l0 is only needed for l < L)."""
    v = max(1, _ceil_pow(lam, J0))
    return v if L is None else min(v, L)


def kappa(lam, j, L):
    """kappa^(j)(l) = kappa_lambda(lam^-j l) = sqrt(k(l/lam^(j+1)) - k(l/lam^j)), l < L.
    The difference is evaluated as one integral over the gap between the two
    arguments (same quantity; avoids cancellation next to the support ends)."""
    h = lib()
    out = np.zeros(L)
    for l in range(L):
        out[l] = math.sqrt(max(h.orc_k_diff(float(lam), l / lam ** (j + 1), l / lam ** j), 0.0))
    return out


def phi_scaling(lam, J0, L):
    """sqrt(4pi/(2l+1)) Phi_l0 = sqrt(k_lambda(lam^-J0 l)) (scaling function, Sec. II-B)."""
    l = np.arange(L, dtype=np.float64)
    return np.sqrt(k_lambda(lam, l / lam ** J0))


def zeta(lam, j, s, Lj):
    """Directional component rotated to the North pole, zeta_lk = sum_n
    d^l_kn(vartheta^j) zeta~_ln with zeta~_{l,l} = 1/sqrt2, zeta~_{l,-l} = (-1)^l/sqrt2
    (reading delta_{l|m|} in the printed definition), vartheta^j = arccos(-s/lam^j).
    Zero for l < |s|. Returns [Lj][2Lj-1] (real)."""
    N = 2 * Lj - 1
    th = math.acos(-s / lam ** j)
    sh, ch = math.sin(th / 2), math.cos(th / 2)
    out = np.zeros((Lj, N))
    for l in range(abs(s), Lj):
        if l == 0:
            out[0, Lj - 1] = lib().orc_d_edge(0, 0, sh, ch) / math.sqrt(2)
            continue
        dp = np.zeros(2 * l + 1)
        dm = np.zeros(2 * l + 1)
        lib().orc_d_edge_row(l, 1, sh, ch, _p(dp))   # d^l_{k,l}(vartheta)
        lib().orc_d_edge_row(l, -1, sh, ch, _p(dm))  # d^l_{k,-l}(vartheta)
        out[l, Lj - 1 - l: Lj + l] = (dp + (-1) ** l * dm) / math.sqrt(2)
    return out


def zeta_unrotated(s, Lj):
    """Directional component of the unrotated curvelets s-psi~ (Sec. II-B, printed
    definition read with delta_{l|m|}): zeta~_{l,l} = 1/sqrt2, zeta~_{l,-l} =
    (-1)^l/sqrt2, zeta~_00 = 1/sqrt2; zero for l < |s|. Returns [Lj][2Lj-1] (real)."""
    out = np.zeros((Lj, 2 * Lj - 1))
    for l in range(abs(s), Lj):
        out[l, Lj - 1 + l] = 1.0 / math.sqrt(2)
        if l > 0:
            out[l, Lj - 1 - l] = (-1) ** l / math.sqrt(2)
    return out


def psi(lam, j, s, Lj, unrotated=False):
    """Curvelet harmonic coefficients sPsi^(j)_ln = sqrt((2l+1)/8pi^2) kappa^(j)(l) zeta_ln
    (Eq. wav_factorized), [Lj][2Lj-1], real; with unrotated=True those of s-psi~^(j),
    with zeta~ in place of zeta (nonzero for |n| = l only)."""
    l = np.arange(Lj, dtype=np.float64)
    fac = np.sqrt((2 * l + 1) / (8 * np.pi ** 2)) * kappa(lam, j, Lj)
    z = zeta_unrotated(s, Lj) if unrotated else zeta(lam, j, s, Lj)
    return np.ascontiguousarray(fac[:, None] * z)


def euler_matrix(alpha, beta, gamma):
    """Rotation R(alpha, beta, gamma) = R_z(alpha) R_y(beta) R_z(gamma) of R^3, the
    rotation whose Wigner matrix is D^l_mn = e^{-i m alpha} d^l_mn(beta) e^{-i n gamma}."""
    def rz(t):
        c, s_ = math.cos(t), math.sin(t)
        return np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])

    def ry(t):
        c, s_ = math.cos(t), math.sin(t)
        return np.array([[c, 0.0, s_], [0.0, 1.0, 0.0], [-s_, 0.0, c]])
    return rz(alpha) @ ry(beta) @ rz(gamma)


def euler_angles(R):
    """(alpha, beta, gamma) of a rotation matrix in the convention of euler_matrix
    (beta in [0, pi]; generic rotations, sin beta != 0)."""
    beta = math.acos(max(-1.0, min(1.0, R[2, 2])))
    alpha = math.atan2(R[1, 2], R[0, 2])
    gamma = math.atan2(R[2, 1], -R[2, 0])
    return alpha, beta, gamma


def analysis_point(flm, psi_j, Lj, alpha, beta, gamma):
    """W(rho) at one arbitrary rotation rho = (alpha, beta, gamma) by the direct sum of
    Eq. (wav_analysis_harmonic), D^{l*}_mn = e^{i m alpha} d^l_mn(beta) e^{i n gamma},
    d from the factorial sum. Tiny Lj only."""
    acc = 0j
    for l in range(Lj):
        for m in range(-l, l + 1):
            for n in range(-l, l + 1):
                c = flm[l * l + l + m] * psi_j[l, n + Lj - 1]
                if c != 0:
                    acc += c * wigner_d_factsum(l, m, n, beta) * np.exp(1j * (m * alpha + n * gamma))
    return acc


# --------------------------------------------------------------------------
# Curvelet analysis (Sec. II-D-1)
# --------------------------------------------------------------------------
def analysis_rings(flm, lam, j, s, L, rings=None, psi_j=None, method="risbo", unrotated=False):
    """W^(j)(alpha_a, beta_b, gamma_g) at the requested rings b, by direct evaluation
    of Eq. (wav_analysis_harmonic) with D^{l*}_mn = e^{i m a} d^l_mn(b) e^{i n g};
    d^l(beta_b) by Risbo's recursion at beta_b (method="risbo") or by the
    l-recurrence ("lrec"). unrotated=True: W~ of the unrotated curvelets.
    Returns complex [len(rings)][2Lj-1 (a)][2Lj-1 (g)]."""
    Lj = band_limit(lam, j, L)
    N = 2 * Lj - 1
    if rings is None:
        rings = range(Lj)
    rings = list(rings)
    ps = psi(lam, j, s, Lj, unrotated) if psi_j is None else psi_j
    f = np.ascontiguousarray(np.asarray(flm, dtype=np.complex128)[: Lj * Lj])
    out = np.empty((len(rings), N, N), dtype=np.complex128)
    X = np.empty((N, N), dtype=np.complex128)
    for i, b in enumerate(rings):
        sh, ch = half_angles(Lj, b)
        fn = lib().orc_analysis_ring if method == "risbo" else lib().orc_analysis_ring_lrec
        fn(Lj, _p(f.view(np.float64)), _p(ps), float(sh), float(ch), _p(X.view(np.float64)))
        # sum_m sum_n X_mn e^{i m alpha_a} e^{i n gamma_g}
        out[i] = N * N * np.fft.ifft2(np.fft.ifftshift(X))
    return out


def scaling_map(flm, lam, J0, L):
    """Scaling coefficients W^Phi on the MW grid of band limit ceil(lam^J0): inverse
    spin-0 SHT of sqrt(4pi/(2l+1)) f_lm Phi*_l0 (Eq. swav_harmonic_coeff)."""
    Lp = L_phi(lam, J0, L)
    ph = phi_scaling(lam, J0, Lp)
    c = np.zeros(Lp * Lp, dtype=np.complex128)
    for l in range(min(Lp, L)):
        c[l * l: (l + 1) * (l + 1)] = ph[l] * flm[l * l: (l + 1) * (l + 1)]
    return sht_inverse(c, Lp, 0)


def analysis_from_flm(flm, lam, J0, s, L, rings=None, unrotated=False):
    J = J_max(lam, L)
    W = {}
    for j in range(J0, J + 1):
        W[j] = analysis_rings(flm, lam, j, s, L, None if rings is None else rings.get(j, None), unrotated=unrotated)
    return W, scaling_map(flm, lam, J0, L)


def analysis(fmap, lam, J0, s, L, rings=None, unrotated=False):
    """Curvelet analysis of a map: (f_lm, {W_j}, W^Phi); unrotated=True gives the W~_j of
    the unrotated curvelets (the scaling map is the same)."""
    flm = sht_forward(fmap, L, s)
    W, Wphi = analysis_from_flm(flm, lam, J0, s, L, rings, unrotated)
    return flm, W, Wphi


# --------------------------------------------------------------------------
# Curvelet synthesis (Sec. II-D-2) through the forward Wigner quadrature (Sec. III-A-2)
# --------------------------------------------------------------------------
def wigner_forward_Y(Wj, Lj):
    """Eqs. (Fmn), (TildaFmn), (Fmnmp), (gmnmp): from W on the SO(3) grid
    [b][a][g] to Y_{m n m'} (returned as [m][n][m'], centred)."""
    N = 2 * Lj - 1
    Wj = np.asarray(Wj).reshape(Lj, N, N)
    X = np.fft.fftshift(np.fft.fft2(Wj, axes=(1, 2)), axes=(1, 2)) / (N * N)  # [b][m][n]
    m = np.arange(-(Lj - 1), Lj)
    Y = (2 * np.pi) ** 2 * _theta_quadrature(X, Lj, (m[:, None] + m[None, :])[None, :, :])  # [m][n][m']
    return np.ascontiguousarray(Y)


def wigner_forward_coeffs(Wj, Lj):
    """Wigner coefficients (W)^l_mn of W on the grid, dense [l][m][n] (Eq. flml in
    general-n form)."""
    N = 2 * Lj - 1
    Y = wigner_forward_Y(Wj, Lj)
    wl = np.zeros((Lj, N, N), dtype=np.complex128)
    f = np.zeros(Lj * Lj, dtype=np.complex128)
    zero_psi = np.zeros((Lj, N))
    lib().orc_wigner_fwd_contract(Lj, _p(Y.view(np.float64)), _p(zero_psi), _p(f.view(np.float64)), _p(wl.view(np.float64)))
    return wl


def synthesis_flm(W, Wphi, lam, J0, s, L, scales=None, unrotated=False):
    """f_lm from curvelet and scaling coefficients, Eq. (wav_synthesis_harmonic).
    W maps scale j -> [Lj][2Lj-1][2Lj-1]; scales missing from W contribute nothing.
    unrotated=True: W holds the W~_j of the unrotated curvelets."""
    J = J_max(lam, L)
    f = np.zeros(L * L, dtype=np.complex128)
    for j in range(J0, J + 1):
        if j not in W or (scales is not None and j not in scales):
            continue
        Lj = band_limit(lam, j, L)
        Y = wigner_forward_Y(W[j], Lj)
        ps = psi(lam, j, s, Lj, unrotated)
        part = np.zeros(Lj * Lj, dtype=np.complex128)
        lib().orc_wigner_fwd_contract(Lj, _p(Y.view(np.float64)), _p(ps), _p(part.view(np.float64)), None)
        f[: Lj * Lj] += part
    if Wphi is not None:
        Lp = L_phi(lam, J0, L)
        c = sht_forward(Wphi, Lp, 0)
        ph = phi_scaling(lam, J0, Lp)
        for l in range(min(Lp, L)):
            f[l * l: (l + 1) * (l + 1)] += ph[l] * c[l * l: (l + 1) * (l + 1)]
    f[: s * s] = 0.0
    return f


def synthesis(W, Wphi, lam, J0, s, L, unrotated=False):
    """Curvelet synthesis back to the MW map (complex [L][2L-1])."""
    return sht_inverse(synthesis_flm(W, Wphi, lam, J0, s, L, unrotated=unrotated), L, s)


# --------------------------------------------------------------------------
# Rotation of Wigner coefficients (Sec. III-A-1, Eqs. curvelet_Wigner,
# curvelet_Wigner_inverse and rotateWigner)
# --------------------------------------------------------------------------
def _edge_d(l, th):
    """Columns n = +l and n = -l of d^l(vartheta) as arrays over k = -l..l (Risbo)."""
    d = risbo_matrix(l, th)
    if MUTATION["rotation_transposed"]:
        d = d.T
    return d[:, 2 * l], d[:, 0]


def rotate_wigner(wt, lam, j, s, Lj):
    """Wigner coefficients of the rotated curvelet coefficients from those of the unrotated
    ones. W(rho) = W~(rho rho*) with rho* = (0, vartheta^j, 0) (Eq. rotateWigner) and
    D^l(rho rho*) = D^l(rho) D^l(rho*) give (W)^l_mk = sum_n (W~)^l_mn d^l_kn(vartheta^j),
    and (W~)^l_mn vanishes unless |n| = l (Eq. curvelet_Wigner_property), so two terms:
        (W)^l_mk = (W~)^l_{m,l} d^l_{k,l}(vartheta) + (W~)^l_{m,-l} d^l_{k,-l}(vartheta).
    wt: [2][Lj][2Lj-1] complex, wt[0][l][m + Lj - 1] = (W~)^l_{m,l}, wt[1][...] = (W~)^l_{m,-l}
    (wt[1][0] unused: at l = 0 the two coincide). Returns dense [Lj][2Lj-1][2Lj-1] (m, k)."""
    N = 2 * Lj - 1
    th = math.acos(-s / lam ** j)
    out = np.zeros((Lj, N, N), dtype=np.complex128)
    for l in range(Lj):
        dp, dm = _edge_d(l, th)
        ms = slice(Lj - 1 - l, Lj + l)
        a = wt[0][l, ms]
        out[l, ms, ms] = a[:, None] * dp[None, :]
        if l > 0:
            out[l, ms, ms] += wt[1][l, ms][:, None] * dm[None, :]
    return out


def rotate_wigner_adjoint(w, lam, j, s, Lj):
    """Adjoint of rotate_wigner: (W~)^l_{m,+-l} = sum_k (W)^l_mk d^l_{k,+-l}(vartheta^j); the
    inverse on coefficients of the form rotate_wigner(wt) (d^l is orthogonal). Returns
    [2][Lj][2Lj-1] as rotate_wigner takes it (wt[1][0] = 0)."""
    N = 2 * Lj - 1
    th = math.acos(-s / lam ** j)
    wt = np.zeros((2, Lj, N), dtype=np.complex128)
    for l in range(Lj):
        dp, dm = _edge_d(l, th)
        ms = slice(Lj - 1 - l, Lj + l)
        blk = w[l, ms, ms]
        wt[0][l, ms] = blk @ dp
        if l > 0:
            wt[1][l, ms] = blk @ dm
    return wt
