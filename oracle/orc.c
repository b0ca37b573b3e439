/*
 * Plain FP64 CPU oracle for the second-generation spherical curvelet transform
 * (Chan, Leistedt, Kitching, McEwen, arXiv:1511.05578).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do. It shares no code, table or helper with the CUDA path.
 *
 * This file holds the inner loops that are too slow in numpy: Wigner small-d
 * functions (two independent methods), the Delta = d(pi/2) matrices by Risbo's
 * half-integer recursion, the O(L^4) sums of the curvelet analysis (Eq.
 * wav_analysis_harmonic, evaluated directly), and the Delta contractions of the
 * forward Wigner and spin-SHT quadratures (Eq. flml). The numpy layer in
 * oracle/curvelet.py chains these in the paper's order.
 *
 * Complex arrays are interleaved (re, im) doubles, as numpy complex128.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double _Complex cplx;

/* ------------------------------------------------------------------------ */
/* Eq. (wigner_sum_reln): explicit factorial sum for d^l_{mn}(beta).          */
/* Long double; only meant for small l (it cancels catastrophically).         */
/* ------------------------------------------------------------------------ */
static long double factl(int k) {
  long double r = 1.0L;
  for (int i = 2; i <= k; ++i) r *= (long double)i;
  return r;
}

double orc_d_factsum(int l, int m, int n, double beta) {
  if (l < 0 || abs(m) > l || abs(n) > l) return 0.0;
  long double sh = sinl((long double)beta / 2), ch = cosl((long double)beta / 2);
  long double pre = sqrtl(factl(l + m) * factl(l - m) * factl(l + n) * factl(l - n));
  long double sum = 0.0L;
  for (int k = 0; k <= 2 * l; ++k) {
    if (l - m - k < 0 || l - n - k < 0 || m + n + k < 0) continue;
    int ps = 2 * l - m - n - 2 * k, pc = m + n + 2 * k;
    long double t = (ps ? powl(sh, ps) : 1.0L) * (pc ? powl(ch, pc) : 1.0L) /
                    (factl(k) * factl(l - m - k) * factl(l - n - k) * factl(m + n + k));
    sum += (k & 1) ? -t : t;
  }
  long double sgn = ((l - n) & 1) ? -1.0L : 1.0L;
  return (double)(sgn * pre * sum);
}

/* ------------------------------------------------------------------------ */
/* Exponent-extended doubles: value = v * 2^e. Used so that seeds of size     */
/* 2^-2000 (near the poles, at large l) neither underflow nor lose bits.      */
/* ------------------------------------------------------------------------ */
typedef struct { double v; long e; } xnum;

static xnum xn_norm(xnum x) {
  if (x.v == 0.0) { x.e = 0; return x; }
  int k; x.v = frexp(x.v, &k); x.e += k; return x;
}
static xnum xn_mul_d(xnum x, double d) { x.v *= d; return xn_norm(x); }
static xnum xn_pow(double b, long p) { /* b > 0 */
  xnum r = {1.0, 0}, base = xn_norm((xnum){b, 0});
  while (p > 0) {
    if (p & 1) { r.v *= base.v; r.e += base.e; r = xn_norm(r); }
    base.v *= base.v; base.e *= 2; base = xn_norm(base);
    p >>= 1;
  }
  return r;
}

/* A(l0,k) = sqrt(C(2 l0, l0+k)) sh^(l0-k) ch^(l0+k), for |k| <= l0, by the
 * exact ratio A(l0,k+1)/A(l0,k) = sqrt((l0-k)/(l0+k+1)) ch/sh. This is
 * d^{l0}_{k,l0}(beta) read off Eq. (wigner_sum_reln) (only the k=0 term of the
 * sum survives when n = l). */
static xnum seed_A(int l0, int k, double sh, double ch) {
  xnum x;
  if (sh == 0.0) { x.v = (k == l0) ? 1.0 : 0.0; x.e = 0; if (k == l0) x = xn_pow(ch, 2L * l0); return x; }
  if (ch == 0.0) { x.v = (k == -l0) ? 1.0 : 0.0; x.e = 0; if (k == -l0) x = xn_pow(sh, 2L * l0); return x; }
  x = xn_pow(sh, 2L * l0);
  double r = ch / sh;
  for (int i = -l0; i < k; ++i) x = xn_mul_d(x, sqrt((double)(l0 - i) / (double)(l0 + i + 1)) * r);
  return x;
}

/* ------------------------------------------------------------------------ */
/* d^l_{mn}(beta) for l = 0..L-1 at fixed (m, n, beta) by the three-term     */
/* recurrence in l (Jacobi-polynomial form):                                  */
/*   l sqrt((l+1)^2-m^2) sqrt((l+1)^2-n^2) d^{l+1}                            */
/*     = (2l+1) (l(l+1) cos b - m n) d^l - (l+1) sqrt(l^2-m^2) sqrt(l^2-n^2) d^{l-1}  */
/* seeded at l0 = max(|m|,|n|) with the closed forms read off Eq.              */
/* (wigner_sum_reln). The beta argument is given as sh = sin(b/2), ch =        */
/* cos(b/2) so that grid points such as b = pi are exact.                     */
/* ------------------------------------------------------------------------ */
/* Seed choice for (m, n): d^{l0}_{mn} with l0 = max(|m|,|n|) equals
 * sign * A(l0, kseed). */
static void seed_index(int m, int n, int* l0, int* kseed, double* sgn) {
  int am = abs(m), an = abs(n);
  *l0 = am > an ? am : an; *sgn = 1.0;
  if (am >= an) {
    if (m >= 0) { *kseed = n; if ((*l0 - n) & 1) *sgn = -1.0; } /* d^l_{l,n} */
    else { *kseed = -n; }                                       /* d^l_{-l,n} */
  } else {
    if (n >= 0) { *kseed = m; }                                 /* d^l_{m,l} */
    else { *kseed = -m; if ((*l0 - m) & 1) *sgn = -1.0; }      /* d^l_{m,-l} */
  }
}

/* sq[l*(L+1)+k] = sqrt(l^2 - k^2), 0 <= k <= l <= L. */
static double* sqrt_table(int L) {
  double* sq = (double*)malloc(sizeof(double) * (size_t)(L + 1) * (L + 1));
  for (int l = 0; l <= L; ++l)
    for (int k = 0; k <= L; ++k) sq[(size_t)l * (L + 1) + k] = (k <= l) ? sqrt((double)l * l - (double)k * k) : 0.0;
  return sq;
}

/* The recurrence itself, from a given seed. */
static void d_lrec_core(int L, int m, int n, double cb, xnum seed, double sgn, const double* sq, double* out) {
  int am = abs(m), an = abs(n);
  int l0 = am > an ? am : an;
  for (int l = 0; l < L; ++l) out[l] = 0.0;
  if (l0 >= L || seed.v == 0.0) return;
  double v_prev = 0.0, v = sgn * seed.v;
  long e = seed.e;
  out[l0] = (e < -100000) ? 0.0 : ldexp(v, (int)e);
  const size_t W = (size_t)L + 1;
  for (int l = l0; l + 1 < L; ++l) {
    double vn;
    if (l == 0) {
      vn = cb * v; /* d^1_00 = cos(beta) d^0_00 */
    } else {
      double dl = (double)l;
      double a = (2 * dl + 1) * (dl * (dl + 1) * cb - (double)m * n);
      double b = (dl + 1) * sq[l * W + am] * sq[l * W + an];
      double c = dl * sq[(l + 1) * W + am] * sq[(l + 1) * W + an];
      vn = (a * v - b * v_prev) / c;
    }
    v_prev = v; v = vn;
    if (fabs(v) > 0x1p400) { v = ldexp(v, -400); v_prev = ldexp(v_prev, -400); e += 400; }
    out[l + 1] = (e < -100000) ? 0.0 : ldexp(v, (int)e);
  }
}

void orc_d_lrec(int L, int m, int n, double sh, double ch, double* out) {
  int l0, ks; double sgn;
  seed_index(m, n, &l0, &ks, &sgn);
  for (int l = 0; l < L; ++l) out[l] = 0.0;
  if (l0 >= L) return;
  double* sq = sqrt_table(L);
  d_lrec_core(L, m, n, ch * ch - sh * sh, seed_A(l0, ks, sh, ch), sgn, sq, out);
  free(sq);
}

/* d^{l0}_{mn}(beta) at l0 = max(|m|,|n|) (the closed-form edge values read off
 * Eq. wigner_sum_reln); used for the rotated directional component. */
double orc_d_edge(int m, int n, double sh, double ch) {
  int l0, ks; double sgn;
  seed_index(m, n, &l0, &ks, &sgn);
  xnum x = seed_A(l0, ks, sh, ch);
  if (x.v == 0.0 || x.e < -100000) return 0.0;
  return sgn * ldexp(x.v, (int)x.e);
}

/* Row version: out[k + l] = d^l_{k, n}(beta) for n = +l or -l (nsign = +1/-1),
 * k = -l..l, by the same closed form (A(l,k) with the ratio recursion). */
void orc_d_edge_row(int l, int nsign, double sh, double ch, double* out) {
  for (int k = -l; k <= l; ++k) out[k + l] = 0.0;
  if (sh == 0.0 || ch == 0.0) {
    for (int k = -l; k <= l; ++k) out[k + l] = orc_d_edge(k, nsign * l, sh, ch);
    return;
  }
  xnum x = xn_pow(sh, 2L * l);
  double r = ch / sh;
  for (int k = -l; k <= l; ++k) {
    /* x = A(l, k) = d^l_{k,l}; d^l_{k,-l} = (-1)^{l-k} A(l, -k) */
    double v = (x.e < -100000) ? 0.0 : ldexp(x.v, (int)x.e);
    if (nsign > 0) out[k + l] = v;
    else out[-k + l] = (((l + k) & 1) ? -1.0 : 1.0) * v;
    x = xn_mul_d(x, sqrt((double)(l - k) / (double)(l + k + 1)) * r);
  }
}

/* All seeds A(l0, k) for l0 < L at one beta: tab[l0*l0 + l0 + k]. */
static xnum* seed_table(int L, double sh, double ch) {
  xnum* t = (xnum*)malloc(sizeof(xnum) * (size_t)L * L);
  for (int l0 = 0; l0 < L; ++l0) {
    xnum x;
    if (sh == 0.0 || ch == 0.0) {
      for (int k = -l0; k <= l0; ++k) t[l0 * l0 + l0 + k] = seed_A(l0, k, sh, ch);
      continue;
    }
    x = xn_pow(sh, 2L * l0);
    double r = ch / sh;
    for (int k = -l0; k <= l0; ++k) {
      t[l0 * l0 + l0 + k] = x;
      x = xn_mul_d(x, sqrt((double)(l0 - k) / (double)(l0 + k + 1)) * r);
    }
  }
  return t;
}

/* ------------------------------------------------------------------------ */
/* Risbo's recursion for the full matrix d^j(beta), in half-integer steps j -> */
/* j+1/2, derived from the two-spinor (Schwinger) form of the rotation         */
/* operator: |j m'> = [sqrt(j+m') a+ |j-1/2,m'-1/2> + sqrt(j-m') b+ |j-1/2,m'+1/2>]/(2j), */
/* U a+ U^-1 = c a+ + s b+, U b+ U^-1 = -s a+ + c b+, so                       */
/*   2j d^j_{m,m'} = sqrt(j+m') [c sqrt(j+m) d_{m-1/2,m'-1/2} + s sqrt(j-m) d_{m+1/2,m'-1/2}] */
/*                 + sqrt(j-m') [-s sqrt(j+m) d_{m-1/2,m'+1/2} + c sqrt(j-m) d_{m+1/2,m'+1/2}] */
/* (d = d^{j-1/2}), with c = cos(beta/2), s = sin(beta/2). No small divisors.  */
/* Matrix index i = j - m, k = j - m'. A different method from the product's  */
/* Delta recursion.                                                             */
/* ------------------------------------------------------------------------ */
typedef struct { int J2, cap; double *cur, *tmp; double s, c; } risbo_t;

static void risbo_init(risbo_t* R, int lmax, double sh, double ch) {
  R->cap = 2 * lmax + 1;
  R->cur = (double*)calloc((size_t)R->cap * R->cap, sizeof(double));
  R->tmp = (double*)calloc((size_t)R->cap * R->cap, sizeof(double));
  R->J2 = 0; R->s = sh; R->c = ch; R->cur[0] = 1.0;
}
static void risbo_free(risbo_t* R) { free(R->cur); free(R->tmp); }

static void risbo_halfstep(risbo_t* R) {
  int J2 = R->J2 + 1, P = R->J2 + 1, D = J2 + 1; /* P: previous dim, D: new dim */
  const double* p = R->cur; double* d = R->tmp;
  double s = R->s, c = R->c, inv = 1.0 / (double)J2;
  double* rt = (double*)malloc(sizeof(double) * (size_t)(J2 + 1));
  for (int i = 0; i <= J2; ++i) rt[i] = sqrt((double)i);
#define PP(i, k) (((i) >= 0 && (i) < P && (k) >= 0 && (k) < P) ? p[(i) * P + (k)] : 0.0)
#pragma omp parallel for schedule(static) if (D > 64)
  for (int i = 0; i < D; ++i) {
    double a = rt[J2 - i], b = rt[i];
    for (int k = 0; k < D; ++k) {
      double ak = rt[J2 - k], bk = rt[k];
      double v = ak * (c * a * PP(i, k) + s * b * PP(i - 1, k)) + bk * (-s * a * PP(i, k - 1) + c * b * PP(i - 1, k - 1));
      d[i * D + k] = v * inv;
    }
  }
#undef PP
  free(rt);
  R->tmp = R->cur; R->cur = d; R->J2 = J2;
}
/* Advance to integer l (two half steps). Afterwards Delta^l_{m m'} =
 * cur[(l-m)*(2l+1) + (l-m')]. */
static void risbo_next(risbo_t* R) { risbo_halfstep(R); risbo_halfstep(R); }

#define RIS(R, l, m, mp) ((R)->cur[(size_t)((l) - (m)) * (2 * (l) + 1) + ((l) - (mp))])

/* Full matrix d^l(beta) as out[(m+l)*(2l+1) + (n+l)]. */
void orc_risbo_matrix(int l, double sh, double ch, double* out) {
  risbo_t R; risbo_init(&R, l, sh, ch);
  for (int k = 0; k < l; ++k) risbo_next(&R);
  int D = 2 * l + 1;
  for (int m = -l; m <= l; ++m)
    for (int n = -l; n <= l; ++n) out[(m + l) * D + (n + l)] = RIS(&R, l, m, n);
  risbo_free(&R);
}

static cplx ipow(int k) { /* i^k */
  switch (((k % 4) + 4) % 4) { case 0: return 1.0; case 1: return I; case 2: return -1.0; default: return -I; }
}

/* ------------------------------------------------------------------------ */
/* Spin-SHT quadrature, last step (the sphere analogue of Eq. flml with      */
/* n = -s):                                                                   */
/*   f_lm = (-1)^s i^{m+s} sqrt((2l+1)/4pi) sum_{m'} D^l_{m'm} D^l_{m',-s} G_{m m'} */
/* G is [2L-1 (m)][2L-1 (m')], index m+L-1. f_lm at l*l+l+m (zero for l<|s|). */
/* ------------------------------------------------------------------------ */
void orc_sht_fwd_contract(int L, int s, const double* Gd, double* fd) {
  const cplx* G = (const cplx*)Gd; cplx* f = (cplx*)fd;
  int N = 2 * L - 1;
  memset(f, 0, sizeof(cplx) * (size_t)L * L);
  risbo_t R; risbo_init(&R, L - 1, sqrt(0.5), sqrt(0.5));
  for (int l = 0; l < L; ++l) {
    if (l > 0) risbo_next(&R);
    if (l < abs(s)) continue;
    double nrm = ((s & 1) ? -1.0 : 1.0) * sqrt((2.0 * l + 1) / (4 * M_PI));
#pragma omp parallel for schedule(static)
    for (int m = -l; m <= l; ++m) {
      cplx acc = 0;
      for (int mp = -l; mp <= l; ++mp)
        acc += RIS(&R, l, mp, m) * RIS(&R, l, mp, -s) * G[(size_t)(m + L - 1) * N + (mp + L - 1)];
      f[l * l + l + m] = nrm * ipow(m + s) * acc;
    }
  }
  risbo_free(&R);
}

/* ------------------------------------------------------------------------ */
/* Forward Wigner quadrature, last step, Eq. (flml) in its general-n form:   */
/*   (W)^l_mn = i^{m-n} sum_{m'} D^l_{m'm} D^l_{m'n} Y_{m n m'}               */
/* then the synthesis sum of Eq. (wav_synthesis_harmonic):                    */
/*   f_lm += sum_n (W)^l_mn Psi_ln.                                            */
/* Y is [2Lj-1 (m)][2Lj-1 (n)][2Lj-1 (m')]; psi is [Lj][2Lj-1] (Psi_ln real). */
/* If wl is non-null the coefficients are also written as wl[l][m][n] dense.  */
/* ------------------------------------------------------------------------ */
void orc_wigner_fwd_contract(int Lj, const double* Yd, const double* psi, double* fd, double* wld) {
  const cplx* Y = (const cplx*)Yd; cplx* f = (cplx*)fd; cplx* wl = (cplx*)wld;
  int N = 2 * Lj - 1;
  risbo_t R; risbo_init(&R, Lj - 1, sqrt(0.5), sqrt(0.5));
  for (int l = 0; l < Lj; ++l) {
    if (l > 0) risbo_next(&R);
#pragma omp parallel for schedule(static)
    for (int m = -l; m <= l; ++m) {
      cplx fsum = 0;
      for (int n = -l; n <= l; ++n) {
        const cplx* y = Y + ((size_t)(m + Lj - 1) * N + (n + Lj - 1)) * N;
        cplx acc = 0;
        for (int mp = -l; mp <= l; ++mp) acc += RIS(&R, l, mp, m) * RIS(&R, l, mp, n) * y[mp + Lj - 1];
        cplx w = ipow(m - n) * acc;
        if (wl) wl[((size_t)l * N + (m + Lj - 1)) * N + (n + Lj - 1)] = w;
        fsum += w * psi[(size_t)l * N + (n + Lj - 1)];
      }
      f[l * l + l + m] += fsum;
    }
  }
  risbo_free(&R);
}

/* ------------------------------------------------------------------------ */
/* Curvelet analysis at one SO(3) ring beta_b, Eq. (wav_analysis_harmonic)   */
/* with D^{l*}_mn(a,b,g) = e^{i m a} d^l_mn(b) e^{i n g}:                      */
/*   X[m][n] = sum_l f_lm Psi*_ln d^l_mn(beta)   (Psi real)                    */
/* d^l(beta) comes from Risbo's recursion run at beta itself (stable near the */
/* poles). The (alpha, gamma) sums are done by the numpy layer.               */
/* X is [2Lj-1 (m)][2Lj-1 (n)].                                                */
/* ------------------------------------------------------------------------ */
void orc_analysis_ring(int Lj, const double* fd, const double* psi, double sh, double ch, double* Xd) {
  const cplx* f = (const cplx*)fd; cplx* X = (cplx*)Xd;
  int N = 2 * Lj - 1;
  memset(X, 0, sizeof(cplx) * (size_t)N * N);
  risbo_t R; risbo_init(&R, Lj - 1, sh, ch);
  for (int l = 0; l < Lj; ++l) {
    if (l > 0) risbo_next(&R);
#pragma omp parallel for schedule(static) if (l > 32)
    for (int m = -l; m <= l; ++m) {
      cplx fl = f[l * l + l + m];
      if (fl == 0) continue;
      cplx* x = X + (size_t)(m + Lj - 1) * N + (Lj - 1);
      const double* ps = psi + (size_t)l * N + (Lj - 1);
      for (int n = -l; n <= l; ++n) x[n] += fl * ps[n] * RIS(&R, l, m, n);
    }
  }
  risbo_free(&R);
}

/* The same ring by the l-recurrence (kept for cross-checks at moderate L). */
void orc_analysis_ring_lrec(int Lj, const double* fd, const double* psi, double sh, double ch, double* Xd) {
  const cplx* f = (const cplx*)fd; cplx* X = (cplx*)Xd;
  int N = 2 * Lj - 1;
  double* sq = sqrt_table(Lj);
  xnum* seeds = seed_table(Lj, sh, ch);
  double cb = ch * ch - sh * sh;
#pragma omp parallel
  {
    double* d = (double*)malloc(sizeof(double) * (size_t)Lj);
#pragma omp for schedule(dynamic, 4)
    for (int m = -(Lj - 1); m <= Lj - 1; ++m) {
      for (int n = -(Lj - 1); n <= Lj - 1; ++n) {
        int l0, ks; double sgn;
        seed_index(m, n, &l0, &ks, &sgn);
        d_lrec_core(Lj, m, n, cb, seeds[l0 * l0 + l0 + ks], sgn, sq, d);
        cplx acc = 0;
        for (int l = l0; l < Lj; ++l) acc += f[l * l + l + m] * psi[(size_t)l * N + (n + Lj - 1)] * d[l];
        X[(size_t)(m + Lj - 1) * N + (n + Lj - 1)] = acc;
      }
    }
    free(d);
  }
  free(seeds); free(sq);
}

/* ------------------------------------------------------------------------ */
/* Inverse spin SHT, theta part, Eq. (spin_sphericalHarmonics) summed over l: */
/*   g[r][m] = sum_l f_lm (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}(theta_r)          */
/* for nr colatitudes given by (sh, ch) = (sin, cos)(theta_r/2).              */
/* ------------------------------------------------------------------------ */
void orc_sht_inv_rings(int L, int s, const double* fd, int nr, const double* sh, const double* ch, double* gd) {
  const cplx* f = (const cplx*)fd; cplx* g = (cplx*)gd;
  int N = 2 * L - 1;
  double* sq = sqrt_table(L);
  for (int r = 0; r < nr; ++r) {
    xnum* seeds = seed_table(L, sh[r], ch[r]);
    double cb = ch[r] * ch[r] - sh[r] * sh[r];
#pragma omp parallel
    {
      double* d = (double*)malloc(sizeof(double) * (size_t)L);
#pragma omp for schedule(dynamic, 4)
      for (int m = -(L - 1); m <= L - 1; ++m) {
        int l0, ks; double sgn;
        seed_index(m, -s, &l0, &ks, &sgn);
        d_lrec_core(L, m, -s, cb, (l0 < L) ? seeds[l0 * l0 + l0 + ks] : (xnum){0.0, 0}, sgn, sq, d);
        cplx acc = 0;
        for (int l = l0; l < L; ++l) acc += f[l * l + l + m] * sqrt((2.0 * l + 1) / (4 * M_PI)) * d[l];
        g[(size_t)r * N + (m + L - 1)] = ((s & 1) ? -1.0 : 1.0) * acc;
      }
      free(d);
    }
    free(seeds);
  }
  free(sq);
}

/* ------------------------------------------------------------------------ */
/* Radial kernel pieces: s(t), s_lambda(t) and k_lambda(t) of Sec. II-B, with */
/* the integrals by adaptive Simpson quadrature.                               */
/* ------------------------------------------------------------------------ */
static double schwartz_s(double t) { return (t > -1.0 && t < 1.0) ? exp(-1.0 / (1.0 - t * t)) : 0.0; }
static double s_lambda(double lam, double t) { return schwartz_s(2.0 * lam / (lam - 1.0) * (t - 1.0 / lam) - 1.0); }
static double k_integrand(double lam, double t) { double v = s_lambda(lam, t); return v * v / t; }

static double simpson_rec(double lam, double a, double b, double fa, double fm, double fb, double whole, double eps, int depth) {
  double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  double flm = k_integrand(lam, lm), frm = k_integrand(lam, rm);
  double left = (m - a) / 6.0 * (fa + 4 * flm + fm), right = (b - m) / 6.0 * (fm + 4 * frm + fb);
  double diff = left + right - whole;
  double tol = 15.0 * eps;
  double floor_ = 64.0 * 2.2e-16 * (fabs(left) + fabs(right)); /* rounding level */
  if (depth <= 0 || fabs(diff) <= (tol > floor_ ? tol : floor_)) return left + right + diff / 15.0;
  return simpson_rec(lam, a, m, fa, flm, fm, left, eps / 2, depth - 1) +
         simpson_rec(lam, m, b, fm, frm, fb, right, eps / 2, depth - 1);
}
static double integrate_k(double lam, double a, double b) {
  if (b <= a) return 0.0;
  /* split into 16 panels first so that the bump is always sampled */
  double acc = 0.0, h = (b - a) / 16.0;
  for (int p = 0; p < 16; ++p) {
    double x0 = a + p * h, x1 = (p == 15) ? b : a + (p + 1) * h;
    double f0 = k_integrand(lam, x0), f1 = k_integrand(lam, x1), fm = k_integrand(lam, 0.5 * (x0 + x1));
    double whole = (x1 - x0) / 6.0 * (f0 + 4 * fm + f1);
    acc += simpson_rec(lam, x0, x1, f0, fm, f1, whole, 1e-18, 40);
  }
  return acc;
}
/* k_lambda(a) - k_lambda(b) for a <= b, as one normalised integral over
 * [max(a, 1/lambda), min(b, 1)] (no cancellation where the two are close). */
double orc_k_diff(double lam, double a, double b) {
  double lo = a < 1.0 / lam ? 1.0 / lam : a, hi = b > 1.0 ? 1.0 : b;
  if (hi <= lo) return 0.0;
  return integrate_k(lam, lo, hi) / integrate_k(lam, 1.0 / lam, 1.0);
}

/* s_lambda(t) itself (Sec. II-B), exported for the pins of the radial kernel. */
double orc_s_lambda(double lam, double t) { return s_lambda(lam, t); }

double orc_k_lambda(double lam, double t) {
  if (t < 1.0 / lam) return 1.0;
  if (t >= 1.0) return 0.0;
  return integrate_k(lam, t, 1.0) / integrate_k(lam, 1.0 / lam, 1.0);
}
