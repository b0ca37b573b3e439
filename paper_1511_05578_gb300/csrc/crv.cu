// libcrv host side: plan construction, per-scale pipelines and the C ABI of
// include/crv.h. Device work lives in delta.cu, transforms.cuh, contract.cuh,
// tc_contract.cu, tc_ozaki.cu, df_fft.cu and rotate.cu.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <atomic>
#include <set>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/crv.h"
#include "contract.cuh"
#include "rotate.cuh"
#include "tc_contract.cuh"
#include "tc_ozaki.cuh"
#include "df_fft.cuh"

namespace crv {

static thread_local std::string g_err;

// NVTX range over a scope: the ABI calls, plan creation and the per-scale phases show as named
// ranges in Nsight tools (ncu --nvtx filters on them); without a tool attached a push/pop
// is a no-op.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  NvtxRange(const char* what, int j) {
    char b[64];
    snprintf(b, sizeof b, "%s j=%d", what, j);
    nvtxRangePushA(b);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---- optional per-kind event timing -------------------------------------------
static const char* kKindNames[K_NKINDS] = {"delta", "sht_contract", "sht_rows", "beta_synth", "beta_quad",
                                           "ring_inv_n", "ring_inv_m", "ring_fwd_g", "ring_fwd_a",
                                           "contract_analysis", "contract_synthesis", "tc_analysis",
                                           "tc_synthesis", "misc", "sht_beta", "rotate",
                                           "oz_analysis", "oz_synthesis"};
const char* kind_name(int k) { return (k >= 0 && k < K_NKINDS) ? kKindNames[k] : "?"; }
struct ProfState {
  std::mutex mu;
  std::atomic<unsigned> mask{0};
  struct Pair { int kind; cudaEvent_t a, b; };
  std::vector<Pair> pending;
  std::vector<cudaEvent_t> free_events;
  unsigned long long launches[K_NKINDS] = {0};
  double ms[K_NKINDS] = {0};
  cudaEvent_t get() {
    if (!free_events.empty()) { cudaEvent_t e = free_events.back(); free_events.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void drain(size_t upto) {  // caller holds mu
    for (size_t i = 0; i < upto && i < pending.size(); ++i) {
      cudaEventSynchronize(pending[i].b);
      float t = 0;
      cudaEventElapsedTime(&t, pending[i].a, pending[i].b);
      ms[pending[i].kind] += t;
      free_events.push_back(pending[i].a);
      free_events.push_back(pending[i].b);
    }
    pending.erase(pending.begin(), pending.begin() + std::min(upto, pending.size()));
  }
};
static ProfState g_prof;

KTimer::KTimer(int k, cudaStream_t st) : kind(k), s(st) {
  if (!(g_prof.mask.load() & (1u << k))) return;
  std::lock_guard<std::mutex> g(g_prof.mu);
  a = g_prof.get();
  cudaEventRecord(a, s);
}
void KTimer::done() {
  count_launch();
  if (!a) return;
  std::lock_guard<std::mutex> g(g_prof.mu);
  cudaEvent_t b = g_prof.get();
  cudaEventRecord(b, s);
  g_prof.pending.push_back({kind, a, b});
  g_prof.launches[kind] += 1;
  a = nullptr;
  if (g_prof.pending.size() > 32768) g_prof.drain(16384);
}
bool launch_ok(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
  }
  return true;
}
static int fail(int code, const std::string& msg) { g_err = msg; return code; }
void set_error(const std::string& msg) { g_err = msg; }

cudaError_t build_delta(int L, double* Q, float* q32, double* seed_v, int* seed_e, cudaStream_t st);

// ---------------------------------------------------------------------------
// Host numerics for the plan tables
// ---------------------------------------------------------------------------
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1, p2 = 0;
      for (int k = 1; k <= n; ++k) { double p3 = p2; p2 = p1; p1 = ((2.0 * k - 1) * z * p2 - (k - 1.0) * p3) / k; }
      pp = n * (z * p1 - p2) / (z * z - 1);
      double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p1 = 1, p2 = 0;
    for (int k = 1; k <= n; ++k) { double p3 = p2; p2 = p1; p1 = ((2.0 * k - 1) * z * p2 - (k - 1.0) * p3) / k; }
    pp = n * (z * p1 - p2) / (z * z - 1);
    x[i] = z;
    w[i] = 2.0 / ((1 - z * z) * pp * pp);
  }
}

// k_lambda(t) of Sec. II-B: int_t^1 s_lambda(x)^2 / x dx normalised by the integral
// from 1/lambda; composite Gauss-Legendre (64 panels x 20 points).
struct KLambda {
  double lam, norm;
  std::vector<double> gx, gw;
  static double sfun(double t) { return (t > -1 && t < 1) ? std::exp(-1.0 / (1.0 - t * t)) : 0.0; }
  double integrand(double x) const {
    double v = sfun(2 * lam / (lam - 1) * (x - 1 / lam) - 1);
    return v * v / x;
  }
  double integral(double a, double b) const {
    if (b <= a) return 0;
    const int panels = 64;
    double h = (b - a) / panels, acc = 0;
    for (int p = 0; p < panels; ++p) {
      double c = a + (p + 0.5) * h;
      for (size_t i = 0; i < gx.size(); ++i) acc += gw[i] * integrand(c + 0.5 * h * gx[i]);
    }
    return acc * 0.5 * h;
  }
  explicit KLambda(double l) : lam(l) { gauss_legendre(20, gx, gw); norm = integral(1 / lam, 1); }
  double operator()(double t) const {
    if (t < 1 / lam) return 1.0;
    if (t >= 1) return 0.0;
    return integral(t, 1) / norm;
  }
  // k(a) - k(b), a <= b, as one integral over [max(a,1/lam), min(b,1)]: no
  // cancellation next to the ends of the support, where kappa^2 is tiny.
  double diff(double a, double b) const {
    const double lo = std::max(a, 1 / lam), hi = std::min(b, 1.0);
    return hi > lo ? integral(lo, hi) / norm : 0.0;
  }
};

static int ceil_pow(double lam, int e) {
  double v = std::pow(lam, e), r = std::round(v);
  if (std::fabs(v - r) < 1e-9 * std::max(1.0, v)) return (int)r;
  return (int)std::ceil(v);
}

// d^l_{k,l}(theta) for k = -l..l: sqrt(C(2l,l+k)) sin(t/2)^{l-k} cos(t/2)^{l+k}
// (Eq. wigner_sum_reln, one surviving term), by ratios from the largest entry and
// normalised with sum_k d^2 = 1 (a column of an orthogonal matrix).
static void edge_row(int l, double sh, double ch, std::vector<double>& out) {
  out.assign(2 * l + 1, 0.0);
  if (l == 0) { out[0] = 1.0; return; }
  if (sh == 0.0) { out[2 * l] = 1.0; return; }
  if (ch == 0.0) { out[0] = 1.0; return; }
  const double rat = ch / sh;
  // ratio r_k = d_{k+1}/d_k = sqrt((l-k)/(l+k+1)) * ch/sh; peak where r_k crosses 1
  int kp = -l;
  while (kp < l && std::sqrt((double)(l - kp) / (l + kp + 1)) * rat > 1.0) ++kp;
  out[kp + l] = 1.0;
  for (int k = kp; k < l; ++k) {
    double v = out[k + l] * std::sqrt((double)(l - k) / (l + k + 1)) * rat;
    out[k + 1 + l] = v;
    if (v < 1e-300) break;
  }
  for (int k = kp; k > -l; --k) {
    double v = out[k + l] / (std::sqrt((double)(l - k + 1) / (l + k)) * rat);
    out[k - 1 + l] = v;
    if (v < 1e-300) break;
  }
  double s2 = 0;
  for (double v : out) s2 += v * v;
  const double nrm = 1.0 / std::sqrt(s2);
  for (double& v : out) v *= nrm;
}

static void host_fft(std::vector<std::complex<double>>& a, int sign) {
  const int n = (int)a.size();
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < len / 2; ++k) {
        double ang = sign * 2 * M_PI * k / len;
        std::complex<double> w(std::cos(ang), std::sin(ang));
        std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

static int next_pow2(int n) { int p = 1; while (p < n) p <<= 1; return p; }

}  // namespace crv

using namespace crv;

// ---------------------------------------------------------------------------
// The plan
// ---------------------------------------------------------------------------
struct FftSet {
  DftTab<double> d; DftTab<float> f; DftTab<df> x;  // x: double-float (FP64 plans, P = 4096)
  CorrTab<double> cd; CorrTab<float> cf; CorrTab<df> cx2;
};

// Device allocations of the read-only tables of a plan (Delta, Delta Psi tensor-core
// tables, FFT tables, kernels): one set per crv_plan_create, shared by the plan and its clones
// (crv_plan_clone) and freed with the last of them.
// A guard region (CRV_F_GUARD plans): the kGuardBytes after the end of one device buffer,
// filled with kGuardByte at allocation and compared by crv_plan_check_guards.
constexpr size_t kGuardBytes = 4096;
constexpr unsigned char kGuardByte = 0xA5;
struct Guard {
  unsigned char* p;
  size_t size;  // the buffer's own size (the guard starts there)
};

struct TableSet {
  std::vector<void*> allocs;
  std::vector<Guard> guards;
  size_t bytes = 0;
  TableSet() = default;
  TableSet(const TableSet&) = delete;
  TableSet& operator=(const TableSet&) = delete;
  ~TableSet() {
    for (void* p : allocs) cudaFree(p);
  }
};

// The (m, n) column set of a scale of band limit Lb: m >= 0 only for real signals (conjugate
// symmetry); even n only for rotated spin-0 curvelets (zeta_lk = 0 for odd k at vartheta =
// pi/2), while the unrotated ones sit at n = +-l, which covers every n.
static ColSet colset_for(int Lb, bool real, int spin, bool unrot) {
  ColSet c;
  c.Mc = real ? Lb : 2 * Lb - 1;
  c.m0 = real ? 0 : -(Lb - 1);
  c.nstep = (spin == 0 && !unrot) ? 2 : 1;
  c.n0 = -(Lb - 1);
  if (c.nstep == 2 && (c.n0 & 1)) c.n0 += 1;
  c.Nc = (-c.n0 - c.n0) / c.nstep + 1;
  c.extra = 0;
  c.fNc = FastDiv((uint32_t)c.Nc);
  return c;
}

struct crv_plan_s {
  int L = 0, J0 = 0, J = 0, spin = 0, max_batch = 0, Lphi = 1;
  unsigned flags = 0;
  double lambda = 2;
  bool real = false, mixed = false, wfp32 = false;
  bool unrot = false;  // coefficients of the unrotated curvelets (CRV_F_UNROTATED)
  // per scale, the smallest l >= |s| with kappa^(j)(l) > 0: Psi_ln = 0 below it, so the
  // tensor-core K runs (analysis) and l-tiles (synthesis) start there; in unrotated plans
  // also the columns with |n| below it are zero, as are those with |m| > |n|, and dpmap
  // lists the column pairs that are not zero, the only ones the beta transforms visit
  std::vector<int> nlo;
  std::vector<int*> dpmap;
  std::vector<int> npmap;
  std::vector<int> Lj;
  std::vector<double> kappa;  // [J+1][L]
  std::vector<double> phi;    // [L]
  std::vector<std::vector<double>> psi;  // per j: [Lj][2Lj-1]
  std::vector<double*> dedge;            // per j: d^l_{k,l}(vartheta^j) at [l][k + Lj - 1] (rotation of Wigner coefficients)
  double* dQ = nullptr;
  float* dQ32 = nullptr;
  std::vector<double*> dpsi;
  std::vector<float*> dpsi32;
  double* dphi = nullptr;
  std::map<int, FftSet> fft;  // keyed by band limit Lb
  // workspace
  cx<double>* wflm = nullptr;
  cx<double>* wflm2 = nullptr;
  cx<float>* wflm32 = nullptr;  // FP32 copy of the analysed f_lm (tensor-core operand source)
  cx<double>* wF = nullptr;
  cx<double>* wG = nullptr;
  void* wX = nullptr;
  void* wXb = nullptr;
  void* wR = nullptr;
  bool use_tc = false;   // tensor-core contractions (mixed plans)
  std::vector<TcTab> tabA, tabS;  // per scale: B operand tables of the two contractions
  std::vector<TcATab> tabAA;        // per scale: chunk offsets of the per-map A tables (one buffer)
  int* d_err = nullptr;   // [0]: set by kernels whose bounded waits gave up; [1]: tile counter of the tensor-core engine
  size_t vol_bytes = 0, ring_bytes = 0;
  long long a_chunks = 0;  // chunks of the per-map A tables of the analysis (largest scale)
  // FP64 tensor-core contractions (CRV_F_FP64_TC): per scale the sliced B tables of the two
  // contractions, and the layout of the per-map A tables with the passes over m' that keep
  // one pass's A table within oz_cap chunks (one buffer per instance)
  bool use_oz = false;
  bool df_fft = false;  // FP64 plans: the P = 4096 Wigner FFTs of real signals in double-float
  struct OzA {
    const long long* base = nullptr;
    const int2* range = nullptr;
    int ntiles = 0;
    std::vector<long long> cum;  // chunk offset of m' (its first tile)
    std::vector<int> cuts;       // pass boundaries over m': cuts[i] .. cuts[i + 1]
  };
  std::vector<OzTab> ozBA, ozBS;
  std::vector<OzA> ozAA, ozAS;
  long long oz_cap = 0;  // chunks of the A buffer
  int oz_bits = 7;       // digit width: 7 while every K range is <= 1024, else 6
  int oz_mp_cap = 0;     // largest number of m' in a pass (rows of the exponent buffer)
  float* oz_av = nullptr;
  int* oz_ae = nullptr;
  std::shared_ptr<TableSet> tabs;  // read-only tables, shared with clones
  std::vector<void*> allocs;       // this instance's workspace
  size_t bytes = 0;
  // Maps of one call run concurrently on worker instances: clones of this plan (shared tables,
  // own workspace), each on a stream of its own forked from the caller's stream by an event
  // and joined back into it (workers[w - 1] on wstreams[w - 1]; worker 0 is the plan itself).
  std::vector<crv_plan_s*> workers;
  std::vector<cudaStream_t> wstreams;
  std::vector<cudaEvent_t> wdone;
  cudaEvent_t fork_ev = nullptr;
  int nworkers = 1;                // workers a call uses (<= 1 + workers.size())
  bool tuned = false;              // nworkers and ring_bytes chosen by the autotuner

  bool guard = false;         // CRV_F_GUARD: every buffer followed by a checked guard region
  std::vector<Guard> guards;  // this instance's workspace guards

  // One device buffer of b bytes; with guards, kGuardBytes more, filled with kGuardByte and
  // recorded in `gl`.
  void* raw_alloc(size_t b, int* status, std::vector<Guard>* gl) {
    void* p = nullptr;
    if (b == 0) b = 16;
    cudaError_t e = cudaMalloc(&p, guard ? b + kGuardBytes : b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *status = fail(CRV_ENOMEM, "cudaMalloc of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
      return nullptr;
    }
    if (guard) {
      unsigned char* g = (unsigned char*)p + b;
      if (cudaMemset(g, kGuardByte, kGuardBytes) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(p);
        *status = fail(CRV_ECUDA, "guard region initialisation failed");
        return nullptr;
      }
      gl->push_back(Guard{g, b});
    }
    return p;
  }
  // workspace (per instance)
  template <class P> P* dalloc(size_t n, int* status) {
    if (*status != CRV_OK) return nullptr;
    void* p = raw_alloc(n * sizeof(P), status, &guards);
    if (!p) return nullptr;
    allocs.push_back(p);
    bytes += std::max<size_t>(n * sizeof(P), 16);
    return (P*)p;
  }
  // read-only tables (shared)
  template <class P> P* talloc(size_t n, int* status) {
    if (*status != CRV_OK) return nullptr;
    void* p = raw_alloc(n * sizeof(P), status, &tabs->guards);
    if (!p) return nullptr;
    tabs->allocs.push_back(p);
    tabs->bytes += std::max<size_t>(n * sizeof(P), 16);
    return (P*)p;
  }
  ~crv_plan_s() {
    for (crv_plan_s* w : workers) delete w;
    for (cudaStream_t st : wstreams) cudaStreamDestroy(st);
    for (cudaEvent_t e : wdone) cudaEventDestroy(e);
    if (fork_ev) cudaEventDestroy(fork_ev);
    for (void* p : allocs) cudaFree(p);
  }
  ColSet colset(int Lb) const { return colset_for(Lb, real, spin, unrot); }
  int mc(int Lb) const { return colset(Lb).Mc; }
  int m0(int Lb) const { return colset(Lb).m0; }
  int nstep() const { return colset(1).nstep; }
  int n0(int Lb) const { return colset(Lb).n0; }
  int nc(int Lb) const { return colset(Lb).Nc; }
};

// The A table of pass [cuts[i], cuts[i + 1]) of a per-map A layout, in the plan's buffer.
static OzTab oz_pass(const crv_plan_s* p, const crv_plan_s::OzA& a, int i) {
  OzTab t;
  t.mp0 = a.cuts[i];
  t.mp1 = a.cuts[i + 1];
  t.v = p->oz_av;
  t.e = p->oz_ae;
  t.base = a.base + (size_t)t.mp0 * a.ntiles;
  t.range = a.range + (size_t)t.mp0 * a.ntiles;
  t.ntiles = a.ntiles;
  t.rows = a.ntiles * OZ_AROWS;
  t.c0 = a.cum[t.mp0];
  t.bits = p->oz_bits;
  return t;
}

template <class T> static const DftTab<T>& dft_of(const FftSet& s);
template <> const DftTab<double>& dft_of<double>(const FftSet& s) { return s.d; }
template <> const DftTab<df>& dft_of<df>(const FftSet& s) { return s.x; }
template <> const DftTab<float>& dft_of<float>(const FftSet& s) { return s.f; }
template <class T> static const CorrTab<T>& corr_of(const FftSet& s);
template <> const CorrTab<double>& corr_of<double>(const FftSet& s) { return s.cd; }
template <> const CorrTab<df>& corr_of<df>(const FftSet& s) { return s.cx2; }
template <> const CorrTab<float>& corr_of<float>(const FftSet& s) { return s.cf; }

static int build_fft(crv_plan_s* p, int Lb) {
  if (p->fft.count(Lb)) return CRV_OK;
  const int N = 2 * Lb - 1;
  const int P = std::max(16, next_pow2(2 * N - 1));
  const int Q = P;  // 2N - 1 = 4Lb - 3: the correlation of Eq. gmnmp fits the same length
  int lp = 0;
  while ((1 << lp) < P) ++lp;
  const int R0 = (lp % 4) ? (1 << (lp % 4)) : 16;
  const int nst = 1 + (lp - (R0 == 16 ? 4 : lp % 4)) / 4;
  // stage twiddles of the P-point FFT: stage s >= 1 with Ns = R0 16^(s-1) done holds
  // [e][k] = e^{-2 pi i k 2^e / (16 Ns)}, e < 4, k < Ns
  std::vector<std::complex<double>> stw;
  for (int s = 1, Ns = R0; s < nst; ++s, Ns *= 16)
    for (int e = 0; e < 4; ++e)
      for (int k = 0; k < Ns; ++k) stw.push_back(std::polar(1.0, -2 * M_PI * (double)k * (1 << e) / (16.0 * Ns)));
  if (stw.empty()) stw.push_back(1.0);
  std::vector<std::complex<double>> chirp(N), kf(P, 0.0), ki(P, 0.0), wv(Q, 0.0), hp(N), bsyn(N), bquad(N);
  for (int j = 0; j < N; ++j) {  // e^{i pi m/N} with m = j or j - N (|m| < Lb)
    const int m = (j < Lb) ? j : j - N;
    hp[j] = std::polar(1.0, M_PI * (double)m / N);
  }
  for (int t = 0; t < N; ++t) {
    long long r = ((long long)t * t) % (2LL * N);
    chirp[t] = std::polar(1.0, -M_PI * (double)r / N);
  }
  for (int j = 0; j < N; ++j) {
    bsyn[j] = hp[j] * std::conj(chirp[j]);
    bquad[j] = chirp[j] * std::conj(hp[j]) / (double)N;
  }
  for (int t = -(N - 1); t <= N - 1; ++t) {
    const int a = t < 0 ? -t : t;
    kf[((t % P) + P) % P] = std::conj(chirp[a]);  // forward: b_t = conj(h_t)
    ki[((t % P) + P) % P] = chirp[a];             // inverse: b_t = conj(conj(h_t))
  }
  host_fft(kf, -1);
  host_fft(ki, -1);
  for (auto& v : kf) v /= (double)P;
  for (auto& v : ki) v /= (double)P;
  // v[t] = w_e(-t) = w_e(t), t in [-(2Lb-2), 2Lb-2]: the even part of the weights
  // w(p) = int_0^pi sin(b) e^{i p b} db, i.e. 2 / (1 - p^2) for even p and 0 for odd p (the
  // odd part, +-i pi/2 at p = +-1, cancels in the folded quadrature)
  for (int t = -(2 * Lb - 2); t <= 2 * Lb - 2; ++t) {
    const int pp = -t;
    const double w = (pp % 2 == 0) ? 2.0 / (1.0 - (double)pp * pp) : 0.0;
    wv[((t % Q) + Q) % Q] = w;
  }
  host_fft(wv, -1);
  for (auto& v : wv) v /= (double)Q;

  int st = CRV_OK;
  FftSet s;
  auto up = [&](const std::vector<std::complex<double>>& v, cx<double>*& dd, cx<float>*& df) {
    dd = p->talloc<cx<double>>(v.size(), &st);
    df = p->talloc<cx<float>>(v.size(), &st);
    if (st != CRV_OK) return;
    std::vector<cx<double>> hd(v.size());
    std::vector<cx<float>> hf(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      hd[i] = mk(v[i].real(), v[i].imag());
      hf[i] = mk((float)v[i].real(), (float)v[i].imag());
    }
    cudaMemcpy(dd, hd.data(), v.size() * sizeof(cx<double>), cudaMemcpyHostToDevice);
    cudaMemcpy(df, hf.data(), v.size() * sizeof(cx<float>), cudaMemcpyHostToDevice);
  };
  cx<double>* d; cx<float>* f;
  s.d.N = s.f.N = N; s.d.P = s.f.P = P;
  s.d.R0 = s.f.R0 = R0; s.d.nst = s.f.nst = nst;
  up(stw, d, f); s.d.stw = d; s.f.stw = f;
  up(chirp, d, f); s.d.chirp = d; s.f.chirp = f;
  up(kf, d, f); s.d.khat_f = d; s.f.khat_f = f;
  up(ki, d, f); s.d.khat_i = d; s.f.khat_i = f;
  up(hp, d, f); s.d.hphase = d; s.f.hphase = f;
  up(bsyn, d, f); s.d.bsyn = d; s.f.bsyn = f;
  up(bquad, d, f); s.d.bquad = d; s.f.bquad = f;
  s.cd.Q = s.cf.Q = Q;
  up(wv, d, f); s.cd.what = d; s.cf.what = f;
  if ((P == 4096 || P == 2048) && !p->mixed) {  // double-float copies (hi + lo of every double), FP64 plans
    auto upx = [&](const std::vector<std::complex<double>>& v) -> const cx<df>* {
      cx<df>* dx = p->talloc<cx<df>>(v.size(), &st);
      if (st != CRV_OK) return nullptr;
      std::vector<cx<df>> hx(v.size());
      for (size_t i = 0; i < v.size(); ++i) hx[i] = mk(df(v[i].real()), df(v[i].imag()));
      cudaMemcpy(dx, hx.data(), v.size() * sizeof(cx<df>), cudaMemcpyHostToDevice);
      return dx;
    };
    s.x.N = N; s.x.P = P; s.x.R0 = R0; s.x.nst = nst;
    s.x.stw = upx(stw); s.x.chirp = upx(chirp); s.x.khat_f = upx(kf); s.x.khat_i = upx(ki);
    s.x.hphase = upx(hp); s.x.bsyn = upx(bsyn); s.x.bquad = upx(bquad);
    s.cx2.Q = Q; s.cx2.what = upx(wv);
  }
  if (st != CRV_OK) return st;
  p->fft[Lb] = s;
  return CRV_OK;
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------

// Function attributes and device properties are per device: both caches are keyed by the
// device ordinal current at the call.
namespace crv {
static std::mutex g_dev_mu;
bool func_attr_once(const void* kernel, int bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  static std::map<std::pair<const void*, int>, int> done;
  std::lock_guard<std::mutex> g(g_dev_mu);
  auto it = done.find({kernel, dev});
  if (it != done.end() && it->second >= bytes) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
    g_err = "cudaFuncSetAttribute(max dynamic smem) failed";
    return false;
  }
  done[{kernel, dev}] = bytes;
  return true;
}
int device_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  static std::map<int, int> sms;
  std::lock_guard<std::mutex> g(g_dev_mu);
  auto it = sms.find(dev);
  if (it != sms.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  sms[dev] = n;
  return n;
}
}  // namespace crv

template <class K>
static bool set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return true;
  return func_attr_once((const void*)kernel, (int)bytes);
}

// Shared-memory carveout of a kernel set to what `blocks` resident blocks of `bytes` each need
// (and no more), so that the rest of the SM's unified L1/shared storage stays L1: the ring
// transforms' strided loads depend on L1 capacity. Once per kernel and device.
void crv::carveout_for(const void* kernel, size_t bytes, int blocks) {
  int dev = 0;
  cudaGetDevice(&dev);
  static std::set<std::pair<const void*, int>> done;
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  if (done.count({kernel, dev})) return;
  int maxsm = 0;
  if (cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || maxsm <= 0) {
    cudaGetLastError();
    return;
  }
  const size_t need = (size_t)blocks * (bytes + 1024);  // + the per-block reservation
  const int pct = (int)std::min<size_t>(100, (need * 100 + maxsm - 1) / maxsm);
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess)
    cudaGetLastError();  // a preference only: the launch works either way
  done.insert({kernel, dev});
}

static int num_sms() { return device_sms(); }

// Persistent FFT blocks (one or two per SM, by shared memory and registers), each
// looping over groups of G sequences.
template <class T, int NT, bool COLS, int PT, class Ld, class St>
static bool run_dft_nt(int kind, const DftTab<T>& tb, int sign, int nseq, Ld ld, St st, cudaStream_t s) {
  const int G = NT / (tb.P / 16);
  if (G < 1) { g_err = "FFT length too large for the block"; return false; }
  const size_t smem = fft_smem_bytes<T>(NT);
  auto kern = dft_kernel<T, NT, COLS, PT, Ld, St>;
  if (!set_smem(kern, smem)) return false;
  const int bps = FftMinBlocks<T, NT>::value;
  carveout_for((const void*)kern, smem, bps);
  const int grid = std::max(1, std::min((nseq + G - 1) / G, num_sms() * bps));
  KTimer kt(kind, s);
  kern<<<grid, NT, smem, s>>>(tb, sign, nseq, ld, st);
  kt.done();
  return launch_ok(kind_name(kind));
}
// FP32: 256 threads (two blocks per SM); FP64: 256 threads, one block per SM. The lengths
// of the two largest band limits get kernels compiled for their P (both precisions).
template <class T, bool COLS, class Ld, class St>
static bool run_dft(int kind, const DftTab<T>& tb, int sign, int nseq, Ld ld, St st, cudaStream_t s) {
  if (nseq <= 0) return true;
  if (tb.P == 4096) return run_dft_nt<T, 256, COLS, 4096>(kind, tb, sign, nseq, ld, st, s);
  if (tb.P == 2048) return run_dft_nt<T, 256, COLS, 2048>(kind, tb, sign, nseq, ld, st, s);
  return run_dft_nt<T, 256, COLS, 0>(kind, tb, sign, nseq, ld, st, s);
}
template <class T, class Ld, class St>
static bool run_rows(int kind, const DftTab<T>& tb, int sign, int n, Ld ld, St st, cudaStream_t s) {
  return run_dft<T, false>(kind, tb, sign, n, ld, st, s);
}
template <class T, class Ld, class St>
static bool run_cols(int kind, const DftTab<T>& tb, int sign, int n, Ld ld, St st, cudaStream_t s) {
  return run_dft<T, true>(kind, tb, sign, n, ld, st, s);
}

// Beta transforms: 512 FP32 threads (two adjacent column pairs per load), each block on a
// contiguous run of pairs (neighbouring columns share sectors through L1; measured).
template <class T, int NT, int PT>
static bool run_beta_synth_nt(const DftTab<T>& tb, int Lb, int ncols, const cx<T>* X, cx<T>* Y, ColSet cs,
                              int kind, PairMap pm, cudaStream_t s) {
  const int G = NT / (tb.P / 16);
  if (G < 1) { g_err = "FFT length too large for the block"; return false; }
  const size_t smem = fft_smem_bytes_tabs<T>(NT, tb.P, 1);
  if (!set_smem(beta_synth_kernel<T, NT, PT>, smem)) return false;
  const int bps = FftMinBlocks<T, NT>::value;
  const int npair = pm.idx ? pm.n : num_col_pairs(cs);
  if (npair <= 0) return true;
  const int grid = std::max(1, std::min((npair + G - 1) / G, num_sms() * bps));
  KTimer kt(kind, s);
  beta_synth_kernel<T, NT, PT><<<grid, NT, smem, s>>>(tb, ncols, Lb, X, Y, cs, pm);
  kt.done();
  return launch_ok("beta_synth_kernel");
}
// Synthesis over beta of all column pairs: X[m'][c] -> Y[b][c].
template <class T>
static bool run_beta_synth(const DftTab<T>& tb, int Lb, int ncols, const cx<T>* X, cx<T>* Y, ColSet cs, int kind,
                           cudaStream_t s, PairMap pm = PairMap()) {
  if (ncols <= 0) return true;
  constexpr int NT = sizeof(T) == 4 ? 512 : 256;
  if (tb.P == 4096) return run_beta_synth_nt<T, NT, 4096>(tb, Lb, ncols, X, Y, cs, kind, pm, s);
  if (tb.P == 2048) return run_beta_synth_nt<T, NT, 2048>(tb, Lb, ncols, X, Y, cs, kind, pm, s);
  return run_beta_synth_nt<T, NT, 0>(tb, Lb, ncols, X, Y, cs, kind, pm, s);
}

template <class T, int NT, int PT>
static bool run_beta_quad_nt(const DftTab<T>& tb, const CorrTab<T>& ct, int Lb, int ncols, const cx<T>* Xb, cx<T>* Y,
                             ColSet cs, T scale, int pa, int pb, int pc, PairMap pm, int kind, cudaStream_t s) {
  const int G = NT / (tb.P / 16);
  if (G < 1) { g_err = "FFT length too large for the block"; return false; }
  const size_t smem = fft_smem_bytes_tabs<T>(NT, tb.P, 2);
  if (!set_smem(beta_quad_kernel<T, NT, PT>, smem)) return false;
  const int bps = FftMinBlocks<T, NT>::value;
  const int npair = pm.idx ? pm.n : num_col_pairs(cs);
  if (npair <= 0) return true;
  const int grid = std::max(1, std::min((npair + G - 1) / G, num_sms() * bps));
  KTimer kt(kind, s);
  beta_quad_kernel<T, NT, PT><<<grid, NT, smem, s>>>(tb, ct, ncols, Lb, Xb, Y, cs, scale, pa, pb, pc, pm);
  kt.done();
  return launch_ok("beta_quad_kernel");
}
template <class T>
static bool run_beta_quad(const FftSet& fs, int Lb, int ncols, const cx<T>* Xb, cx<T>* Y, ColSet cs, T scale,
                          int pa, int pb, int pc, cudaStream_t s, PairMap pm = PairMap(), int kind = K_BETA_QUAD) {
  const DftTab<T>& tb = dft_of<T>(fs);
  const CorrTab<T>& ct = corr_of<T>(fs);
  if (ct.Q != tb.P) { g_err = "beta quadrature needs Q == P"; return false; }
  if (ncols <= 0) return true;
  constexpr int NT = sizeof(T) == 4 ? 512 : 256;
  if (tb.P == 4096) return run_beta_quad_nt<T, NT, 4096>(tb, ct, Lb, ncols, Xb, Y, cs, scale, pa, pb, pc, pm, kind, s);
  if (tb.P == 2048) return run_beta_quad_nt<T, NT, 2048>(tb, ct, Lb, ncols, Xb, Y, cs, scale, pa, pb, pc, pm, kind, s);
  return run_beta_quad_nt<T, NT, 0>(tb, ct, Lb, ncols, Xb, Y, cs, scale, pa, pb, pc, pm, kind, s);
}

// ---------------------------------------------------------------------------
// Spin SHT on the MW grid (always FP64)
// ---------------------------------------------------------------------------
static bool sht_forward(crv_plan_s* p, const double* map, cx<double>* flm, int Ls, int s, bool real, cudaStream_t st) {
  const FftSet& fs = p->fft.at(Ls);
  const int N = 2 * Ls - 1;
  const int Mc = real ? Ls : N, m0 = real ? 0 : -(Ls - 1);
  LdMapRowT<double> ld{LdMapRow{map, N, real}};
  StSHTRow<double> sr{p->wF, Mc, m0, N, 1.0 / N};
  if (!run_rows<double>(K_SHT_ROWS, fs.d, -1, Ls, ld, sr, st)) return false;
  ColSet cs{Mc, m0, 1, 0, 1, s};
  if (!run_beta_quad<double>(fs, Ls, Mc, p->wF, p->wG, cs, 2 * M_PI, 1, 0, imod(3 * s, 4), st, PairMap(), K_SHT_BETA))
    return false;
  cudaMemsetAsync(flm, 0, sizeof(cx<double>) * Ls * Ls, st);
  dim3 g((Mc + 127) / 128, Ls);
  {
    KTimer kt(K_SHT_CONTRACT, st);
    sht_fwd_contract_kernel<<<g, 128, 0, st>>>(p->dQ, p->L, p->wG, Ls, s, Mc, m0, flm);
    kt.done();
  }
  if (!launch_ok("sht_fwd_contract_kernel")) return false;
  KTimer kt(K_MISC, st);
  flm_finish_kernel<<<(Ls * Ls + 255) / 256, 256, 0, st>>>(flm, Ls, s, real);
  kt.done();
  return launch_ok("flm_finish_kernel");
}

static bool sht_inverse(crv_plan_s* p, const cx<double>* flm, double* map, int Ls, int s, bool real, cudaStream_t st) {
  const FftSet& fs = p->fft.at(Ls);
  const int N = 2 * Ls - 1;
  const int Mc = real ? Ls : N, m0 = real ? 0 : -(Ls - 1);
  dim3 g((Mc + 127) / 128, Ls);
  KTimer kt(K_SHT_CONTRACT, st);
  sht_inv_contract_kernel<<<g, 128, (size_t)Ls * sizeof(double), st>>>(p->dQ, p->L, flm, Ls, s, Mc, m0, p->wG);
  kt.done();
  if (!launch_ok("sht_inv_contract_kernel")) return false;
  ColSet cs{Mc, m0, 1, 0, 1, s};
  if (!run_beta_synth<double>(fs.d, Ls, Mc, p->wG, p->wF, cs, K_SHT_BETA, st)) return false;
  LdSHTRow<double> lr{p->wF, Mc, m0, N, real};
  StMapRow sm{map, N, real};
  return run_rows<double>(K_SHT_ROWS, fs.d, +1, Ls, lr, sm, st);
}

// ---------------------------------------------------------------------------
// Wigner transforms of one scale
// ---------------------------------------------------------------------------
template <class T> static const T* q_of(crv_plan_s* p);
template <> const double* q_of<double>(crv_plan_s* p) { return p->dQ; }
template <> const float* q_of<float>(crv_plan_s* p) { return p->dQ32; }
template <class T> static const T* psi_of(crv_plan_s* p, int j);
template <> const double* psi_of<double>(crv_plan_s* p, int j) { return p->dpsi[j]; }
template <> const float* psi_of<float>(crv_plan_s* p, int j) { return p->dpsi32[j]; }

// Rings per chunk of the ring buffer: real signals hold [a][h] (N x Nh) per ring, complex
// ones [m][g] with rows padded to N + 1 (analysis) or [a][n] (synthesis).
static int ring_chunk(crv_plan_s* p, int Lb, size_t elem) {
  const int N = 2 * Lb - 1;
  const ColSet cs = p->colset(Lb);
  const size_t per = p->real ? (size_t)N * (cs.Nc - (-cs.n0 / cs.nstep)) * elem
                             : (size_t)(N + 1) * std::max(p->mc(Lb), p->nc(Lb)) * elem;
  return (int)std::max<size_t>(1, std::min<size_t>((size_t)Lb, p->ring_bytes / per));
}

// Ring steps of the analysis for rings b0 .. b0 + nr - 1 (Eq. inverse_feul over (m, n));
// Z: unrotated plans, whose columns below nlo and entries |m| > |n| are zero.
template <class T, class OutT, bool Z>
static bool ring_inverse(crv_plan_s* p, const FftSet& fs, const ColSet& cs, const cx<T>* Xb, cx<T>* R, OutT* W, int b0,
                         int nr, int N, int ni0, int Nh, int h0, int nlo, size_t wstride, cudaStream_t st) {
  const int Nhs = Nh - h0;
  if (p->real) {
    // m step on the n >= 0 columns, then the n step with real output, rows in pairs
    if (Nhs > 0) {
      LdRingMHalf<T, Z> lm{Xb + (size_t)b0 * cs.pitch(), cs, ni0, N, Nhs, FastDiv((uint32_t)Nhs), h0};
      StRingMHalf<T> sm{R, N, Nhs, FastDiv((uint32_t)Nhs), Nh, h0};
      if (!run_cols<T>(K_RING_INV_M, dft_of<T>(fs), +1, nr * Nhs, lm, sm, st)) return false;
    }
    const int npair = (N + 1) / 2;
    LdRingNHerm<T, Z> ln{R, N, Nh, cs.nstep, npair, FastDiv((uint32_t)npair), nlo};
    StWRowPair<T, OutT> sw{W + (size_t)b0 * wstride, N, npair, FastDiv((uint32_t)npair)};
    return run_rows<T>(K_RING_INV_N, dft_of<T>(fs), +1, nr * npair, ln, sw, st);
  }
  LdRingN<T, Z> ln{Xb + (size_t)b0 * cs.pitch(), cs, N, FastDiv((uint32_t)cs.Mc), nlo};
  StContig<T> sc{R, N + 1};
  if (!run_rows<T>(K_RING_INV_N, dft_of<T>(fs), +1, nr * cs.Mc, ln, sc, st)) return false;
  LdRingM<T> lm{R, cs.Mc, cs.m0, N, N + 1, false, FastDiv((uint32_t)N)};
  StW<T, OutT> sw{W + (size_t)b0 * wstride, N, false, FastDiv((uint32_t)N)};
  return run_cols<T>(K_RING_INV_M, dft_of<T>(fs), +1, nr * N, lm, sw, st);
}

// Values of an FP64 plan's (m, n, m') volume between FP64 (contractions) and double-float
// (FFTs), in place: both take 16 bytes per complex value.
template <bool TO_DF>
__global__ void convert_volume_kernel(void* v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if constexpr (TO_DF) {
      const cx<double> a = reinterpret_cast<cx<double>*>(v)[i];
      reinterpret_cast<cx<df>*>(v)[i] = mk(df(a.re), df(a.im));
    } else {
      const cx<df> a = reinterpret_cast<cx<df>*>(v)[i];
      reinterpret_cast<cx<double>*>(v)[i] = mk((double)a.re, (double)a.im);
    }
  }
}
template <bool TO_DF>
static bool convert_volume(void* v, size_t n, cudaStream_t st) {
  if (n == 0) return true;
  const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 8);
  KTimer kt(K_MISC, st);
  convert_volume_kernel<TO_DF><<<grid, 256, 0, st>>>(v, n);
  kt.done();
  return launch_ok("convert_volume_kernel");
}

// Whether scale j of a plan runs its FFTs in double-float: FP64 plans, real signals, rotated
// coefficients, the lengths P = 4096 and 2048 (band limits 513..1024 and 257..512), with the FP64
// tables split at creation.
static bool df_scale(const crv_plan_s* p, int j) {
  const int P = p->fft.at(p->Lj[j]).x.P;
  return p->df_fft && p->real && !p->unrot && (P == 4096 || P == 2048);
}

// The FFT steps of the analysis of scale j in double-float (real signals, P = 4096 or 2048): the steps
// of the FP64 path (beta synthesis, the m step on the n >= 0 columns, the n step with real output
// in row pairs) on the kernels compiled in df_fft.cu and df_fft2048.cu.
static bool analysis_ffts_df(crv_plan_s* p, int j, double* W, cudaStream_t st) {
  const int Lb = p->Lj[j], N = 2 * Lb - 1;
  const DftTab<df>& tb = p->fft.at(Lb).x;
  const ColSet cs = p->colset(Lb);
  cx<df>* X = (cx<df>*)p->wX;
  cx<df>* Xb = (cx<df>*)p->wXb;
  cx<df>* R = (cx<df>*)p->wR;
  if (!df_beta_synth(tb, Lb, (int)cs.pitch(), X, Xb, cs, st)) return false;
  const int Rr = ring_chunk(p, Lb, sizeof(cx<df>));
  const size_t wstride = (size_t)N * N;
  const int ni0 = -cs.n0 / cs.nstep, Nh = cs.Nc - ni0, npair = (N + 1) / 2;
  for (int b0 = 0; b0 < Lb; b0 += Rr) {
    const int nr = std::min(Rr, Lb - b0);
    if (Nh > 0) {
      LdRingMHalf<df, false> lm{Xb + (size_t)b0 * cs.pitch(), cs, ni0, N, Nh, FastDiv((uint32_t)Nh), 0};
      StRingMHalf<df> sm{R, N, Nh, FastDiv((uint32_t)Nh), Nh, 0};
      if (!df_ring_m(tb, nr * Nh, lm, sm, st)) return false;
    }
    LdRingNHerm<df, false> ln{R, N, Nh, cs.nstep, npair, FastDiv((uint32_t)npair), 0};
    StWRowPair<df, double> sw{W + (size_t)b0 * wstride, N, npair, FastDiv((uint32_t)npair)};
    if (!df_ring_n(tb, nr * npair, ln, sw, st)) return false;
  }
  return true;
}

// The FFT steps of the synthesis of scale j in double-float (real signals, P = 4096 or 2048): g step on
// real row pairs, a step on the n >= 0 columns, beta quadrature into the Y planes.
static bool synthesis_ffts_df(crv_plan_s* p, int j, const double* W, cudaStream_t st) {
  const int Lb = p->Lj[j], N = 2 * Lb - 1;
  const FftSet& fs = p->fft.at(Lb);
  const DftTab<df>& tb = fs.x;
  const ColSet cs = p->colset(Lb);
  cx<df>* Y = (cx<df>*)p->wX;
  cx<df>* Xb = (cx<df>*)p->wXb;
  cx<df>* R = (cx<df>*)p->wR;
  const int Rr = ring_chunk(p, Lb, sizeof(cx<df>));
  const size_t wstride = (size_t)N * N;
  const int ni0 = -cs.n0 / cs.nstep, Nh = cs.Nc - ni0;
  const df inv = df(1.0 / N);
  for (int b0 = 0; b0 < Lb; b0 += Rr) {
    const int nr = std::min(Rr, Lb - b0), nrows = nr * N;
    LdWRowPair<df, double> lw{W + (size_t)b0 * wstride, N, nrows};
    StRingNPairHalf<df> sn{R, Nh, cs.nstep, N, nrows, inv, 0};
    if (!df_ring_g(tb, (nrows + 1) / 2, lw, sn, st)) return false;
    if (Nh > 0) {
      LdRingAHalf<df> la{R, N, Nh, FastDiv((uint32_t)Nh), Nh, 0};
      StRingAHalf<df> sa{Xb + (size_t)b0 * cs.pitch(), cs, ni0, N, Nh, inv, FastDiv((uint32_t)Nh), 0};
      if (!df_ring_a(tb, nr * Nh, la, sa, st)) return false;
    }
  }
  return df_beta_quad(tb, fs.cx2, Lb, (int)cs.pitch(), Xb, Y, cs, df(4 * M_PI * M_PI), 1, -1, 0, st);
}

template <class T, class OutT>
static bool wigner_analysis_scale(crv_plan_s* p, int j, const cx<double>* flm, OutT* W, cudaStream_t st) {
  NvtxRange nv("analysis scale", j);
  const int Lb = p->Lj[j], N = 2 * Lb - 1;
  const FftSet& fs = p->fft.at(Lb);
  ColSet cs = p->colset(Lb);
  cx<T>* X = (cx<T>*)p->wX;
  cx<T>* Xb = (cx<T>*)p->wXb;
  cx<T>* R = (cx<T>*)p->wR;
  bool used_tc = false;
  if constexpr (sizeof(T) == 8) {
    if (p->use_oz) {
      const crv_plan_s::OzA& a = p->ozAA[j];
      for (int i = 0; i + 1 < (int)a.cuts.size(); ++i)
        if (!oz_analysis(p->dQ, p->L, flm, oz_pass(p, a, i), p->ozBA[j], Lb, cs, (cx<double>*)X, p->d_err,
                         p->d_err + 1, st))
          return false;
      used_tc = true;
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (p->use_tc) {
      if (!tc_analysis(p->dQ32, p->L, p->wflm32, p->tabA[j], Lb, cs, (cx<float>*)X, p->d_err, p->d_err + 1, st,
                       p->tabAA[j]))
        return false;
      used_tc = true;
    }
  }
  if (p->unrot) {
    constexpr int MPB = UnrotPlanes<T>::value;
    dim3 g((cs.Nc + UA_N - 1) / UA_N, ((cs.Mc + 1) / 2 + UA_PAIRS - 1) / UA_PAIRS, (Lb + MPB - 1) / MPB);
    KTimer kt(K_CONTRACT_A, st);
    unrot_analysis_kernel<T><<<g, 256, 0, st>>>(q_of<T>(p), p->L, flm, psi_of<T>(p, j), Lb, cs, p->nlo[j], X);
    kt.done();
    if (!launch_ok("unrot_analysis_kernel")) return false;
  } else if (!used_tc) {
    dim3 g((cs.Nc + 63) / 64, (cs.Mc + 31) / 32, Lb);
    KTimer kt(K_CONTRACT_A, st);
    contract_analysis_kernel<T><<<g, 256, 0, st>>>(q_of<T>(p), p->L, flm, psi_of<T>(p, j), Lb, cs, X);
    kt.done();
    if (!launch_ok("contract_analysis_kernel")) return false;
  }
  if constexpr (sizeof(T) == 8 && std::is_same<OutT, double>::value) {
    if (df_scale(p, j)) {  // X into double-float in place, then the FFTs on the FP32 pipe
      if (!convert_volume<true>(p->wX, (size_t)Lb * cs.pitch(), st)) return false;
      return analysis_ffts_df(p, j, W, st);
    }
  }
  const int ncols = (int)cs.pitch();
  const PairMap pm = p->unrot ? PairMap{p->dpmap[j], p->npmap[j]} : PairMap();
  if (!run_beta_synth<T>(dft_of<T>(fs), Lb, ncols, X, Xb, cs, K_BETA_SYNTH, st, pm)) return false;
  const int Rr = ring_chunk(p, Lb, sizeof(cx<T>));
  const size_t wstride = (size_t)N * N * (p->real ? 1 : 2);
  const int ni0 = -cs.n0 / cs.nstep, Nh = cs.Nc - ni0;  // columns n >= 0
  // unrotated plans: columns |n| < nlo are zero, so the ring steps skip them (nstep = 1 there)
  const int nlo = p->unrot ? p->nlo[j] : 0, h0 = std::min(nlo, Nh);
  for (int b0 = 0; b0 < Lb; b0 += Rr) {
    const int nr = std::min(Rr, Lb - b0);
    const bool ok = p->unrot ? ring_inverse<T, OutT, true>(p, fs, cs, Xb, R, W, b0, nr, N, ni0, Nh, h0, nlo, wstride, st)
                             : ring_inverse<T, OutT, false>(p, fs, cs, Xb, R, W, b0, nr, N, ni0, Nh, h0, nlo, wstride, st);
    if (!ok) return false;
  }
  return true;
}

template <class T, class InT>
static bool wigner_synthesis_scale(crv_plan_s* p, int j, const InT* W, cx<double>* flm, cudaStream_t st) {
  NvtxRange nv("synthesis scale", j);
  const int Lb = p->Lj[j], N = 2 * Lb - 1;
  const FftSet& fs = p->fft.at(Lb);
  ColSet cs = p->colset(Lb);
  cx<T>* Y = (cx<T>*)p->wX;
  cx<T>* Xb = (cx<T>*)p->wXb;
  cx<T>* R = (cx<T>*)p->wR;
  const int Rr = ring_chunk(p, Lb, sizeof(cx<T>));
  const size_t wstride = (size_t)N * N * (p->real ? 1 : 2);
  const int ni0 = -cs.n0 / cs.nstep, Nh = cs.Nc - ni0;  // columns n >= 0
  // unrotated plans: only the columns |n| >= nlo are needed downstream
  const int nlo = p->unrot ? p->nlo[j] : 0, h0 = std::min(nlo, Nh), Nhs = Nh - h0;
  bool df_done = false;
  if constexpr (sizeof(T) == 8 && std::is_same<InT, double>::value) {
    if (df_scale(p, j)) {  // the FFTs on the FP32 pipe, then Y back to FP64 in place
      if (!synthesis_ffts_df(p, j, W, st)) return false;
      if (!convert_volume<false>(p->wX, (size_t)Lb * cs.pitch(), st)) return false;
      df_done = true;
    }
  }
  for (int b0 = 0; b0 < Lb && !df_done; b0 += Rr) {
    const int nr = std::min(Rr, Lb - b0);
    if (p->real) {
      // g step on real rows in pairs keeping n >= 0, then the a step on those columns,
      // which also fills the n < 0 columns by conjugation
      const int nrows = nr * N;
      LdWRowPair<T, InT> lw{W + (size_t)b0 * wstride, N, nrows};
      StRingNPairHalf<T> sn{R, Nh, cs.nstep, N, nrows, (T)1 / (T)N, h0};
      if (!run_rows<T>(K_RING_FWD_G, dft_of<T>(fs), -1, (nrows + 1) / 2, lw, sn, st)) return false;
      if (Nhs > 0) {
        LdRingAHalf<T> la{R, N, Nhs, FastDiv((uint32_t)Nhs), Nh, h0};
        StRingAHalf<T> sa{Xb + (size_t)b0 * cs.pitch(), cs, ni0, N, Nhs, (T)1 / (T)N, FastDiv((uint32_t)Nhs), h0};
        if (!run_cols<T>(K_RING_FWD_A, dft_of<T>(fs), -1, nr * Nhs, la, sa, st)) return false;
      }
    } else {
      LdWRow<T, InT> lw{W + (size_t)b0 * wstride, N, false};
      StRingN<T> sn{R, cs.Nc, cs.n0, cs.nstep, N, (T)1 / (T)N};
      if (!run_rows<T>(K_RING_FWD_G, dft_of<T>(fs), -1, nr * N, lw, sn, st)) return false;
      LdRingA<T> la{R, cs.Nc, N, FastDiv((uint32_t)cs.Nc)};
      StRingA<T> sa{Xb + (size_t)b0 * cs.pitch(), cs, N, (T)1 / (T)N};
      if (!run_cols<T>(K_RING_FWD_A, dft_of<T>(fs), -1, nr * cs.Nc, la, sa, st)) return false;
    }
  }
  const int ncols = (int)cs.pitch();
  const PairMap pm = p->unrot ? PairMap{p->dpmap[j], p->npmap[j]} : PairMap();
  if (!df_done && !run_beta_quad<T>(fs, Lb, ncols, Xb, Y, cs, (T)(4 * M_PI * M_PI), 1, -1, 0, st, pm)) return false;
  if (p->unrot) {
    // Xb is consumed by the beta quadrature: its buffer holds the per-chunk sums
    const int nchunk = (Lb + US_MPC - 1) / US_MPC;
    cx<double>* P = (cx<double>*)p->wXb;
    dim3 g((Lb + US_L - 1) / US_L, ((cs.Mc + 1) / 2 + US_PAIRS - 1) / US_PAIRS, nchunk);
    KTimer kt(K_CONTRACT_S, st);
    unrot_synthesis_kernel<T><<<g, 256, 0, st>>>(q_of<T>(p), p->L, Y, psi_of<T>(p, j), Lb, cs, nlo, P);
    if (!launch_ok("unrot_synthesis_kernel")) return false;
    unrot_reduce_kernel<<<(Lb * Lb + 255) / 256, 256, 0, st>>>(P, nchunk, Lb, cs.m0, flm);
    count_launch();  // the timer counts the first of its two launches
    kt.done();
    return launch_ok("unrot_reduce_kernel");
  }
  if constexpr (sizeof(T) == 8) {
    // Xb is consumed by the beta quadrature, so its buffer holds the per-m' products
    if (p->use_oz) {
      const crv_plan_s::OzA& a = p->ozAS[j];
      cx<double>* Z = (cx<double>*)p->wXb;
      for (int i = 0; i + 1 < (int)a.cuts.size(); ++i)
        if (!oz_synthesis_products((const cx<double>*)Y, oz_pass(p, a, i), p->ozBS[j], Lb, cs, Z, p->d_err,
                                   p->d_err + 1, st))
          return false;
      return oz_synthesis_reduce(p->dQ, p->L, Z, Lb, cs, flm, st);
    }
  }
  if constexpr (sizeof(T) == 4) {
    // Xb is consumed by the beta quadrature, so its buffer holds the per-m' products
    if (p->use_tc)
      return tc_synthesis(p->dQ32, p->L, (const cx<float>*)Y, p->tabS[j], Lb, cs, (cx<float>*)p->wXb, flm, p->d_err,
                          p->d_err + 1,
                          st);
  }
  const int mchunk = 16;
  dim3 g((Lb + 31) / 32, (cs.Mc + 31) / 32, (Lb + mchunk - 1) / mchunk);
  KTimer kt(K_CONTRACT_S, st);
  contract_synthesis_kernel<T><<<g, 256, 0, st>>>(q_of<T>(p), p->L, Y, psi_of<T>(p, j), Lb, cs, mchunk, flm);
  kt.done();
  return launch_ok("contract_synthesis_kernel");
}

template <class T, class WT>
static bool analysis_from_flm(crv_plan_s* p, const cx<double>* flm, void* const* W, size_t bidx, double* Wphi,
                              cudaStream_t st) {
  if (p->use_tc) {
    const int n = p->L * p->L;
    KTimer kt(K_MISC, st);
    cast_flm_kernel<float><<<(n + 255) / 256, 256, 0, st>>>(flm, p->wflm32, n);
    kt.done();
    if (!launch_ok("cast_flm_kernel")) return false;
  }
  for (int j = p->J0; j <= p->J; ++j) {
    const int Lb = p->Lj[j], N = 2 * Lb - 1;
    const size_t we = (size_t)Lb * N * N * (p->real ? 1 : 2);
    if (!W[j]) { g_err = "W[j] is NULL for a computed scale"; return false; }
    if (!wigner_analysis_scale<T, WT>(p, j, flm, (WT*)W[j] + bidx * we, st)) return false;
  }
  if (Wphi) {
    const int Lp = p->Lphi;
    KTimer kt(K_MISC, st);
    scaling_apply_kernel<<<(Lp * Lp + 255) / 256, 256, 0, st>>>(p->dphi, Lp, flm, p->wflm2, false);
    kt.done();
    if (!launch_ok("scaling_apply_kernel")) return false;
    const size_t pe = (size_t)Lp * (2 * Lp - 1) * (p->real ? 1 : 2);
    if (!sht_inverse(p, p->wflm2, Wphi + bidx * pe, Lp, 0, p->real, st)) return false;
  }
  return true;
}

template <class T, class WT>
static bool synthesis_to_flm(crv_plan_s* p, const void* const* W, size_t bidx, const double* Wphi, cx<double>* flm,
                             cudaStream_t st) {
  cudaMemsetAsync(flm, 0, sizeof(cx<double>) * p->L * p->L, st);
  for (int j = p->J0; j <= p->J; ++j) {
    const int Lb = p->Lj[j], N = 2 * Lb - 1;
    const size_t we = (size_t)Lb * N * N * (p->real ? 1 : 2);
    if (!W[j]) { g_err = "W[j] is NULL for a computed scale"; return false; }
    if (!wigner_synthesis_scale<T, WT>(p, j, (const WT*)W[j] + bidx * we, flm, st)) return false;
  }
  if (Wphi) {
    const int Lp = p->Lphi;
    const size_t pe = (size_t)Lp * (2 * Lp - 1) * (p->real ? 1 : 2);
    if (!sht_forward(p, Wphi + bidx * pe, p->wflm2, Lp, 0, p->real, st)) return false;
    KTimer kt(K_MISC, st);
    scaling_apply_kernel<<<(Lp * Lp + 255) / 256, 256, 0, st>>>(p->dphi, Lp, p->wflm2, flm, true);
    kt.done();
    if (!launch_ok("scaling_apply_kernel")) return false;
  }
  KTimer kt(K_MISC, st);
  flm_finish_kernel<<<(p->L * p->L + 255) / 256, 256, 0, st>>>(flm, p->L, p->spin, p->real);
  kt.done();
  return launch_ok("flm_finish_kernel");
}

// precision dispatch
static bool do_analysis(crv_plan_s* p, const cx<double>* flm, void* const* W, size_t b, double* Wphi, cudaStream_t st) {
  if (p->mixed) return p->wfp32 ? analysis_from_flm<float, float>(p, flm, W, b, Wphi, st)
                                : analysis_from_flm<float, double>(p, flm, W, b, Wphi, st);
  return p->wfp32 ? analysis_from_flm<double, float>(p, flm, W, b, Wphi, st)
                  : analysis_from_flm<double, double>(p, flm, W, b, Wphi, st);
}
static bool do_synthesis(crv_plan_s* p, const void* const* W, size_t b, const double* Wphi, cx<double>* flm,
                         cudaStream_t st) {
  if (p->mixed) return p->wfp32 ? synthesis_to_flm<float, float>(p, W, b, Wphi, flm, st)
                                : synthesis_to_flm<float, double>(p, W, b, Wphi, flm, st);
  return p->wfp32 ? synthesis_to_flm<double, float>(p, W, b, Wphi, flm, st)
                  : synthesis_to_flm<double, double>(p, W, b, Wphi, flm, st);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* crv_last_error(void) { return g_err.c_str(); }

const char* crv_status_string(int s) {
  switch (s) {
    case CRV_OK: return "CRV_OK";
    case CRV_EINVAL: return "CRV_EINVAL";
    case CRV_ENOMEM: return "CRV_ENOMEM";
    case CRV_ECUDA: return "CRV_ECUDA";
    case CRV_ETIMEOUT: return "CRV_ETIMEOUT";
    case CRV_EUNSUPPORTED: return "CRV_EUNSUPPORTED";
    case CRV_EGUARD: return "CRV_EGUARD";
    default: return "unknown status";
  }
}

unsigned long long crv_launch_count(void) { return g_launches.load(); }

int crv_profile_enable(unsigned kind_mask) {
  std::lock_guard<std::mutex> g(g_prof.mu);
  g_prof.mask.store(kind_mask);
  return CRV_OK;
}
int crv_profile_num_kinds(void) { return K_NKINDS; }
const char* crv_profile_kind_name(int k) { return kind_name(k); }
int crv_profile_read(int k, unsigned long long* launches, double* total_ms) {
  if (k < 0 || k >= K_NKINDS) return fail(CRV_EINVAL, "kind out of range");
  std::lock_guard<std::mutex> g(g_prof.mu);
  g_prof.drain(g_prof.pending.size());
  if (launches) *launches = g_prof.launches[k];
  if (total_ms) *total_ms = g_prof.ms[k];
  return CRV_OK;
}
int crv_profile_reset(void) {
  std::lock_guard<std::mutex> g(g_prof.mu);
  g_prof.drain(g_prof.pending.size());
  for (int k = 0; k < K_NKINDS; ++k) { g_prof.launches[k] = 0; g_prof.ms[k] = 0; }
  return CRV_OK;
}

// B operand tables of the tensor-core contractions, per scale (Delta Psi in the engine's
// tile layout; see tc_contract.cuh).
static int build_tc_tables(crv_plan_s* p, cudaStream_t st) {
  int stt = CRV_OK;
  p->tabA.assign(p->J + 1, TcTab());
  p->tabS.assign(p->J + 1, TcTab());
  for (int j = p->J0; j <= p->J; ++j) {
    const int Lb = p->Lj[j];
    const ColSet cs = p->colset(Lb);
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<int2> range;
      int ntiles = 0;
      if (dir == 0) tc_analysis_ranges(Lb, p->nlo[j], cs, range, ntiles);
      else tc_synthesis_ranges(Lb, p->nlo[j], cs, range, ntiles);
      std::vector<long long> base(range.size());
      long long total = 0;
      for (size_t i = 0; i < range.size(); ++i) {
        base[i] = total - range[i].x;
        total += range[i].y;
      }
      const size_t nf = (size_t)std::max<long long>(total, 1) * TC_CHUNK_FLOATS;
      float* hi = p->talloc<float>(nf, &stt);
      float* lo = p->talloc<float>(nf, &stt);
      long long* dbase = p->talloc<long long>(base.size(), &stt);
      int2* drange = p->talloc<int2>(range.size(), &stt);
      if (stt != CRV_OK) return stt;
      cudaMemcpy(dbase, base.data(), base.size() * sizeof(long long), cudaMemcpyHostToDevice);
      cudaMemcpy(drange, range.data(), range.size() * sizeof(int2), cudaMemcpyHostToDevice);
      TcTab t;
      t.hi = hi; t.lo = lo; t.base = dbase; t.range = drange; t.ntiles = ntiles;
      for (const int2& r : range) t.kmax = std::max(t.kmax, r.y);
      t.lmin = p->nlo[j];
      const bool ok = dir == 0 ? tc_fill_analysis_table(p->dQ32, p->L, p->dpsi32[j], Lb, cs, t, hi, lo, st)
                               : tc_fill_synthesis_table(p->dQ32, p->L, p->dpsi32[j], Lb, cs, t, hi, lo, st);
      if (!ok) return CRV_ECUDA;
      (dir == 0 ? p->tabA : p->tabS)[j] = t;
    }
  }
  // per-map A tables of the analysis: offsets per scale, one buffer for the largest scale
  p->tabAA.assign(p->J + 1, TcATab());
  long long amax = 0;
  for (int j = p->J0; j <= p->J; ++j) {
    const ColSet cs = p->colset(p->Lj[j]);
    std::vector<int2> range;
    int nmt = 0;
    tc_analysis_a_ranges(p->Lj[j], p->nlo[j], cs, range, nmt);
    std::vector<long long> base(range.size());
    long long total = 0;
    for (size_t i = 0; i < range.size(); ++i) {
      base[i] = total - range[i].x;
      total += range[i].y;
    }
    amax = std::max(amax, total);
    long long* dbase = p->talloc<long long>(base.size(), &stt);
    int2* drange = p->talloc<int2>(range.size(), &stt);
    if (stt != CRV_OK) return stt;
    cudaMemcpy(dbase, base.data(), base.size() * sizeof(long long), cudaMemcpyHostToDevice);
    cudaMemcpy(drange, range.data(), range.size() * sizeof(int2), cudaMemcpyHostToDevice);
    p->tabAA[j].base = dbase;
    p->tabAA[j].range = drange;
    p->tabAA[j].nmt = nmt;
  }
  p->a_chunks = amax;
  if (stt != CRV_OK) return stt;
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(CRV_ECUDA, "contraction table build failed");
  return CRV_OK;
}

// Sliced tables of the FP64 tensor-core contractions (tc_ozaki.cuh): the B tables of every
// scale, filled here, and the layout of the per-map A tables with the passes over m'.
static int build_oz_tables(crv_plan_s* p, cudaStream_t st) {
  int stt = CRV_OK;
  p->ozBA.assign(p->J + 1, OzTab());
  p->ozBS.assign(p->J + 1, OzTab());
  p->ozAA.assign(p->J + 1, crv_plan_s::OzA());
  p->ozAS.assign(p->J + 1, crv_plan_s::OzA());
  auto layout = [](const std::vector<int2>& range, std::vector<long long>& base) {
    base.resize(range.size());
    long long total = 0;
    for (size_t i = 0; i < range.size(); ++i) {
      base[i] = total - range[i].x;
      total += range[i].y;
    }
    return total;
  };
  // A buffer: CRV_FP64_TC_A_GB (default 4) GB, at least the largest single m'
  double gb = 4.0;
  if (const char* e = getenv("CRV_FP64_TC_A_GB")) gb = std::max(0.01, atof(e));
  long long cap = (long long)(gb * (double)(1ull << 30) / ((double)OZ_ACHUNK * sizeof(float)));
  int kmax = 0;  // longest K range: l < L_j (analysis), the n columns (synthesis)
  for (int j = p->J0; j <= p->J; ++j) kmax = std::max(kmax, std::max(p->Lj[j], p->colset(p->Lj[j]).Nc));
  p->oz_bits = kmax <= 1024 ? 7 : 6;
  if (const char* e = getenv("CRV_FP64_TC_BITS"))  // 6 forces the narrower digits (never wider)
    if (atoi(e) == 6) p->oz_bits = 6;
  for (int j = p->J0; j <= p->J && stt == CRV_OK; ++j) {
    const int Lb = p->Lj[j];
    const ColSet cs = p->colset(Lb);
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<int2> range;
      std::vector<long long> base;
      int ntiles = 0;
      if (dir == 0) oz_ranges_b_analysis(Lb, cs, range, ntiles);
      else oz_ranges_b_synthesis(Lb, cs, range, ntiles);
      const long long total = layout(range, base);
      OzTab t;
      t.v = p->talloc<float>((size_t)std::max<long long>(total, 1) * OZ_BCHUNK, &stt);
      t.e = p->talloc<int>((size_t)Lb * ntiles * OZ_BROWS, &stt);
      long long* dbase = p->talloc<long long>(base.size(), &stt);
      int2* drange = p->talloc<int2>(range.size(), &stt);
      if (stt != CRV_OK) return stt;
      cudaMemcpy(dbase, base.data(), base.size() * sizeof(long long), cudaMemcpyHostToDevice);
      cudaMemcpy(drange, range.data(), range.size() * sizeof(int2), cudaMemcpyHostToDevice);
      t.base = dbase; t.range = drange; t.ntiles = ntiles; t.rows = ntiles * OZ_BROWS;
      t.mp0 = 0; t.mp1 = Lb; t.c0 = 0; t.bits = p->oz_bits;
      const bool ok = dir == 0 ? oz_fill_b_analysis(p->dQ, p->L, p->dpsi[j], Lb, cs, t, st)
                               : oz_fill_b_synthesis(p->dQ, p->L, p->dpsi[j], Lb, cs, t, st);
      if (!ok) return CRV_ECUDA;
      (dir == 0 ? p->ozBA : p->ozBS)[j] = t;
      // A layout
      crv_plan_s::OzA& a = (dir == 0 ? p->ozAA : p->ozAS)[j];
      std::vector<int2> ar;
      std::vector<long long> ab;
      if (dir == 0) oz_ranges_a_analysis(Lb, cs, ar, a.ntiles);
      else oz_ranges_a_synthesis(Lb, cs, ar, a.ntiles);
      layout(ar, ab);
      a.cum.assign(Lb + 1, 0);
      for (int mp = 0; mp < Lb; ++mp) {
        long long c = 0;
        for (int t2 = 0; t2 < a.ntiles; ++t2) c += ar[(size_t)mp * a.ntiles + t2].y;
        a.cum[mp + 1] = a.cum[mp] + c;
        cap = std::max(cap, c);
      }
      long long* dab = p->talloc<long long>(ab.size(), &stt);
      int2* dar = p->talloc<int2>(ar.size(), &stt);
      if (stt != CRV_OK) return stt;
      cudaMemcpy(dab, ab.data(), ab.size() * sizeof(long long), cudaMemcpyHostToDevice);
      cudaMemcpy(dar, ar.data(), ar.size() * sizeof(int2), cudaMemcpyHostToDevice);
      a.base = dab;
      a.range = dar;
    }
  }
  // passes: consecutive m' whose A chunks fit in the buffer
  long long used = 0;
  int mpmax = 0;
  for (int j = p->J0; j <= p->J; ++j)
    for (crv_plan_s::OzA* a : {&p->ozAA[j], &p->ozAS[j]}) {
      const int Lb = (int)a->cum.size() - 1;
      a->cuts.assign(1, 0);
      int mp0 = 0;
      for (int mp = 0; mp < Lb; ++mp)
        if (a->cum[mp + 1] - a->cum[mp0] > cap) {
          a->cuts.push_back(mp);
          mpmax = std::max(mpmax, mp - mp0);
          used = std::max(used, a->cum[mp] - a->cum[mp0]);
          mp0 = mp;
        }
      a->cuts.push_back(Lb);
      mpmax = std::max(mpmax, Lb - mp0);
      used = std::max(used, a->cum[Lb] - a->cum[mp0]);
    }
  p->oz_cap = used;
  p->oz_mp_cap = mpmax;
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(CRV_ECUDA, "FP64 tensor-core table build failed");
  return CRV_OK;
}

// Per-instance workspace of a plan whose tables exist: f_lm buffers, SHT rows, the (m, n, m')
// volumes, the ring buffer, the error flag and the per-map A tables of the tensor-core analysis.
static int alloc_workspace(crv_plan_s* p) {
  int stt = CRV_OK;
  const int L = p->L, Mc = p->mc(L), Nc = p->nc(L), N = 2 * L - 1;
  const size_t el = p->mixed ? sizeof(cx<float>) : sizeof(cx<double>);
  p->vol_bytes = (size_t)L * p->colset(L).pitch() * el;  // (m, n) planes with pair-interleaved columns
  p->wflm = p->dalloc<cx<double>>((size_t)L * L, &stt);
  p->wflm2 = p->dalloc<cx<double>>((size_t)L * L, &stt);
  p->wflm32 = p->dalloc<cx<float>>((size_t)L * L, &stt);
  p->wF = p->dalloc<cx<double>>((size_t)L * (2 * L - 1), &stt);
  p->wG = p->dalloc<cx<double>>((size_t)L * (2 * L - 1), &stt);
  p->wX = p->dalloc<unsigned char>(p->vol_bytes, &stt);
  // Xb; in the mixed path it also holds the synthesis products Z[m'][mi][l] (L x Mc x L)
  p->wXb = p->dalloc<unsigned char>(std::max(p->vol_bytes, (size_t)L * Mc * L * el), &stt);
  p->d_err = p->dalloc<int>(2, &stt);
  if (stt == CRV_OK) cudaMemset(p->d_err, 0, 2 * sizeof(int));
  {
    // ring-chunk buffer: at least one ring, at most all rings, 256 MB (larger chunks: fewer
    // launches; measured 48 -> 120 MB monotonically faster)
    const size_t one = (size_t)(N + 1) * std::max(Mc, Nc) * el;
    p->ring_bytes = std::max(one, std::min((size_t)L * one, (size_t)256 << 20));
  }
  p->wR = p->dalloc<unsigned char>(p->ring_bytes, &stt);
  if (p->use_oz && stt == CRV_OK) {
    int rows = 0;
    for (const auto& a : p->ozAA) rows = std::max(rows, a.ntiles * OZ_AROWS);
    for (const auto& a : p->ozAS) rows = std::max(rows, a.ntiles * OZ_AROWS);
    p->oz_av = p->dalloc<float>((size_t)std::max<long long>(p->oz_cap, 1) * OZ_ACHUNK, &stt);
    p->oz_ae = p->dalloc<int>((size_t)std::max(p->oz_mp_cap, 1) * std::max(rows, 1), &stt);
  }
  if (p->use_tc && stt == CRV_OK) {
    const size_t na = (size_t)std::max<long long>(p->a_chunks, 1) * TC_ACHUNK_FLOATS;
    float* ahi = p->dalloc<float>(na, &stt);
    float* alo = p->dalloc<float>(na, &stt);
    for (int j = p->J0; j <= p->J && stt == CRV_OK; ++j) {
      p->tabAA[j].hi = ahi;
      p->tabAA[j].lo = alo;
    }
  }
  return stt;
}

// A second instance of a plan: the same parameters and table pointers (the table set is
// shared by reference count), a workspace of its own, no workers.
static crv_plan_s* clone_instance(const crv_plan_s* src, int* status) {
  auto* p = new crv_plan_s(*src);
  p->allocs.clear();
  p->guards.clear();
  p->bytes = 0;
  p->workers.clear();
  p->wstreams.clear();
  p->wdone.clear();
  p->fork_ev = nullptr;
  p->nworkers = 1;
  p->wflm = p->wflm2 = nullptr;
  p->wflm32 = nullptr;
  p->wF = p->wG = nullptr;
  p->wX = p->wXb = p->wR = nullptr;
  p->d_err = nullptr;
  for (auto& t : p->tabAA) { t.hi = nullptr; t.lo = nullptr; }
  p->oz_av = nullptr;
  p->oz_ae = nullptr;
  *status = alloc_workspace(p);
  if (*status != CRV_OK) { delete p; return nullptr; }
  return p;
}

// n worker instances (clones) with their streams and events; use `use` of the 1 + n workers.
static int add_workers(crv_plan_s* p, int n, int use) {
  int stt = CRV_OK;
  for (int w = 0; w < n && stt == CRV_OK; ++w) {
    crv_plan_s* q = clone_instance(p, &stt);
    if (!q) break;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (st) cudaStreamDestroy(st);
      delete q;
      return fail(CRV_ECUDA, "worker stream or event creation failed");
    }
    p->workers.push_back(q);
    p->wstreams.push_back(st);
    p->wdone.push_back(ev);
  }
  if (stt != CRV_OK) return stt;
  if (!p->fork_ev && cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(CRV_ECUDA, "event creation failed");
  }
  p->nworkers = std::max(1, std::min(use, 1 + (int)p->workers.size()));
  return CRV_OK;
}

// Run per_map(instance, b, stream) for the B maps of a call: map b on worker b mod K, each
// worker's maps in order on its stream; the workers' streams start after the work already
// queued on st and st continues after all of them (events), so the call stays stream-ordered
// (and capturable into a CUDA graph) for the caller.
}  // extern "C"
template <class F>
static int run_maps(crv_plan_s* p, int B, cudaStream_t st, F&& per_map) {
  const int K = std::min(B, p->nworkers);
  if (K <= 1) {
    for (int b = 0; b < B; ++b)
      if (!per_map(p, b, st)) return CRV_ECUDA;
    return CRV_OK;
  }
  if (cudaEventRecord(p->fork_ev, st) != cudaSuccess) return fail(CRV_ECUDA, "fork event record failed");
  int rc = CRV_OK;
  for (int w = 0; w < K; ++w) {
    crv_plan_s* q = w == 0 ? p : p->workers[w - 1];
    cudaStream_t s = w == 0 ? st : p->wstreams[w - 1];
    if (w > 0 && cudaStreamWaitEvent(s, p->fork_ev, 0) != cudaSuccess) return fail(CRV_ECUDA, "fork wait failed");
    for (int b = w; b < B && rc == CRV_OK; b += K)
      if (!per_map(q, b, s)) rc = CRV_ECUDA;
    if (w > 0) cudaEventRecord(p->wdone[w - 1], s);
  }
  for (int w = 1; w < K; ++w) cudaStreamWaitEvent(st, p->wdone[w - 1], 0);
  return rc;
}
extern "C" {

static void set_ring_bytes(crv_plan_s* p, size_t b) {
  p->ring_bytes = b;
  for (crv_plan_s* w : p->workers) w->ring_bytes = b;
}

// Autotuner (CRV_F_TUNE): time an analysis + synthesis of a batch of zero maps (the work of
// every kernel does not depend on the values) for each number of workers (1, 2, 4, 8 up to
// the batch) and ring-chunk size (64 MB and the default 256 MB, where the rings exceed 64 MB),
// and keep the fastest in the plan. The batch and its coefficients are allocated for the run
// and freed after it.
static int tune_plan(crv_plan_s* p, cudaStream_t st) {
  const int B = std::min(p->max_batch, 1 + (int)p->workers.size());
  const int L = p->L;
  const size_t me = (size_t)L * (2 * L - 1) * (p->real ? 1 : 2);
  const size_t wel = p->wfp32 ? sizeof(float) : sizeof(double);
  size_t wtot = 0;
  std::vector<size_t> woff(p->J + 1, 0);
  for (int j = p->J0; j <= p->J; ++j) {
    const size_t N = 2 * (size_t)p->Lj[j] - 1;
    woff[j] = wtot;
    wtot += (size_t)B * p->Lj[j] * N * N * (p->real ? 1 : 2) * wel;
  }
  const size_t pe = (size_t)p->Lphi * (2 * p->Lphi - 1) * (p->real ? 1 : 2);
  void *maps = nullptr, *W = nullptr, *Wphi = nullptr;
  if (cudaMalloc(&maps, 2 * B * me * sizeof(double)) != cudaSuccess || cudaMalloc(&W, std::max<size_t>(wtot, 16)) != cudaSuccess ||
      cudaMalloc(&Wphi, B * pe * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(maps);
    cudaFree(W);
    return fail(CRV_ENOMEM, "autotuner: no device memory for its trial batch");
  }
  cudaMemsetAsync(maps, 0, 2 * B * me * sizeof(double), st);
  std::vector<void*> Wj(p->J + 1, nullptr);
  for (int j = p->J0; j <= p->J; ++j) Wj[j] = (char*)W + woff[j];
  double* out = (double*)maps + B * me;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  std::vector<int> ks;
  for (int k = 1; k <= B; k *= 2) ks.push_back(k);
  std::vector<size_t> rings = {p->ring_bytes};
  const size_t small = (size_t)64 << 20;
  if (p->ring_bytes > small) rings.push_back(small);
  float best = 1e30f;
  int bestk = p->nworkers;
  size_t bestr = p->ring_bytes;
  int rc = CRV_OK;
  for (size_t rb : rings)
    for (int k : ks) {
      p->nworkers = k;
      set_ring_bytes(p, rb);
      float ms = 0;
      for (int rep = 0; rep < 3 && rc == CRV_OK; ++rep) {  // first run warms up
        if (rep == 1) cudaEventRecord(a, st);
        rc = crv_analysis(p, maps, Wj.data(), Wphi, B, st);
        if (rc == CRV_OK) rc = crv_synthesis(p, Wj.data(), Wphi, out, B, st);
      }
      cudaEventRecord(b, st);
      if (rc != CRV_OK || cudaEventSynchronize(b) != cudaSuccess) { rc = rc ? rc : CRV_ECUDA; break; }
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best) { best = ms; bestk = k; bestr = rb; }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(maps);
  cudaFree(W);
  cudaFree(Wphi);
  p->nworkers = bestk;
  set_ring_bytes(p, bestr);
  p->tuned = true;
  return rc;
}

int crv_plan_create(crv_plan_t* out, int L, double lambda, int J0, int spin, int nrule, unsigned flags,
                    int max_batch, void* stream) {
  NvtxRange nv("crv_plan_create");
  if (!out) return fail(CRV_EINVAL, "out is NULL");
  *out = nullptr;
  if (L < 2 || L > 4096) return fail(CRV_EINVAL, "L must be in [2, 4096]");
  if (L > 1024) return fail(CRV_EUNSUPPORTED, "this build's FFT engine supports L <= 1024 (P <= 4096)");
  if (!(lambda > 1.0) || !std::isfinite(lambda)) return fail(CRV_EINVAL, "lambda must be > 1");
  if (J0 < 0) return fail(CRV_EINVAL, "J0 must be >= 0");
  if (std::abs(spin) >= L) return fail(CRV_EINVAL, "|spin| must be < L");
  if (nrule != CRV_NRULE_CURVELET) return fail(CRV_EINVAL, "unknown nrule");
  if (flags & ~127u) return fail(CRV_EINVAL, "unknown flag bits");
  if ((flags & CRV_F_FP64_TC) && (flags & (CRV_F_MIXED | CRV_F_UNROTATED)))
    return fail(CRV_EINVAL, "CRV_F_FP64_TC is a form of the plain FP64 rotated path (no CRV_F_MIXED, CRV_F_UNROTATED)");
  if ((flags & CRV_F_REAL) && spin != 0) return fail(CRV_EINVAL, "CRV_F_REAL requires spin 0");
  if (max_batch < 1) return fail(CRV_EINVAL, "max_batch must be >= 1");
  int J = 0;
  while (std::pow(lambda, J) < L * (1 - 1e-14)) ++J;
  if (J > 64) return fail(CRV_EINVAL, "lambda too close to 1 (more than 64 scales)");
  if (J0 > J) return fail(CRV_EINVAL, "J0 exceeds the largest scale J");
  if (std::pow(lambda, J0) < std::abs(spin) * (1 - 1e-14))
    return fail(CRV_EINVAL, "lambda^J0 < |spin|: vartheta^j = arccos(-s/lambda^j) undefined");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(CRV_EUNSUPPORTED, "no CUDA device");
  }
  cudaStream_t st = (cudaStream_t)stream;
  auto* p = new crv_plan_s();
  p->tabs = std::make_shared<TableSet>();
  p->L = L; p->lambda = lambda; p->J0 = J0; p->J = J; p->spin = spin; p->flags = flags; p->max_batch = max_batch;
  p->real = flags & CRV_F_REAL; p->mixed = flags & CRV_F_MIXED; p->wfp32 = flags & CRV_F_W_FP32;
  p->unrot = flags & CRV_F_UNROTATED;
  p->use_oz = flags & CRV_F_FP64_TC;
  {
    const char* e = getenv("CRV_FP64_FFT");  // "double" keeps every FFT of the FP64 plans in FP64
    p->df_fft = !p->mixed && !(e && std::strcmp(e, "double") == 0);
  }
  p->guard = flags & CRV_F_GUARD;
  p->Lphi = std::max(1, ceil_pow(lambda, J0));
  p->Lphi = std::min(p->Lphi, L);
  p->Lj.assign(J + 1, 0);
  for (int j = J0; j <= J; ++j) p->Lj[j] = std::min(L, ceil_pow(lambda, j + 1));
  // kernels (Sec. II-B)
  KLambda k(lambda);
  p->kappa.assign((size_t)(J + 1) * L, 0.0);
  for (int j = J0; j <= J; ++j)
    for (int l = 0; l < L; ++l) {
      double v = k.diff(l / std::pow(lambda, j + 1), l / std::pow(lambda, j));
      p->kappa[(size_t)j * L + l] = v > 0 ? std::sqrt(v) : 0.0;
    }
  p->phi.assign(L, 0.0);
  for (int l = 0; l < L; ++l) p->phi[l] = std::sqrt(k(l / std::pow(lambda, J0)));
  p->psi.assign(J + 1, {});
  std::vector<double> dp, dm;
  for (int j = J0; j <= J; ++j) {
    const int Lb = p->Lj[j], N = 2 * Lb - 1;
    std::vector<double>& ps = p->psi[j];
    ps.assign((size_t)Lb * N, 0.0);
    const double th = std::acos(-spin / std::pow(lambda, j));
    const double sh = spin == 0 ? std::sqrt(0.5) : std::sin(th / 2), ch = spin == 0 ? std::sqrt(0.5) : std::cos(th / 2);
    for (int l = std::abs(spin); l < Lb; ++l) {
      const double fac = std::sqrt((2.0 * l + 1) / (8 * M_PI * M_PI)) * p->kappa[(size_t)j * L + l];
      if (fac == 0.0) continue;
      if (l == 0) { ps[Lb - 1] = fac / std::sqrt(2.0); continue; }
      if (p->unrot) {
        // zeta~_{l,l} = 1/sqrt2, zeta~_{l,-l} = (-1)^l/sqrt2 (Sec. II-B, delta_{l|m|})
        ps[(size_t)l * N + (l + Lb - 1)] = fac / std::sqrt(2.0);
        ps[(size_t)l * N + (-l + Lb - 1)] = ((l & 1) ? -fac : fac) / std::sqrt(2.0);
        continue;
      }
      // zeta_lk = (d^l_{k,l}(t) + (-1)^l d^l_{k,-l}(t))/sqrt2, d^l_{k,-l} = (-1)^{l-k} d^l_{-k,l}
      edge_row(l, sh, ch, dp);
      for (int kk = -l; kk <= l; ++kk) {
        if (spin == 0 && (kk & 1)) continue;  // exact zeros at vartheta = pi/2
        double dneg = dp[-kk + l] * (((l - kk) & 1) ? -1.0 : 1.0);
        double z = (dp[kk + l] + ((l & 1) ? -dneg : dneg)) / std::sqrt(2.0);
        ps[(size_t)l * N + (kk + Lb - 1)] = fac * z;
      }
    }
  }
  // edge columns d^l_{k,l}(vartheta^j) per scale, for the rotation of Wigner coefficients
  std::vector<std::vector<double>> edge(J + 1);
  for (int j = J0; j <= J; ++j) {
    const int Lb = p->Lj[j], N = 2 * Lb - 1;
    edge[j].assign((size_t)Lb * N, 0.0);
    const double th = std::acos(-spin / std::pow(lambda, j));
    const double sh = spin == 0 ? std::sqrt(0.5) : std::sin(th / 2), ch = spin == 0 ? std::sqrt(0.5) : std::cos(th / 2);
    for (int l = 0; l < Lb; ++l) {
      edge_row(l, sh, ch, dp);
      for (int kk = -l; kk <= l; ++kk) edge[j][(size_t)l * N + (kk + Lb - 1)] = dp[kk + l];
    }
  }
  p->nlo.assign(J + 1, 0);
  for (int j = J0; j <= J; ++j) {
    int l = std::abs(spin);
    while (l < p->Lj[j] && !(p->kappa[(size_t)j * L + l] > 0)) ++l;
    p->nlo[j] = l;
  }
  int stt = CRV_OK;
  if (p->unrot) {
    // column pairs (m, m+1) at n with a nonzero column: |n| >= nlo and min(|m|, |m+1|) <= |n|
    p->dpmap.assign(J + 1, nullptr);
    p->npmap.assign(J + 1, 0);
    for (int j = J0; j <= J && stt == CRV_OK; ++j) {
      const ColSet cs = p->colset(p->Lj[j]);
      std::vector<int> idx;
      for (int i = 0; i < (cs.Mc + 1) / 2; ++i)
        for (int ni = 0; ni < cs.Nc; ++ni) {
          const int m = cs.m0 + 2 * i, an = std::abs(cs.n0 + ni);
          const bool b_ok = 2 * i + 1 < cs.Mc && std::abs(m + 1) <= an;
          if (an >= p->nlo[j] && (std::abs(m) <= an || b_ok)) idx.push_back(i * cs.Nc + ni);
        }
      p->npmap[j] = (int)idx.size();
      p->dpmap[j] = p->talloc<int>(idx.size(), &stt);
      if (stt == CRV_OK && !idx.empty())
        cudaMemcpy(p->dpmap[j], idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
  }
  // device tables
  const size_t n3 = (size_t)L * L * L;
  p->dQ = p->talloc<double>(n3, &stt);
  if (p->mixed) p->dQ32 = p->talloc<float>(n3, &stt);
  p->dpsi.assign(J + 1, nullptr);
  p->dpsi32.assign(J + 1, nullptr);
  for (int j = J0; j <= J && stt == CRV_OK; ++j) {
    const size_t ne = p->psi[j].size();
    p->dpsi[j] = p->talloc<double>(ne, &stt);
    p->dpsi32[j] = p->talloc<float>(ne, &stt);
    if (stt != CRV_OK) break;
    std::vector<float> f32(p->psi[j].begin(), p->psi[j].end());
    cudaMemcpy(p->dpsi[j], p->psi[j].data(), ne * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(p->dpsi32[j], f32.data(), ne * sizeof(float), cudaMemcpyHostToDevice);
  }
  p->dedge.assign(J + 1, nullptr);
  for (int j = J0; j <= J && stt == CRV_OK; ++j) {
    p->dedge[j] = p->talloc<double>(edge[j].size(), &stt);
    if (stt == CRV_OK) cudaMemcpy(p->dedge[j], edge[j].data(), edge[j].size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  p->dphi = p->talloc<double>(L, &stt);
  if (stt == CRV_OK) cudaMemcpy(p->dphi, p->phi.data(), L * sizeof(double), cudaMemcpyHostToDevice);
  // FFT tables for every band limit in use
  std::set<int> lbs = {L, p->Lphi};
  for (int j = J0; j <= J; ++j) lbs.insert(p->Lj[j]);
  for (int lb : lbs)
    if (stt == CRV_OK) stt = build_fft(p, lb);
  {
    const char* e = getenv("CRV_DISABLE_TC");
    p->use_tc = p->mixed && !p->unrot && !(e && e[0] && e[0] != '0');
  }
  if (stt != CRV_OK) { delete p; return stt; }
  // Delta tables
  double* seed_v = nullptr;
  int* seed_e = nullptr;
  if (cudaMalloc(&seed_v, sizeof(double) * (size_t)L * L) != cudaSuccess ||
      cudaMalloc(&seed_e, sizeof(int) * (size_t)L * L) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(seed_v);
    delete p;
    return fail(CRV_ENOMEM, "seed table allocation failed");
  }
  cudaError_t e = build_delta(L, p->dQ, p->dQ32, seed_v, seed_e, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(seed_v);
  cudaFree(seed_e);
  if (e != cudaSuccess) {
    std::string m = std::string("Delta table build failed: ") + cudaGetErrorString(e) + " " + g_err;
    delete p;
    return fail(CRV_ECUDA, m);
  }
  if (p->use_tc) {
    const int rc = build_tc_tables(p, st);
    if (rc != CRV_OK) { delete p; return rc; }
  }
  if (p->use_oz) {
    const int rc = build_oz_tables(p, st);
    if (rc != CRV_OK) { delete p; return rc; }
  }
  stt = alloc_workspace(p);
  if (stt != CRV_OK) { delete p; return stt; }
  // workers for the maps of a call: up to 4 when a batch is allowed and an instance's workspace
  // is at most 1 GB (L <= 256: the band limits whose kernels are too short to fill the GPU one
  // map at a time)
  const int kmax = (flags & CRV_F_TUNE) ? 8 : 4;
  size_t wlimit = (size_t)1 << 30;
  if (const char* e = getenv("CRV_WORKER_MAX_GB")) wlimit = (size_t)(atof(e) * (1 << 30));
  if (max_batch > 1 && p->bytes <= wlimit) {
    stt = add_workers(p, std::min(max_batch, kmax) - 1, std::min(max_batch, 4));
    if (stt != CRV_OK) { delete p; return stt; }
  } else if (max_batch > 1 && !getenv("CRV_WORKER_MAX_GB")) {
    // larger band limits: one worker (two maps at once) when the two workspaces fit in a
    // quarter of the device memory; each map's kernels already fill the GPU, and the second
    // map fills the tails of the first one's launches (measured +3 % at L = 1024)
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && 2 * p->bytes <= tot / 4 && p->bytes <= fr / 2) {
      stt = add_workers(p, 1, 2);
      if (stt != CRV_OK) { delete p; return stt; }
    } else {
      cudaGetLastError();
    }
  }
  if (flags & CRV_F_TUNE) {
    stt = tune_plan(p, st);
    if (stt != CRV_OK) { delete p; return stt; }
  }
  *out = p;
  return CRV_OK;
}

int crv_plan_clone(crv_plan_t* out, crv_plan_t src, void* stream) {
  if (!out) return fail(CRV_EINVAL, "out is NULL");
  *out = nullptr;
  if (!src) return fail(CRV_EINVAL, "source plan is NULL");
  int stt = CRV_OK;
  crv_plan_s* p = clone_instance(src, &stt);
  if (!p) return stt;
  if (src->workers.size() > 0) {
    stt = add_workers(p, (int)src->workers.size(), src->nworkers);
    if (stt != CRV_OK) { delete p; return stt; }
  }
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    delete p;
    return fail(CRV_ECUDA, "stream synchronisation failed");
  }
  *out = p;
  return CRV_OK;
}

int crv_plan_tuning(crv_plan_t p, int* workers, size_t* ring_bytes, int* tuned) {
  if (!p) return fail(CRV_EINVAL, "plan is NULL");
  if (workers) *workers = p->nworkers;
  if (ring_bytes) *ring_bytes = p->ring_bytes;
  if (tuned) *tuned = p->tuned ? 1 : 0;
  return CRV_OK;
}

int crv_plan_bytes(crv_plan_t p, size_t* table_bytes, size_t* workspace_bytes) {
  if (!p) return fail(CRV_EINVAL, "plan is NULL");
  if (table_bytes) *table_bytes = p->tabs ? p->tabs->bytes : 0;
  if (workspace_bytes) {
    size_t w = p->bytes;
    for (crv_plan_s* q : p->workers) w += q->bytes;
    *workspace_bytes = w;
  }
  return CRV_OK;
}

int crv_plan_destroy(crv_plan_t p) {
  if (!p) return CRV_OK;
  cudaDeviceSynchronize();
  delete p;
  return CRV_OK;
}

int crv_plan_info(crv_plan_t p, int* J, int* Lj, size_t* w_elems, int* L_phi, size_t* workspace_bytes) {
  if (!p) return fail(CRV_EINVAL, "plan is NULL");
  if (J) *J = p->J;
  for (int j = 0; j <= p->J; ++j) {
    const int Lb = p->Lj[j];
    if (Lj) Lj[j] = (j >= p->J0) ? Lb : 0;
    if (w_elems) w_elems[j] = (j >= p->J0) ? (size_t)Lb * (2 * Lb - 1) * (2 * Lb - 1) : 0;
  }
  if (L_phi) *L_phi = p->Lphi;
  if (workspace_bytes) {
    size_t w = p->bytes + (p->tabs ? p->tabs->bytes : 0);
    for (crv_plan_s* q : p->workers) w += q->bytes;
    *workspace_bytes = w;
  }
  return CRV_OK;
}

int crv_plan_check(crv_plan_t p) {
  if (!p) return fail(CRV_EINVAL, "plan is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(CRV_ECUDA, cudaGetErrorString(e));
  int any = 0;
  for (size_t w = 0; w <= p->workers.size(); ++w) {
    crv_plan_s* q = w == 0 ? p : p->workers[w - 1];
    int h = 0;
    cudaMemcpy(&h, q->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (h) {
      cudaMemset(q->d_err, 0, sizeof(int));
      any = 1;
    }
  }
  if (any) return fail(CRV_ETIMEOUT, "a bounded device-side wait gave up (results of the affected call are invalid)");
  return CRV_OK;
}

int crv_plan_check_stream(crv_plan_t p, void* stream) {
  if (!p) return fail(CRV_EINVAL, "plan is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int any = 0;
  // the workers' streams were joined into st by the calls, so st orders their flags too
  for (size_t w = 0; w <= p->workers.size(); ++w) {
    crv_plan_s* q = w == 0 ? p : p->workers[w - 1];
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, q->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(CRV_ECUDA, cudaGetErrorString(e));
    if (h) {
      cudaMemsetAsync(q->d_err, 0, sizeof(int), st);
      cudaStreamSynchronize(st);
      any = 1;
    }
  }
  if (any) return fail(CRV_ETIMEOUT, "a bounded device-side wait gave up (results of the affected call are invalid)");
  return CRV_OK;
}

// The guard regions of a plan: its tables', its own workspace's and its workers'.
static std::vector<Guard> all_guards(const crv_plan_s* p) {
  std::vector<Guard> g = p->tabs->guards;
  for (size_t w = 0; w <= p->workers.size(); ++w) {
    const crv_plan_s* q = w == 0 ? p : p->workers[w - 1];
    g.insert(g.end(), q->guards.begin(), q->guards.end());
  }
  return g;
}

int crv_plan_check_guards(crv_plan_t p, int* nbad) {
  if (!p) return fail(CRV_EINVAL, "plan is NULL");
  if (nbad) *nbad = 0;
  if (!p->guard) return fail(CRV_EINVAL, "plan was created without CRV_F_GUARD");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(CRV_ECUDA, cudaGetErrorString(e));
  const std::vector<Guard> g = all_guards(p);
  std::vector<unsigned char> h(kGuardBytes);
  int bad = 0;
  std::string first;
  for (size_t i = 0; i < g.size(); ++i) {
    if (cudaMemcpy(h.data(), g[i].p, kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(CRV_ECUDA, "guard region read failed");
    size_t k = 0;
    while (k < kGuardBytes && h[k] == kGuardByte) ++k;
    if (k < kGuardBytes) {
      if (!bad)
        first = "guard " + std::to_string(i) + " (after a buffer of " + std::to_string(g[i].size) +
                " bytes) changed at byte " + std::to_string(k) + " past the end";
      ++bad;
    }
  }
  if (nbad) *nbad = bad;
  if (bad) return fail(CRV_EGUARD, std::to_string(bad) + " guard region(s) written: " + first);
  return CRV_OK;
}

int crv_debug_check_tc_ranges(int Lb, int lmin_b, int lmin_a, int real, int spin, int unrot, long long* tiles,
                              long long* bad) {
  if (!bad) return fail(CRV_EINVAL, "bad is NULL");
  if (Lb < 1 || Lb > 1024) return fail(CRV_EINVAL, "Lb must be in [1, 1024]");
  if (lmin_b < 0 || lmin_b > Lb || lmin_a < 0 || lmin_a > Lb) return fail(CRV_EINVAL, "lmin must be in [0, Lb]");
  if (real && spin != 0) return fail(CRV_EINVAL, "real signals have spin 0");
  *bad = tc_check_ranges(Lb, lmin_b, lmin_a, colset_for(Lb, real != 0, spin, unrot != 0), tiles);
  return CRV_OK;
}

int crv_debug_poke_guard(crv_plan_t p, int which) {
  if (!p) return fail(CRV_EINVAL, "plan is NULL");
  if (!p->guard) return fail(CRV_EINVAL, "plan was created without CRV_F_GUARD");
  const std::vector<Guard> g = all_guards(p);
  if (which < 0 || which >= (int)g.size()) return fail(CRV_EINVAL, "no such guard region");
  if (cudaMemset(g[which].p + kGuardBytes / 2, 0, 1) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return fail(CRV_ECUDA, "guard poke failed");
  return CRV_OK;
}

int crv_plan_guard_count(crv_plan_t p, int* n) {
  if (!p || !n) return fail(CRV_EINVAL, "null argument");
  *n = p->guard ? (int)all_guards(p).size() : 0;
  return CRV_OK;
}

int crv_debug_bounded_wait(crv_plan_t p, long polls, void* stream) {
  if (!p) return fail(CRV_EINVAL, "plan is NULL");
  if (polls < 1 || polls > 1000000) return fail(CRV_EINVAL, "polls must be in [1, 1e6]");
  return tc_bounded_wait_probe(p->d_err, polls, (cudaStream_t)stream) ? CRV_OK : CRV_ECUDA;
}

int crv_plan_kernel(crv_plan_t p, int j, double* out) {
  if (!p || !out) return fail(CRV_EINVAL, "null argument");
  if (j < p->J0 || j > p->J) return fail(CRV_EINVAL, "scale out of range");
  std::memcpy(out, p->psi[j].data(), p->psi[j].size() * sizeof(double));
  return CRV_OK;
}

int crv_plan_scaling(crv_plan_t p, double* out) {
  if (!p || !out) return fail(CRV_EINVAL, "null argument");
  std::memcpy(out, p->phi.data(), p->phi.size() * sizeof(double));
  return CRV_OK;
}

int crv_plan_delta(crv_plan_t p, int l, double* out) {
  if (!p || !out) return fail(CRV_EINVAL, "null argument");
  if (l < 0 || l >= p->L) return fail(CRV_EINVAL, "l out of range");
  const size_t L = p->L;
  cudaError_t e = cudaMemcpy2D(out, (l + 1) * sizeof(double), p->dQ + (size_t)l * L, L * L * sizeof(double),
                               (l + 1) * sizeof(double), l + 1, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(CRV_ECUDA, cudaGetErrorString(e));
  return CRV_OK;
}

static int check_batch(crv_plan_t p, int B, const void* a, const void* b) {
  if (!p) return fail(CRV_EINVAL, "plan is NULL");
  if (B < 0 || B > p->max_batch) return fail(CRV_EINVAL, "B must be in [0, max_batch]");
  if (B > 0 && (!a || !b)) return fail(CRV_EINVAL, "null data pointer");
  return CRV_OK;
}

static int check_rotate(crv_plan_t p, int j, int B, const void* a, const void* b) {
  const int s = check_batch(p, B, a, b);
  if (s) return s;
  if (j < p->J0 || j > p->J) return fail(CRV_EINVAL, "scale j out of range [J0, J]");
  return CRV_OK;
}

int crv_rotate_wigner(crv_plan_t p, int j, const void* wt, void* w, int B, void* stream) {
  NvtxRange nv("crv_rotate_wigner");
  int s = check_rotate(p, j, B, wt, w);
  if (s) return s;
  const int Lb = p->Lj[j], N = 2 * Lb - 1;
  for (int b = 0; b < B; ++b)
    if (!rotate_wigner_launch(p->dedge[j], Lb, (const cx<double>*)wt + (size_t)b * 2 * Lb * N,
                              (cx<double>*)w + (size_t)b * Lb * N * N, (cudaStream_t)stream))
      return CRV_ECUDA;
  return CRV_OK;
}

int crv_rotate_wigner_adjoint(crv_plan_t p, int j, const void* w, void* wt, int B, void* stream) {
  NvtxRange nv("crv_rotate_wigner_adjoint");
  int s = check_rotate(p, j, B, w, wt);
  if (s) return s;
  const int Lb = p->Lj[j], N = 2 * Lb - 1;
  for (int b = 0; b < B; ++b)
    if (!rotate_wigner_adjoint_launch(p->dedge[j], Lb, (const cx<double>*)w + (size_t)b * Lb * N * N,
                                      (cx<double>*)wt + (size_t)b * 2 * Lb * N, (cudaStream_t)stream))
      return CRV_ECUDA;
  return CRV_OK;
}

int crv_sht_fwd(crv_plan_t p, const void* map, void* flm, int B, void* stream) {
  NvtxRange nv("crv_sht_fwd");
  int s = check_batch(p, B, map, flm);
  if (s) return s;
  const size_t me = (size_t)p->L * (2 * p->L - 1) * (p->real ? 1 : 2);
  return run_maps(p, B, (cudaStream_t)stream, [&](crv_plan_s* q, int b, cudaStream_t st) {
    return sht_forward(q, (const double*)map + b * me, (cx<double>*)flm + (size_t)b * q->L * q->L, q->L, q->spin,
                       q->real, st);
  });
}

int crv_sht_inv(crv_plan_t p, const void* flm, void* map, int B, void* stream) {
  NvtxRange nv("crv_sht_inv");
  int s = check_batch(p, B, flm, map);
  if (s) return s;
  const size_t me = (size_t)p->L * (2 * p->L - 1) * (p->real ? 1 : 2);
  return run_maps(p, B, (cudaStream_t)stream, [&](crv_plan_s* q, int b, cudaStream_t st) {
    return sht_inverse(q, (const cx<double>*)flm + (size_t)b * q->L * q->L, (double*)map + b * me, q->L, q->spin,
                       q->real, st);
  });
}

int crv_analysis_lm(crv_plan_t p, const void* flm, void* const* W, void* Wphi, int B, void* stream) {
  NvtxRange nv("crv_analysis_lm");
  int s = check_batch(p, B, flm, W);
  if (s) return s;
  return run_maps(p, B, (cudaStream_t)stream, [&](crv_plan_s* q, int b, cudaStream_t st) {
    return do_analysis(q, (const cx<double>*)flm + (size_t)b * q->L * q->L, W, b, (double*)Wphi, st);
  });
}

int crv_analysis(crv_plan_t p, const void* map, void* const* W, void* Wphi, int B, void* stream) {
  NvtxRange nv("crv_analysis");
  int s = check_batch(p, B, map, W);
  if (s) return s;
  const size_t me = (size_t)p->L * (2 * p->L - 1) * (p->real ? 1 : 2);
  return run_maps(p, B, (cudaStream_t)stream, [&](crv_plan_s* q, int b, cudaStream_t st) {
    return sht_forward(q, (const double*)map + b * me, q->wflm, q->L, q->spin, q->real, st) &&
           do_analysis(q, q->wflm, W, b, (double*)Wphi, st);
  });
}

int crv_synthesis_lm(crv_plan_t p, const void* const* W, const void* Wphi, void* flm, int B, void* stream) {
  NvtxRange nv("crv_synthesis_lm");
  int s = check_batch(p, B, W, flm);
  if (s) return s;
  return run_maps(p, B, (cudaStream_t)stream, [&](crv_plan_s* q, int b, cudaStream_t st) {
    return do_synthesis(q, W, b, (const double*)Wphi, (cx<double>*)flm + (size_t)b * q->L * q->L, st);
  });
}

int crv_synthesis(crv_plan_t p, const void* const* W, const void* Wphi, void* map, int B, void* stream) {
  NvtxRange nv("crv_synthesis");
  int s = check_batch(p, B, W, map);
  if (s) return s;
  const size_t me = (size_t)p->L * (2 * p->L - 1) * (p->real ? 1 : 2);
  return run_maps(p, B, (cudaStream_t)stream, [&](crv_plan_s* q, int b, cudaStream_t st) {
    return do_synthesis(q, W, b, (const double*)Wphi, q->wflm, st) &&
           sht_inverse(q, q->wflm, (double*)map + b * me, q->L, q->spin, q->real, st);
  });
}

}  // extern "C"
