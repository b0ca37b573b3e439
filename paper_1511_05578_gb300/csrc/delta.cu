// Delta^l_{mn} = d^l_mn(pi/2) tables (Sec. III-A-2, the matrices behind the
// factorisation d^l_mn(beta) = i^{n-m} sum_m' Delta^l_{m'm} Delta^l_{m'n} e^{i m' beta}).
//
// Stored as the quarter table Q[m'][l][n] = Delta^l_{m'n} for 0 <= m', n <= l < L
// (dense L^3, zero where l < max(m', n)); the other quadrants follow from
// Delta^l_{-m',n} = (-1)^{l+n} Delta^l_{m'n} and Delta^l_{m',-n} = (-1)^{l+m'} Delta^l_{m'n}.
//
// Recursion (Trapani-Navaza form, FP64):
//   edge row   Delta^l_{l,n} = (-1)^{l-n} 2^{-l} sqrt(C(2l, l+n))
//              (the single surviving term of Eq. wigner_sum_reln at beta = pi/2),
//              built per l by the ratio Delta^l_{l,n+1}/Delta^l_{l,n} = -sqrt((l-n)/(l+n+1))
//              from 2^{-l} sqrt(C(2l,l)) = prod_k sqrt((2k-1)/(2k)), both products as
//              row passes (block-wide scans with warp shuffles);
//   columns    Delta^l_{m,n} = 2n/sqrt((l-m)(l+m+1)) Delta^l_{m+1,n}
//                - sqrt((l-m-1)(l+m+2)/((l-m)(l+m+1))) Delta^l_{m+2,n},  m = l-1 .. 0.
// The edge values reach 2^-l, below the double range past l ~ 1022, so every value
// carries its own binary exponent until it is stored (values that are still below
// the double range then flush to zero, where they contribute nothing).
#include "common.cuh"

namespace crv {

// Products of numbers carried as (mantissa, binary exponent): the edge values fall below the
// double range past l ~ 1022. mul() renormalises, so a product of many factors keeps the
// relative precision of a plain double product.
struct MantExp {
  double m;
  int e;
};
__device__ __forceinline__ MantExp me_mul(MantExp a, MantExp b) {
  int k;
  const double m = frexp(a.m * b.m, &k);
  return MantExp{m, a.e + b.e + k};
}
// Inclusive product scan across the 32 lanes of a warp (row pass by warp shuffles).
__device__ __forceinline__ MantExp warp_scan_mul(MantExp x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double m = __shfl_up_sync(0xffffffffu, x.m, o);
    const int e = __shfl_up_sync(0xffffffffu, x.e, o);
    if (lane >= o) x = me_mul(MantExp{m, e}, x);
  }
  return x;
}
constexpr int kSeedThreads = 256;

// Block per l: the edge row Delta^l_{l,n}, n = 0..l, as (mantissa, exponent). Its magnitude is
// |Delta^l_{l,0}| prod_{k<n} r_k with r_k = sqrt((l-k)/(l+k+1)), and |Delta^l_{l,0}| =
// prod_{k=1..l} sqrt((2k-1)/(2k)) (= 2^-l sqrt(C(2l,l)) >= 0.02 for l < 4096); sign (-1)^{l-n}.
// Both products run as row passes over the block: per 256 values a warp-shuffle scan in each
// warp, the warps' totals scanned by warp 0 through shared memory, and a carry into the next
// 256 values.
__global__ void __launch_bounds__(kSeedThreads) delta_seed_kernel(int L, double* __restrict__ seed_v,
                                                                  int* __restrict__ seed_e) {
  const int l = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NW = kSeedThreads / 32;
  __shared__ MantExp wtot[NW];
  __shared__ MantExp carry;
  // block-wide inclusive scan of x (all threads call); adds the running carry and advances it
  auto block_scan = [&](MantExp x) -> MantExp {
    x = warp_scan_mul(x);
    if (lane == 31) wtot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      MantExp w = lane < NW ? wtot[lane] : MantExp{1.0, 0};
      w = warp_scan_mul(w);
      if (lane < NW) wtot[lane] = w;
    }
    __syncthreads();
    if (wid > 0) x = me_mul(wtot[wid - 1], x);
    x = me_mul(carry, x);
    __syncthreads();
    if (tid == kSeedThreads - 1) carry = x;
    __syncthreads();
    return x;
  };
  // |Delta^l_{l,0}| = prod_{k=1..l} sqrt((2k-1)/(2k)): the carry after the scan is the product
  if (tid == 0) carry = MantExp{1.0, 0};
  __syncthreads();
  for (int k0 = 1; k0 <= l; k0 += kSeedThreads) {
    const int k = k0 + tid;
    MantExp f{1.0, 0};
    if (k <= l) {
      int ke;
      const double m = frexp(sqrt((2.0 * k - 1.0) / (2.0 * k)), &ke);
      f = MantExp{m, ke};
    }
    block_scan(f);
  }
  // |Delta^l_{l,n}| = |Delta^l_{l,0}| prod_{k<n} r_k: inclusive scan of the factors f_n = r_{n-1}
  // (f_0 = 1), starting from the carry |Delta^l_{l,0}|
  for (int n0 = 0; n0 <= l; n0 += kSeedThreads) {
    const int n = n0 + tid, k = n - 1;
    MantExp f{1.0, 0};
    if (k >= 0 && k < l) {
      int ke;
      const double m = frexp(sqrt((double)(l - k) / (double)(l + k + 1)), &ke);
      f = MantExp{m, ke};
    }
    const MantExp v = block_scan(f);
    if (n <= l) {
      seed_v[(size_t)l * L + n] = ((l - n) & 1) ? -v.m : v.m;
      seed_e[(size_t)l * L + n] = v.e;
    }
  }
}

// Block per (l, 128 consecutive n). Writes Q (double) and, if q32 != null, a float copy.
__global__ void __launch_bounds__(128) delta_column_kernel(int L, const double* __restrict__ seed_v,
                                                           const int* __restrict__ seed_e, double* __restrict__ Q,
                                                           float* __restrict__ q32) {
  extern __shared__ double coef[];  // [2*l]: a[m], b[m] for m < l
  const int l = blockIdx.y;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x * blockDim.x > l) return;  // whole block beyond the row
  for (int m = threadIdx.x; m < l; m += blockDim.x) {
    const double den = (double)(l - m) * (double)(l + m + 1);
    const double a = 1.0 / sqrt(den);
    coef[m] = a;
    coef[l + m] = (m + 1 < l) ? sqrt((double)(l - m - 1) * (double)(l + m + 2)) * a : 0.0;
  }
  __syncthreads();
  if (n > l) return;
  const size_t LL = (size_t)L * L;
  double v1 = seed_v[(size_t)l * L + n], v2 = 0.0;  // Delta_{m+1,n}, Delta_{m+2,n}
  int e = seed_e[(size_t)l * L + n];
  auto store = [&](int m, double v) {
    const double t = (e < -2000) ? 0.0 : ldexp(v, e);
    const size_t idx = (size_t)m * LL + (size_t)l * L + n;
    Q[idx] = t;
    if (q32) q32[idx] = (float)t;
  };
  store(l, v1);
  const double twon = 2.0 * n;
  for (int m = l - 1; m >= 0; --m) {
    const double v = twon * coef[m] * v1 - coef[l + m] * v2;
    v2 = v1;
    v1 = v;
    if (fabs(v1) > 0x1p600) {
      v1 = ldexp(v1, -600);
      v2 = ldexp(v2, -600);
      e += 600;
    }
    store(m, v1);
  }
}

cudaError_t build_delta(int L, double* Q, float* q32, double* seed_v, int* seed_e, cudaStream_t st) {
  const size_t n3 = (size_t)L * L * L;
  cudaError_t err = cudaMemsetAsync(Q, 0, n3 * sizeof(double), st);
  if (err != cudaSuccess) return err;
  if (q32) {
    err = cudaMemsetAsync(q32, 0, n3 * sizeof(float), st);
    if (err != cudaSuccess) return err;
  }
  {
    KTimer kt(K_DELTA, st);
    delta_seed_kernel<<<L, kSeedThreads, 0, st>>>(L, seed_v, seed_e);
    kt.done();
  }
  if (!launch_ok("delta_seed_kernel")) return cudaErrorLaunchFailure;
  const size_t smem = sizeof(double) * 2 * (size_t)L;
  if (smem > 48 * 1024) {
    err = cudaFuncSetAttribute(delta_column_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  dim3 grid((L + 127) / 128, L);
  KTimer kt(K_DELTA, st);
  delta_column_kernel<<<grid, 128, smem, st>>>(L, seed_v, seed_e, Q, q32);
  kt.done();
  if (!launch_ok("delta_column_kernel")) return cudaErrorLaunchFailure;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Allocation-free build of the Delta table for callers that cannot allocate
// device memory (see crv_delta_table_noalloc in include/crv.h). The seed row
// scratch lives in file-scope device arrays sized for L <= CRV_NOALLOC_MAX_L;
// every GPU that loads the library holds them (3 MB) until the process exits.
// ---------------------------------------------------------------------------
constexpr int kNoallocMaxL = 512;
static __device__ __align__(256) double g_noalloc_seed_v[kNoallocMaxL * kNoallocMaxL];
static __device__ __align__(256) int g_noalloc_seed_e[kNoallocMaxL * kNoallocMaxL];

}  // namespace crv

#include <mutex>
#include <string>
#include "../../include/crv.h"

namespace crv {
void set_error(const std::string& msg);  // crv.cu: message returned by crv_last_error()
}

namespace {
// Device addresses of the scratch arrays, looked up once per device. Host code must
// not hand the symbols themselves to a kernel: on the host they are stand-ins, not
// device addresses.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_v[kMaxDevices] = {nullptr};
int* g_noalloc_e[kMaxDevices] = {nullptr};
}  // namespace

extern "C" int crv_delta_table_noalloc(int L, double* Q, void* stream) {
  if (L < 1 || L > crv::kNoallocMaxL) {
    crv::set_error("crv_delta_table_noalloc: L must be in [1, " + std::to_string(crv::kNoallocMaxL) + "]");
    return CRV_EINVAL;
  }
  if (!Q) { crv::set_error("crv_delta_table_noalloc: Q is NULL"); return CRV_EINVAL; }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    crv::set_error("crv_delta_table_noalloc: no usable current device");
    return CRV_ECUDA;
  }
  double* sv;
  int* se;
  {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_v[dev]) {
      void* pv = nullptr;
      void* pe = nullptr;
      cudaError_t e1 = cudaGetSymbolAddress(&pv, crv::g_noalloc_seed_v);
      cudaError_t e2 = (e1 == cudaSuccess) ? cudaGetSymbolAddress(&pe, crv::g_noalloc_seed_e) : e1;
      if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        crv::set_error(std::string("crv_delta_table_noalloc: cudaGetSymbolAddress failed: ") +
                       cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        return CRV_ECUDA;
      }
      g_noalloc_v[dev] = (double*)pv;
      g_noalloc_e[dev] = (int*)pe;
    }
    sv = g_noalloc_v[dev];
    se = g_noalloc_e[dev];
  }
  // the seed kernel writes every entry the column kernel reads (n <= l < L), so the
  // scratch needs no clearing; the output table is cleared by build_delta.
  cudaError_t e = crv::build_delta(L, Q, nullptr, sv, se, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    crv::set_error(std::string("crv_delta_table_noalloc: ") + cudaGetErrorString(e));
    return CRV_ECUDA;
  }
  return CRV_OK;
}

