// tcgen05 split-FP32 GEMM engine (sm_103a) of the Delta contractions of the mixed path.
//
// D[128 x BN] = sum_k A[128 x k] B[BN x k]^T with FP32 operands produced on the fly by a
// problem object or copied from pre-split tables. Each operand x is split into TF32
// hi = rna(x), lo = rna(x - hi); a K-step issues hi*hi + hi*lo + lo*hi into one FP32 TMEM
// accumulator (split-FP32, ~2^-22 per product), or with Prob::split set the two small
// products into a second accumulator (below). Operand stages sit in shared memory in the
// canonical K-major no-swizzle layout (8-row x 16-byte core matrices); one thread issues
// tcgen05.mma and commits to mbarriers; every wait is bounded and sets an error flag
// instead of hanging; TMEM is drained with tcgen05.ld. Two forms:
//   tc_gemm_kernel     one output tile per CTA, all 256 threads build the operands, two
//                      stages, two CTAs per SM (one's prologue and epilogue overlap the
//                      other's MMAs);
//   tc_gemm_ws_kernel  persistent and warp-specialised, one CTA per SM: operand producers
//                      (or bulk copies of pre-split tables), a copy lane, an MMA lane and
//                      epilogue warps around a four-stage ring and two TMEM accumulators,
//                      tiles taken in order from a global counter.
#pragma once
#include <cstdint>
#include <type_traits>
#include <utility>

#include "transforms.cuh"

namespace crv {
namespace tc {

constexpr int BM = 128, BK = 16, STAGES = 2, NT = 256;
constexpr int A_BYTES = BM * BK * 4;             // 8 KB per A tile (hi or lo)
constexpr int GROUP_BYTES = BK / 4 * 128;       // one 8-row group of core matrices (512 B)
constexpr long kWaitLimit = 1L << 22;            // bounded spin on mbarriers

// Tile geometry for an accumulator of BN columns (BN in {64, 128, 192, 256}).
template <int BN>
struct Geo {
  static constexpr int B_BYTES = BN * BK * 4;                       // B tile (hi or lo)
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 2048;  // + alignment slack and barriers
  static constexpr int TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  // instruction descriptor: D f32, A/B tf32, K-major A and B, N = BN, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(BM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of the 16-byte chunk (row r, k-quad q) in a [rows x BK] tf32 tile:
// core matrix (8 rows x 16 B) at (r/8, q); K-adjacent core matrices 128 B apart,
// 8-row groups GROUP_BYTES apart.
__device__ __forceinline__ uint32_t chunk_off(int r, int q) {
  return (uint32_t)((r >> 3) * GROUP_BYTES + q * 128 + (r & 7) * 16);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;   // leading byte offset: next core matrix along K
  d |= (uint64_t)((uint32_t)GROUP_BYTES >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
  return d;                           // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count = 1) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, long limit = kWaitLimit) {
  for (long it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) atomicExch(err, 1);
  return false;
}
// Arm an mbarrier for one arrival carrying tx bytes of asynchronous copies.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bulk copy global -> shared (16-byte aligned, multiple of 16 bytes) completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// Wait (bounded) until every MMA this thread has issued is complete: one more commit to a
// fresh mbarrier, which tcgen05.commit arms for all prior asynchronous tcgen05 operations of
// the thread. Run by the issuing thread on every exit path, so that TMEM is never
// deallocated under MMAs still in flight (a wait elsewhere may have given up mid-tile).
__device__ __forceinline__ void mma_drain(uint64_t* bar, int* err) {
  mma_commit(bar);
  mbar_wait(bar, 0u, err);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Store four FP32 values as tf32 hi and lo into the (r, q) chunk of the hi and lo tiles.
__device__ __forceinline__ void put4(unsigned char* hi_tile, unsigned char* lo_tile, int r, int q, const float* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = tf32_rna(x[i]);
    l[i] = tf32_rna(x[i] - __uint_as_float(h[i]));
  }
  const uint32_t off = chunk_off(r, q);
  *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ float dq(const float* __restrict__ Q, int Lmax, int a, int l, int b) {
  const int ab = b < 0 ? -b : b;
  float v = __ldg(Q + ((size_t)a * Lmax + l) * Lmax + ab);
  return (b < 0 && ((l + a) & 1)) ? -v : v;
}

// ---------------------------------------------------------------------------
// The GEMM kernel: one 128 x BN output tile per CTA.
//   Prob::tile(bx, by, bz, z, r0, c0, kb, ke) tile coordinates and K range of tile (bx, by, bz)
//   Prob::a4(z, r0, k0, r, q, x[4])           A[r0 + r][k0 + 4q .. +3]
//   Prob::store16(z, r0, c0, r, cc, d[16])    D[r0 + r][c0 + cc .. +15] (all 32 lanes call it)
//   Prob::zero16(z, r0, c0, r, cc)            same for a tile with an empty K range
// and for B either (Prob::kBulkB false)
//   Prob::b4(z, c0, k0, c, q, x[4])           B[c0 + c][k0 + 4q .. +3], split by the threads
// or (Prob::kBulkB true) the stage's B tiles already split and laid out, copied by one thread
// with cp.async.bulk on the stage's full barrier:
//   Prob::b_tiles(z, c0, k0, hi, lo)          device addresses of the hi and lo tiles (B_BYTES each)
// ---------------------------------------------------------------------------
// Prob::kPairLoads: a4 gives, to lane j of each group of four lanes (four
// consecutive rows r = 4p + j), the four rows 4p .. 4p+3 at the one K index 4q + j; the
// producers transpose the group's 4 x 4 values by shuffles (Prob::a_rows then zeroes rows out
// of range) before storing, so that one 16-byte load per lane feeds four rows.
template <class P, class = void> struct PairLoads { static constexpr bool value = false; };
template <class P> struct PairLoads<P, std::enable_if_t<P::kPairLoads>> { static constexpr bool value = true; };
// 4 x 4 transpose within each group of four lanes: lane j holds x[i] = M[i][j] on entry and
// x[i] = M[j][i] on exit. Lane j needs M[j][s] = x_s[j] from lane s. With a[k] = x[(j - k) & 3]
// every round k sends a fixed index: lane j reads a[k] of lane (j + k) & 3, which is
// M[j][(j + k) & 3], and rotating those back by j gives the row.
__device__ __forceinline__ void rot4(float (&x)[4], int by) {  // x[k] <- x[(k - by) & 3]
  float t[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) t[k] = (by & 1) ? x[(k + 3) & 3] : x[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) x[k] = (by & 2) ? t[(k + 2) & 3] : t[k];
}
__device__ __forceinline__ void transpose4(float (&x)[4], int lane) {
  const int j = lane & 3, g = lane & ~3;
  float a[4] = {x[0], x[3], x[2], x[1]};  // a[k] = x[(-k) & 3]
  rot4(a, j);                             // a[k] = x[(j - k) & 3]
  float b[4];
  b[0] = a[0];
#pragma unroll
  for (int k = 1; k < 4; ++k) b[k] = __shfl_sync(0xffffffffu, a[k], g | ((j + k) & 3));
  rot4(b, j);  // b[i] = M[j][i]
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = b[i];
}
template <class P, class = void> struct BulkB { static constexpr bool value = false; };
template <class P> struct BulkB<P, std::enable_if_t<P::kBulkB>> { static constexpr bool value = true; };
// Prob::kBulkA (persistent engine only): the A tiles are also in tables, Prob::a_tiles(z, r0, k0, hi, lo)
template <class P, class = void> struct BulkA { static constexpr bool value = false; };
template <class P> struct BulkA<P, std::enable_if_t<P::kBulkA>> { static constexpr bool value = true; };
// Prob::split: hi*hi and the corrections in separate accumulators (both engine forms)
template <class P, class = void> struct HasSplit { static constexpr bool value = false; };
template <class P> struct HasSplit<P, std::void_t<decltype(std::declval<P>().split)>> {
  static constexpr bool value = true;
};
template <class P> __host__ __device__ __forceinline__ bool split_of(const P& pb) {
  if constexpr (HasSplit<P>::value) return pb.split;
  else return false;
}
template <class Prob, int BN>
__global__ void __launch_bounds__(NT, 2) tc_gemm_kernel(Prob pb, int* err) {
  using G = Geo<BN>;
  constexpr int B_BYTES = G::B_BYTES, STAGE_BYTES = G::STAGE_BYTES;
  extern __shared__ unsigned char smraw[];
  const uint32_t raw = smem_u32(smraw);
  unsigned char* base = smraw + (((raw + 1023u) & ~1023u) - raw);  // 1024-byte aligned stage buffers
  constexpr bool BULK = BulkB<Prob>::value;
  // with Prob::split the corrections go to a second accumulator BN columns on (the launch
  // then keeps one CTA per SM, so that the two CTAs never wait for each other's TMEM)
  const bool SA = split_of(pb);
  const uint32_t TCOLS = SA ? 2 * G::TMEM_COLS : G::TMEM_COLS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);  // MMAs of the stage done
  uint64_t* full = bars + STAGES;                                             // B copies of the stage landed
  uint64_t* drain = full + STAGES;                                            // all MMAs of the CTA done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  const int tid = threadIdx.x, warp = tid >> 5;

  int mp, r0, c0g, kb, ke;
  pb.tile(blockIdx.x, blockIdx.y, blockIdx.z, mp, r0, c0g, kb, ke);
  const int nchunks = (ke > kb) ? (ke - kb + BK - 1) / BK : 0;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&bars[s]);
      mbar_init(&full[s]);
    }
    mbar_init(drain);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  uint32_t pend = 0;      // thread 0: stages with B copies in flight (bit s), issued at chunk pend_c[s]
  int pend_c[STAGES];
  // Operand quads of one K chunk per thread: A 128 rows x BK/4 k-quads, B BN rows x BK/4.
  // The loads of chunk c + 1 are issued as soon as chunk c is in shared memory, so their
  // latency overlaps the barrier and the MMAs of chunk c.
  constexpr int NA = BM * (BK / 4) / NT, NB = BULK ? 1 : BN * (BK / 4) / NT;
  float xa[NA][4], xb[NB][4];
  auto load_chunk = [&](int c) {
    const int k0 = kb + c * BK;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int it = tid + i * NT;
      pb.a4(mp, r0, k0, it % BM, it / BM, xa[i]);
    }
    if constexpr (!BULK) {
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int it = tid + i * NT;
        pb.b4(mp, c0g, k0, it % BN, it / BN, xb[i]);
      }
    }
  };
  // thread 0: bulk copies of chunk c's B tiles into its stage, completing on full[stage]
  auto issue_b = [&](int c) {
    const int sc = c % STAGES;
    unsigned char* stc = base + sc * STAGE_BYTES;
    const void *bhi, *blo;
    pb.b_tiles(mp, c0g, kb + c * BK, bhi, blo);
    mbar_expect_tx(&full[sc], 2u * B_BYTES);
    bulk_g2s(stc + 2 * A_BYTES, bhi, B_BYTES, &full[sc]);
    bulk_g2s(stc + 2 * A_BYTES + B_BYTES, blo, B_BYTES, &full[sc]);
    pend |= 1u << sc;
    pend_c[sc] = c;
  };
  if constexpr (BULK) {
    if (tid == 0 && nchunks > 0) issue_b(0);
  }
  if (nchunks > 0) load_chunk(0);
  for (int c = 0; c < nchunks; ++c) {
    const int s = c % STAGES;
    if (c >= STAGES) ok = mbar_wait(&bars[s], (uint32_t)((c / STAGES) - 1) & 1u, err) && ok;
    unsigned char* st = base + s * STAGE_BYTES;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int it = tid + i * NT;
      if constexpr (PairLoads<Prob>::value) {
        transpose4(xa[i], tid & 31);
        pb.a_rows(r0, it % BM, xa[i]);
      }
      put4(st, st + A_BYTES, it % BM, it / BM, xa[i]);
    }
    if constexpr (!BULK) {
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int it = tid + i * NT;
        put4(st + 2 * A_BYTES, st + 2 * A_BYTES + B_BYTES, it % BN, it / BN, xb[i]);
      }
    }
    if (c + 1 < nchunks) load_chunk(c + 1);
    fence_proxy_async();
    __syncthreads();
    if constexpr (BULK) {
      if (tid == 0 && (pend & (1u << s))) {
        ok = mbar_wait(&full[s], (uint32_t)(c / STAGES) & 1u, err) && ok;
        if (ok) pend &= ~(1u << s);
      }
    }
    if (tid == 0 && ok) {
      fence_after();
      const uint32_t sa = smem_u32(st);
#pragma unroll
      for (int ks = 0; ks < BK / 8; ++ks) {
        const uint32_t koff = ks * 256;  // two core matrices (8 tf32) per K-step
        const uint64_t ahi = smem_desc(sa + koff), alo = smem_desc(sa + A_BYTES + koff);
        const uint64_t bhi = smem_desc(sa + 2 * A_BYTES + koff), blo = smem_desc(sa + 2 * A_BYTES + B_BYTES + koff);
        const uint32_t first = (c == 0 && ks == 0) ? 0u : 1u;
        const uint32_t acc_c = SA ? tmem + (uint32_t)BN : tmem;
        mma_tf32(acc_c, alo, bhi, G::IDESC, first);
        mma_tf32(acc_c, ahi, blo, G::IDESC, 1u);
        mma_tf32(tmem, ahi, bhi, G::IDESC, SA ? first : 1u);
      }
      mma_commit(&bars[s]);
    }
    if constexpr (BULK) {
      // B tiles of chunk c + 1 into the other stage once its MMAs (chunk c - 1) are done, so
      // the copies overlap the next iteration's A build
      if (tid == 0 && ok && c + 1 < nchunks) {
        const int s1 = (c + 1) % STAGES;
        if (c + 1 >= STAGES) ok = mbar_wait(&bars[s1], (uint32_t)(((c + 1) / STAGES) - 1) & 1u, err) && ok;
        if (ok) issue_b(c + 1);
      }
    }
  }
  if (nchunks > 0) {
    const int last = nchunks - 1;
    ok = mbar_wait(&bars[last % STAGES], (uint32_t)(last / STAGES) & 1u, err) && ok;
  }
  if constexpr (BULK) {  // a wait that gave up may leave copies in flight: let them land first
    if (tid == 0)
      for (int s = 0; s < STAGES; ++s)
        if (pend & (1u << s)) mbar_wait(&full[s], (uint32_t)(pend_c[s] / STAGES) & 1u, err);
  }
  if (tid == 0 && nchunks > 0) mma_drain(drain, err);
  fence_after();
  // Epilogue on all warps: warp w reads TMEM lanes 32 (w % 4) .. +31 (the lanes it may
  // access) and the w / 4-th quarter of the BN columns.
  {
    constexpr int QCOLS = BN / (NT / 128);
    const int r = (warp & 3) * 32 + (tid & 31);
    const int cbeg = (warp >> 2) * QCOLS;
    for (int cc = cbeg; cc < cbeg + QCOLS; cc += 16) {
      if (nchunks > 0 && ok) {
        float d[16];
        tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cc, d);
        if (SA) {
          float e[16];
          tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)BN + (uint32_t)cc, e);
#pragma unroll
          for (int i = 0; i < 16; ++i) d[i] += e[i];
        }
        pb.store16(mp, r0, c0g, r, cc, d);
      } else {
        pb.zero16(mp, r0, c0g, r, cc);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised persistent form of the same GEMM (one CTA per SM, 704 threads):
//   warps 0-15 build the A operand of each K chunk (two chunks of loads in flight per
//              thread; four warps per scheduler hide each other's latency) into a ring of
//              WS_STAGES stages and arrive on the stage's a_full;
//              thread 0 also takes the CTA's next tile from a global counter (tiles in the
//              order x fastest, then y, then z, so that the CTAs of the GPU work on
//              neighbouring tiles at any time and share the B chunks and Delta rows in L2)
//              and posts it in a small ring of tile indices;
//   warp 16    (one lane) bulk-copies the pre-split B tiles into the ring, up to
//              WS_STAGES chunks ahead, completing on b_full;
//   warp 17    (one lane) issues the MMAs of a stage once both halves have landed, commits
//              to the stage's empty barrier, and after a tile's last chunk to acc_full;
//   warps 18-21 drain the accumulator of the previous tile (two TMEM accumulators of BN
//              columns alternate), then arrive on acc_empty.
// Prob::split (a run-time flag of problems that have it): the two TMEM regions instead hold
// one tile as a pair, the hi*hi products
// in one and the hi*lo + lo*hi corrections in the other, which the epilogue adds. The
// tensor core's FP32 accumulation behaves like truncation: each MMA step into the running
// sum S loses about half an ulp of S, always towards zero, so the bias grows with the number
// of steps at full magnitude. The corrections are ~2^-11 of S, so in their own accumulator
// their steps cost almost nothing, and the full-size sum takes one step per K-step instead
// of three (a third of the bias, measured on the analysis contraction). The price is that
// the next tile's MMAs wait for the epilogue (one accumulator pair, not two alternating).
// Every mbarrier wait is bounded and made by one lane whose result the warp shares, so
// lanes never disagree; a role whose wait gives up records the error and stops, the others
// then give up in turn, and B copies still in flight are waited for before the CTA exits.
// The producer warps meet at a named barrier once per tile (all of them, on every path).
// With Prob::kBulkA the A tiles come from tables too: warp 0 only schedules tiles, and the
// copy lane fetches A and B of a stage together (PW = 1 producer warp, 224 threads).
// Requires Prob::kBulkB; *ctr must be 0 at launch.
// ---------------------------------------------------------------------------
constexpr int WS_STAGES = 4, WS_TRING = 4;
template <class Prob> struct WsWarps { static constexpr int value = BulkA<Prob>::value ? 1 : 16; };  // producer warps
// K chunks of A whose loads a producer thread keeps in flight ahead of the one it stores
template <class Prob> struct WsPrefetch { static constexpr int value = 4; };
template <int BN> struct GeoWS {
  static constexpr int SMEM_BYTES = WS_STAGES * Geo<BN>::STAGE_BYTES + 1024 + 512;
  static constexpr uint32_t TMEM_COLS = 2 * Geo<BN>::TMEM_COLS;
};

template <int PW> __device__ __forceinline__ void producers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(PW * 32) : "memory");
}
// Bounded wait by lane 0 of the calling warp, result shared with the warp (all lanes call).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* err) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, err) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

template <class Prob, int BN>
__global__ void __launch_bounds__((WsWarps<Prob>::value + 6) * 32, 1)
    tc_gemm_ws_kernel(Prob pb, int gx, int gy, int ntiles, int* ctr, int* err) {
  using G = Geo<BN>;
  constexpr int B_BYTES = G::B_BYTES, STAGE_BYTES = G::STAGE_BYTES, S = WS_STAGES, D = WS_TRING;
  constexpr bool BA = BulkA<Prob>::value;
  const bool SA = split_of(pb);
  constexpr int PW = WsWarps<Prob>::value, WS_WB = PW, WS_WM = PW + 1;
  static_assert(BulkB<Prob>::value, "the B operand comes from tables");
  static_assert(GeoWS<BN>::TMEM_COLS <= 512, "two accumulators fit in TMEM");
  extern __shared__ unsigned char smraw[];
  const uint32_t raw = smem_u32(smraw);
  unsigned char* base = smraw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* a_full = reinterpret_cast<uint64_t*>(base + S * STAGE_BYTES);
  uint64_t* b_full = a_full + S;
  uint64_t* empty = b_full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* tr_full = acc_empty + 2;
  uint64_t* tr_empty = tr_full + D;
  uint64_t* drain = tr_empty + D;  // the MMA issuer's MMAs all done (every exit path)
  int* tring = reinterpret_cast<int*>(drain + 1);
  int* abort_flag = tring + D;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(abort_flag + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&a_full[i], PW);
      mbar_init(&b_full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
    }
    for (int i = 0; i < D; ++i) {
      mbar_init(&tr_full[i], 1);
      mbar_init(&tr_empty[i], 6);  // B producer, MMA issuer, four epilogue warps
    }
    mbar_init(drain);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(GeoWS<BN>::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  // tile t -> coordinates and number of K chunks
  auto tile_of = [&](int t, int& mp, int& r0, int& c0, int& kb, int& nch) {
    int ke;
    pb.tile(t % gx, (t / gx) % gy, t / (gx * gy), mp, r0, c0, kb, ke);
    nch = (ke > kb) ? (ke - kb + BK - 1) / BK : 0;
  };
  // consumers: the j-th tile of this CTA from the ring (every lane of the warp gets it)
  auto next_tile = [&](uint32_t j, int& t) -> bool {
    const int sl = j % D;
    if (!warp_wait(&tr_full[sl], (j / D) & 1u, err)) return false;
    t = tring[sl];
    __syncwarp();
    if (lane == 0) mbar_arrive(&tr_empty[sl]);
    return true;
  };

  if (warp < PW) {
    // ---- A producers: thread tid covers row tid % 128 of the A tile, k-quads q = tid / 128 + j * PQ ----
    constexpr int PQ = BA ? 1 : PW * 32 / BM, NQ = (BK / 4) / PQ;
    static_assert(BA || NQ * PQ == BK / 4, "producer threads tile the stage");
    const int pr = tid % BM, pq = tid / BM;
    uint32_t u = 0;
    for (uint32_t j = 0;; ++j) {
      const int sl = j % D;
      if (tid == 0) {
        int t = ntiles;  // terminal value on any failure
        if (!*abort_flag && mbar_wait(&tr_empty[sl], ((j / D) + 1) & 1u, err)) t = min(atomicAdd(ctr, 1), ntiles);
        else *abort_flag = 1;
        tring[sl] = t;
        mbar_arrive(&tr_full[sl]);
      }
      __syncwarp();
      producers_sync<PW>();
      const int t = tring[sl];  // the same value for every producer thread: all leave together
      if (t >= ntiles) break;
      int mp, r0, c0, kb, nch;
      tile_of(t, mp, r0, c0, kb, nch);
      if (BA) nch = 0;  // A arrives with B
      // the loads of the next PD chunks are in flight while a chunk is split and stored
      constexpr int PD = WsPrefetch<Prob>::value;
      float xs[PD][NQ][4];
#pragma unroll
      for (int d = 0; d < PD; ++d)
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          if (nch > d) pb.a4(mp, r0, kb + d * BK, pr, pq + q * PQ, xs[d][q]);
      for (int c = 0; c < nch; ++c, ++u) {
        float xn[NQ][4];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          if (c + PD < nch) pb.a4(mp, r0, kb + (c + PD) * BK, pr, pq + q * PQ, xn[q]);
        const int s = u % S;
        if (!warp_wait(&empty[s], ((u / S) + 1) & 1u, err)) {
          *abort_flag = 1;
          break;
        }
        unsigned char* st = base + s * STAGE_BYTES;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          if constexpr (PairLoads<Prob>::value) {
            transpose4(xs[0][q], lane);
            pb.a_rows(r0, pr, xs[0][q]);
          }
          put4(st, st + A_BYTES, pr, pq + q * PQ, xs[0][q]);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[s]);
#pragma unroll
        for (int d = 0; d + 1 < PD; ++d)
#pragma unroll
          for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int i = 0; i < 4; ++i) xs[d][q][i] = xs[d + 1][q][i];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int i = 0; i < 4; ++i) xs[PD - 1][q][i] = xn[q][i];
      }
      __syncwarp();
      producers_sync<PW>();  // a failure in any warp (abort_flag) ends the loop at the next tile
    }
  } else if (warp == WS_WB) {
    // ---- B producer ----
    if (lane == 0) {
      uint32_t u = 0;
      int last[S];
      for (int i = 0; i < S; ++i) last[i] = -1;
      bool ok = true;
      for (uint32_t j = 0; ok; ++j) {
        int t;
        const int sl = j % D;
        if (!mbar_wait(&tr_full[sl], (j / D) & 1u, err)) break;
        t = tring[sl];
        mbar_arrive(&tr_empty[sl]);
        if (t >= ntiles) break;
        int mp, r0, c0, kb, nch;
        tile_of(t, mp, r0, c0, kb, nch);
        for (int c = 0; c < nch; ++c, ++u) {
          const int s = u % S;
          if (!mbar_wait(&empty[s], ((u / S) + 1) & 1u, err)) { ok = false; break; }
          unsigned char* st = base + s * STAGE_BYTES;
          const void *bhi, *blo;
          pb.b_tiles(mp, c0, kb + c * BK, bhi, blo);
          if constexpr (BA) {
            const void *ahi, *alo;
            pb.a_tiles(mp, r0, kb + c * BK, ahi, alo);
            mbar_expect_tx(&b_full[s], 2u * (A_BYTES + B_BYTES));
            bulk_g2s(st, ahi, A_BYTES, &b_full[s]);
            bulk_g2s(st + A_BYTES, alo, A_BYTES, &b_full[s]);
          } else {
            mbar_expect_tx(&b_full[s], 2u * B_BYTES);
          }
          bulk_g2s(st + 2 * A_BYTES, bhi, B_BYTES, &b_full[s]);
          bulk_g2s(st + 2 * A_BYTES + B_BYTES, blo, B_BYTES, &b_full[s]);
          last[s] = (int)u;
        }
      }
      // copies issued and possibly not consumed (an error elsewhere) land before exit
      for (int i = 0; i < S; ++i)
        if (last[i] >= 0) mbar_wait(&b_full[i], ((uint32_t)last[i] / S) & 1u, err);
    }
  } else if (warp == WS_WM) {
    // ---- MMA issuer ----
    if (lane == 0) {
      uint32_t u = 0;
      bool ok = true, issued = false;
      for (uint32_t j = 0; ok; ++j) {
        const int sl = j % D;
        if (!mbar_wait(&tr_full[sl], (j / D) & 1u, err)) break;
        const int t = tring[sl];
        mbar_arrive(&tr_empty[sl]);
        if (t >= ntiles) break;
        int mp, r0, c0, kb, nch;
        tile_of(t, mp, r0, c0, kb, nch);
        // the accumulator (pair) of tile j: alternating, or the one pair for every tile
        const uint32_t a = SA ? 0u : (j & 1u), use = SA ? j : (j >> 1);
        if (!mbar_wait(&acc_empty[a], (use + 1) & 1u, err)) break;
        fence_after();
        const uint32_t acc = tmem + a * (uint32_t)BN;
        const uint32_t acc_c = SA ? tmem + (uint32_t)BN : acc;  // where hi*lo and lo*hi go
        for (int c = 0; c < nch; ++c, ++u) {
          const int s = u % S;
          if ((!BA && !mbar_wait(&a_full[s], (u / S) & 1u, err)) || !mbar_wait(&b_full[s], (u / S) & 1u, err)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sa = smem_u32(base + s * STAGE_BYTES);
#pragma unroll
          for (int ks = 0; ks < BK / 8; ++ks) {
            const uint32_t koff = ks * 256;
            const uint64_t ahi = smem_desc(sa + koff), alo = smem_desc(sa + A_BYTES + koff);
            const uint64_t bhi = smem_desc(sa + 2 * A_BYTES + koff), blo = smem_desc(sa + 2 * A_BYTES + B_BYTES + koff);
            const uint32_t first = (c == 0 && ks == 0) ? 0u : 1u;
            mma_tf32(acc_c, alo, bhi, G::IDESC, first);
            mma_tf32(acc_c, ahi, blo, G::IDESC, 1u);
            mma_tf32(acc, ahi, bhi, G::IDESC, SA ? first : 1u);
          }
          issued = true;
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        if (nch > 0) mma_commit(&acc_full[a]);
        else mbar_arrive(&acc_full[a]);
      }
      if (issued) mma_drain(drain, err);
    }
  } else {
    // ---- epilogue: warp w may read TMEM lanes 32 (w % 4) .. + 31 ----
    const int lq = warp & 3, r = lq * 32 + lane;
    for (uint32_t j = 0;; ++j) {
      int t;
      if (!next_tile(j, t) || t >= ntiles) break;
      int mp, r0, c0, kb, nch;
      tile_of(t, mp, r0, c0, kb, nch);
      const uint32_t a = SA ? 0u : (j & 1u), use = SA ? j : (j >> 1);
      if (!warp_wait(&acc_full[a], use & 1u, err)) break;
      fence_after();
      for (int cc = 0; cc < BN; cc += 16) {
        if (nch > 0) {
          float d[16];
          tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + a * (uint32_t)BN + (uint32_t)cc, d);
          if (SA) {
            float e[16];
            tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)BN + (uint32_t)cc, e);
#pragma unroll
            for (int i = 0; i < 16; ++i) d[i] += e[i];
          }
          pb.store16(mp, r0, c0, r, cc, d);
        } else {
          pb.zero16(mp, r0, c0, r, cc);
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[a]);
    }
  }
  __syncwarp();
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GeoWS<BN>::TMEM_COLS)
                 : "memory");
  }
}

}  // namespace tc

template <class Prob, int BN>
bool launch_tc_gemm(const Prob& pb, dim3 grid, int* err, cudaStream_t st, int kind) {
  // a split accumulator takes all of TMEM: more than half of the SM's shared memory keeps a
  // second CTA of the kernel off the SM
  constexpr int smem_split = tc::Geo<BN>::SMEM_BYTES < 120 * 1024 ? 120 * 1024 : tc::Geo<BN>::SMEM_BYTES;
  static_assert(!tc::HasSplit<Prob>::value || 2 * tc::Geo<BN>::TMEM_COLS <= 512, "the pair fits in TMEM");
  const int smem = tc::split_of(pb) ? smem_split : tc::Geo<BN>::SMEM_BYTES;
  if (!func_attr_once((const void*)tc::tc_gemm_kernel<Prob, BN>,
                      tc::HasSplit<Prob>::value ? smem_split : tc::Geo<BN>::SMEM_BYTES))
    return false;
  KTimer kt(kind, st);
  tc::tc_gemm_kernel<Prob, BN><<<grid, tc::NT, smem, st>>>(pb, err);
  kt.done();
  return launch_ok(kind_name(kind));
}

// Persistent warp-specialised launch over the tiles of grid (one CTA per SM at most);
// ctr: a device int, zeroed here on the stream before the launch.
template <class Prob, int BN>
bool launch_tc_gemm_ws(const Prob& pb, dim3 grid, int nsm, int* ctr, int* err, cudaStream_t st, int kind) {
  if (!func_attr_once((const void*)tc::tc_gemm_ws_kernel<Prob, BN>, tc::GeoWS<BN>::SMEM_BYTES)) return false;
  const long long nt = (long long)grid.x * grid.y * grid.z;
  if (nt <= 0) return true;
  if (nt > 0x7fffffffLL) return false;
  const int ctas = (int)std::min<long long>(nt, nsm);
  if (cudaMemsetAsync(ctr, 0, sizeof(int), st) != cudaSuccess) return false;
  KTimer kt(kind, st);
  constexpr int threads = (tc::WsWarps<Prob>::value + 6) * 32;
  tc::tc_gemm_ws_kernel<Prob, BN><<<ctas, threads, tc::GeoWS<BN>::SMEM_BYTES, st>>>(pb, (int)grid.x, (int)grid.y,
                                                                                  (int)nt, ctr, err);
  kt.done();
  return launch_ok(kind_name(kind));
}

}  // namespace crv
