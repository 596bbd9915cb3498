// Reduction GEMMs of the mixed-precision Liouvillian on the 5th-generation tensor
// cores (tcgen05, TF32 operands in shared memory, FP32 accumulators in TMEM).
//
//   C[b][m][n] = sum_k conj(A[b % amod][m][k]) B[b][n][k]        (complex)
//
// used for the Kleinman-Bylander projections <beta|x> (V_NL in Eq. H0_k_plus_q)
// and the occupied-state overlaps <U_kq|h> of P_c (Eqs. P_minus_q2, P_plus_q2).
//
// Complex -> real: with interleaved (re, im) rows, Re C = A_int . B_int and
// Im C = A_rot . B_int where A_rot = (-a.y, a.x) per element, so one real GEMM
// with the 2M rows [A_int; A_rot] against the rows of B gives both parts
// (2M <= 128 = the MMA's M).  The batches that share one A (b = a + j amod) are
// stacked as the N rows of one tile (N <= 256).  For 64 < M <= 128 the roles swap
// (tc_gemm_tnt_kernel): 128 stacked B rows are the MMA's M, the 2M rows its N.
//
// 3xTF32: every FP32 operand x is split into hi = tf32(x) and lo = tf32(x - hi)
// while it is staged into shared memory, and D += Ahi Bhi + Ahi Blo + Alo Bhi
// keeps FP32-level accuracy (the dropped lo*lo term is ~2^-22 relative).
//
// Shared-memory operands use the canonical K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes; the leading byte offset steps between 16-byte
// K chunks, the stride byte offset between 8-row groups.  One CTA per
// (A batch, N tile, K split); a two-stage pipeline overlaps the staging of K tile
// t+1 (global loads, TF32 split) with the MMAs of tile t; the partial sums go to
// a split-K buffer that a second kernel reduces in fixed order.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "engine.cuh"
#include "tc_gemm.cuh"

namespace tdlz {

namespace {

constexpr int kTcThreads = 256;
constexpr int kKT = 16;                      // K tile: 16 reals (8 complex) = 64 bytes per row
constexpr int kChunks = kKT / 4;             // 16-byte chunks per row in a K tile
constexpr uint32_t kATile = 128 * kKT * 4;   // bytes of one A tile (hi or lo)
constexpr long long kSpinLimit = 1LL << 26;  // bounded mbarrier waits
constexpr int kRowStep = kTcThreads / kChunks;  // rows staged per pass (64)
constexpr int kMaxA = 64 / kRowStep;            // A rows per thread (M <= 64)
constexpr int kMaxB = 256 / kRowStep;           // B rows per thread (N tile <= 256)

__device__ int g_tc_timeout = 0;
__device__ int g_tc_inject = 0;  // test hook: expiries to report after real completion

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major, no swizzle: start address, leading (K chunk) and stride (8-row group) offsets.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

__device__ __forceinline__ void split4(float4 v, float4 &hi, float4 &lo) {
  hi = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
  lo = make_float4(tf32_rna(v.x - hi.x), tf32_rna(v.y - hi.y), tf32_rna(v.z - hi.z),
                   tf32_rna(v.w - hi.w));
}

// byte offset of (row r, 16-byte chunk c) in a canonical tile whose chunks are `lbo` apart
__device__ __forceinline__ uint32_t tile_off(int r, int c, uint32_t lbo) {
  return (uint32_t)c * lbo + (uint32_t)(r >> 3) * 128u + (uint32_t)(r & 7) * 16u;
}

__device__ __forceinline__ bool mbar_wait_raw(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kSpinLimit; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Bounded wait for the phase `parity` of barrier `bar`.  A pending test injection
// (g_tc_inject > 0, set on the host) makes one completed wait report expiry: the
// abort path then runs with every MMA of the CTA finished.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (!mbar_wait_raw(bar, parity)) return false;
  int v = *(volatile int *)&g_tc_inject;
  while (v > 0) {
    const int old = atomicCAS(&g_tc_inject, v, v - 1);
    if (old == v) return false;
    v = old;
  }
  return true;
}

// End of the MMA loop of a CTA that committed its first `committed` K tiles (all of
// them, or those before an expired wait at tile abort_it): wait for the last commit,
// which covers every MMA issued before it, so that TMEM is neither read nor released
// while an MMA may still write it.  Without an earlier expiry the wait is the drain
// and may itself report expiry; after one, the wait ignores test injections.  If the
// GPU really stopped answering for the whole bounded wait the CTA releases TMEM
// anyway (the context is then unusable: the host reports TDLZ_ERR_TIMEOUT).
__device__ __forceinline__ void quiesce(uint64_t *mbar, int &abort_flag, int abort_it,
                                        int nloc) {
  const int committed = abort_flag ? abort_it : nloc;
  if (committed > 0) {
    const int last = committed - 1;
    const uint32_t bar = smem_u32(&mbar[last & 1]), par = (uint32_t)((last >> 1) & 1);
    if (!abort_flag && !mbar_wait(bar, par)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) mbar_wait_raw(bar, par);
  }
  __syncthreads();
}

struct TcArgs {
  const float2 *A;
  long long lda, sA;
  int amod;
  const float2 *B;
  long long ldb, sB;
  int M, N;        // complex output rows (A rows) and columns per batch (B rows)
  long long K;     // complex contraction length
  int nj;          // batches per A (batch / amod)
  int ntot, nt;    // stacked B rows (nj * N) and rows per N tile (multiple of 16)
  int ntiles, nsplit, kt_per_split, nkt;
  uint32_t tmem_cols;
  float *part;     // [nsplit][amod][ntiles][128][nt]; transposed form [..][128][nm]
  int nm;          // transposed form: the MMA's N, 2M rounded up to 16
};

__global__ void __launch_bounds__(kTcThreads, 2) tc_gemm_tn_kernel(const TcArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, abort_it;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nt = g.nt;
  const uint32_t lboA = 16 * 128, lboB = (uint32_t)(nt / 8) * 128;
  static_assert(kKT / 8 >= 1 && kChunks % 4 == 0, "K tile of whole MMA steps, 4-chunk groups");
  const uint32_t bTile = (uint32_t)nt * kKT * 4;
  const uint32_t stage_bytes = 2 * kATile + 2 * bTile;
  // CTA coordinates: x = N tile, y = A batch, z = K split
  const int tile = blockIdx.x, a = blockIdx.y, z = blockIdx.z;
  const int kt0 = z * g.kt_per_split;
  const int kt1 = min(g.nkt, kt0 + g.kt_per_split);
  const int nloc = kt1 - kt0;

  // zero both stages once (rows >= 2M of A and rows >= ntot of B stay zero)
  for (uint32_t i = tid; i < 2 * stage_bytes / 16; i += blockDim.x)
    reinterpret_cast<float4 *>(tc_smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
    abort_it = nloc;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(g.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = (1u << 4)                           // D: F32
                         | (2u << 7) | (2u << 10)             // A, B: TF32
                         | ((uint32_t)(nt >> 3) << 17)        // N >> 3
                         | ((uint32_t)(128 >> 4) << 24);      // M >> 4
  const float2 *Ab = g.A + (long long)a * g.sA;
  // staging map: lanes 0-7 of a warp take 8 consecutive rows of one 16-byte chunk, so
  // each group of 8 stores fills one 128-byte core-matrix row block (no bank conflicts);
  // the 4 lane groups take 4 chunks, kChunks / 4 consecutive warps the K tile's chunks
  constexpr int kWarpsPerRow = kChunks / 4;
  const int lane = tid & 31;
  const int sub = (lane >> 3) + 4 * (warp % kWarpsPerRow);   // 16-byte chunk
  const int rbase = (warp / kWarpsPerRow) * 8 + (lane & 7);  // first row; then every kRowStep
  const int rstep = kRowStep;

  // global loads of K tile t into registers (read-only path); issued one tile ahead
  // of the shared-memory stores so that their latency overlaps the proxy fence, the
  // barrier, the MMA issue and the wait for the stage
  float4 va[kMaxA], vb[kMaxB];
  auto load_tile = [&](int t) {
    const long long kc = (long long)(kt0 + t) * (kKT / 2) + 2 * sub;  // complex pair
#pragma unroll
    for (int i = 0; i < kMaxA; ++i) {
      const int m = rbase + i * rstep;
      va[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < g.M && kc < g.K) {
        const float2 *row = Ab + (long long)m * g.lda;
        const float2 t0 = __ldg(row + kc);
        const float2 t1 = kc + 1 < g.K ? __ldg(row + kc + 1) : make_float2(0.f, 0.f);
        va[i] = make_float4(t0.x, t0.y, t1.x, t1.y);
      }
    }
#pragma unroll
    for (int i = 0; i < kMaxB; ++i) {
      const int r = rbase + i * rstep;
      const int R = tile * nt + r;
      vb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < nt && R < g.ntot && kc < g.K) {
        const int j = R / g.N, n = R - j * g.N;
        const float2 *row =
            g.B + (long long)(a + (long long)j * g.amod) * g.sB + (long long)n * g.ldb;
        const float2 t0 = __ldg(row + kc);
        const float2 t1 = kc + 1 < g.K ? __ldg(row + kc + 1) : make_float2(0.f, 0.f);
        vb[i] = make_float4(t0.x, t0.y, t1.x, t1.y);
      }
    }
  };
  if (nloc > 0) load_tile(0);
  for (int it = 0; it < nloc; ++it) {
    const int s = it & 1;
    // tile it's loads are in flight while the MMAs of tile it-2 release stage s
    if (it >= 2) {
      if (!mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((it - 2) >> 1) & 1))) {
        abort_flag = 1;
        abort_it = it;
      }
    }
    __syncthreads();
    if (abort_flag) break;
    unsigned char *st = tc_smem + (size_t)s * stage_bytes;
    unsigned char *Ahi = st, *Alo = st + kATile, *Bhi = st + 2 * kATile, *Blo = Bhi + bTile;
    // A rows [A_int; A_rot]
#pragma unroll
    for (int i = 0; i < kMaxA; ++i) {
      const int m = rbase + i * rstep;
      if (m < g.M) {
        float4 hi, lo;
        split4(va[i], hi, lo);
        *reinterpret_cast<float4 *>(Ahi + tile_off(m, sub, lboA)) = hi;
        *reinterpret_cast<float4 *>(Alo + tile_off(m, sub, lboA)) = lo;
        split4(make_float4(-va[i].y, va[i].x, -va[i].w, va[i].z), hi, lo);
        *reinterpret_cast<float4 *>(Ahi + tile_off(g.M + m, sub, lboA)) = hi;
        *reinterpret_cast<float4 *>(Alo + tile_off(g.M + m, sub, lboA)) = lo;
      }
    }
    // B rows of this N tile: stacked (j, n) -> batch a + j amod, row n
#pragma unroll
    for (int i = 0; i < kMaxB; ++i) {
      const int r = rbase + i * rstep;
      if (r < nt) {
        float4 hi, lo;
        split4(vb[i], hi, lo);
        *reinterpret_cast<float4 *>(Bhi + tile_off(r, sub, lboB)) = hi;
        *reinterpret_cast<float4 *>(Blo + tile_off(r, sub, lboB)) = lo;
      }
    }
    if (it + 1 < nloc) load_tile(it + 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi),
                     bl = smem_u32(Blo);
#pragma unroll
      for (int ks = 0; ks < kKT / 8; ++ks) {
        const uint32_t oa = 2 * ks * lboA, ob = 2 * ks * lboB;
        const uint64_t dah = smem_desc(ah + oa, lboA, 128), dal = smem_desc(al + oa, lboA, 128);
        const uint64_t dbh = smem_desc(bh + ob, lboB, 128), dbl = smem_desc(bl + ob, lboB, 128);
        const uint32_t acc0 = (it > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
        asm volatile(
            "{\n.reg .pred p;\nsetp.eq.u32 p, 1, 1;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %4, %5, %3, p;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbl), "r"(idesc), "l"(dal), "l"(dbh));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar[s])));
    }
  }
  quiesce(mbar, abort_flag, abort_it, nloc);
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool ok = !abort_flag && nloc > 0;
  if (!ok && tid == 0 && abort_flag) atomicExch(&g_tc_timeout, 1);
  // epilogue: warp w reads TMEM lanes (rows) 32 (w & 3) .. + 31 (its lane quarter),
  // the two warps of a quarter take alternate 8-column chunks
  const int quarter = warp & 3;
  const int row = 32 * quarter + (tid & 31);
  float *out = g.part + ((((long long)z * gridDim.y + a) * g.ntiles + tile) * 128 + row) * nt;
  for (int c0 = 8 * (warp >> 2); c0 < nt; c0 += 16) {
    uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (ok) {  // TMEM is read only after the last commit's barrier completed
      const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
    }
    if (row < 2 * g.M) {
      float4 *o = reinterpret_cast<float4 *>(out + c0);
      if (ok) {
        o[0] = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]),
                           __uint_as_float(r[3]));
        o[1] = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]),
                           __uint_as_float(r[7]));
      } else {
        o[0] = o[1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(g.tmem_cols));
}

// Transposed form for 64 < M <= 128 (2M rows do not fit the MMA's M): the MMA's M = 128
// stacked B rows (R = j N + n of the batches b = a + j amod sharing A), its N = the 2M
// rows [A_int; A_rot] rounded up to 16 (<= 256), so D[R][m] = Re C[m][n] and
// D[R][M + m] = Im C[m][n] of TMEM lane R.  Staging, pipeline and the bounded waits are
// those of tc_gemm_tn_kernel with the operands' roles exchanged.
__global__ void __launch_bounds__(kTcThreads, 2) tc_gemm_tnt_kernel(const TcArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, abort_it;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nm = g.nm;
  const uint32_t lboX = 16 * 128, lboA = (uint32_t)(nm / 8) * 128;
  const uint32_t xTile = 128 * kKT * 4, aTile = (uint32_t)nm * kKT * 4;
  const uint32_t stage_bytes = 2 * xTile + 2 * aTile;
  // CTA coordinates: x = 128-row tile of the stacked B rows, y = A batch, z = K split
  const int tile = blockIdx.x, a = blockIdx.y, z = blockIdx.z;
  const int kt0 = z * g.kt_per_split;
  const int kt1 = min(g.nkt, kt0 + g.kt_per_split);
  const int nloc = kt1 - kt0;
  for (uint32_t i = tid; i < 2 * stage_bytes / 16; i += blockDim.x)
    reinterpret_cast<float4 *>(tc_smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
    abort_it = nloc;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(g.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = (1u << 4)                           // D: F32
                         | (2u << 7) | (2u << 10)             // A, B: TF32
                         | ((uint32_t)(nm >> 3) << 17)        // N >> 3
                         | ((uint32_t)(128 >> 4) << 24);      // M >> 4
  const float2 *Ab = g.A + (long long)a * g.sA;
  constexpr int kWarpsPerRow = kChunks / 4;
  const int lane = tid & 31;
  const int sub = (lane >> 3) + 4 * (warp % kWarpsPerRow);
  const int rbase = (warp / kWarpsPerRow) * 8 + (lane & 7);
  const int rstep = kRowStep;
  constexpr int kX = 128 / kRowStep, kA = 128 / kRowStep;  // rows per thread (M <= 128)
  float4 vx[kX], va[kA];
  auto load_tile = [&](int t) {
    const long long kc = (long long)(kt0 + t) * (kKT / 2) + 2 * sub;
#pragma unroll
    for (int i = 0; i < kX; ++i) {
      const int r = rbase + i * rstep;
      const int R = tile * 128 + r;
      vx[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (R < g.ntot && kc < g.K) {
        const int j = R / g.N, n = R - j * g.N;
        const float2 *row =
            g.B + (long long)(a + (long long)j * g.amod) * g.sB + (long long)n * g.ldb;
        const float2 t0 = __ldg(row + kc);
        const float2 t1 = kc + 1 < g.K ? __ldg(row + kc + 1) : make_float2(0.f, 0.f);
        vx[i] = make_float4(t0.x, t0.y, t1.x, t1.y);
      }
    }
#pragma unroll
    for (int i = 0; i < kA; ++i) {
      const int m = rbase + i * rstep;
      va[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < g.M && kc < g.K) {
        const float2 *row = Ab + (long long)m * g.lda;
        const float2 t0 = __ldg(row + kc);
        const float2 t1 = kc + 1 < g.K ? __ldg(row + kc + 1) : make_float2(0.f, 0.f);
        va[i] = make_float4(t0.x, t0.y, t1.x, t1.y);
      }
    }
  };
  if (nloc > 0) load_tile(0);
  for (int it = 0; it < nloc; ++it) {
    const int s = it & 1;
    if (it >= 2) {
      if (!mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((it - 2) >> 1) & 1))) {
        abort_flag = 1;
        abort_it = it;
      }
    }
    __syncthreads();
    if (abort_flag) break;
    unsigned char *st = tc_smem + (size_t)s * stage_bytes;
    unsigned char *Xhi = st, *Xlo = st + xTile, *Ahi = st + 2 * xTile, *Alo = Ahi + aTile;
#pragma unroll
    for (int i = 0; i < kX; ++i) {
      const int r = rbase + i * rstep;
      float4 hi, lo;
      split4(vx[i], hi, lo);
      *reinterpret_cast<float4 *>(Xhi + tile_off(r, sub, lboX)) = hi;
      *reinterpret_cast<float4 *>(Xlo + tile_off(r, sub, lboX)) = lo;
    }
#pragma unroll
    for (int i = 0; i < kA; ++i) {
      const int m = rbase + i * rstep;
      if (m < g.M) {
        float4 hi, lo;
        split4(va[i], hi, lo);
        *reinterpret_cast<float4 *>(Ahi + tile_off(m, sub, lboA)) = hi;
        *reinterpret_cast<float4 *>(Alo + tile_off(m, sub, lboA)) = lo;
        split4(make_float4(-va[i].y, va[i].x, -va[i].w, va[i].z), hi, lo);
        *reinterpret_cast<float4 *>(Ahi + tile_off(g.M + m, sub, lboA)) = hi;
        *reinterpret_cast<float4 *>(Alo + tile_off(g.M + m, sub, lboA)) = lo;
      }
    }
    if (it + 1 < nloc) load_tile(it + 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t xh = smem_u32(Xhi), xl = smem_u32(Xlo), ah = smem_u32(Ahi),
                     al = smem_u32(Alo);
#pragma unroll
      for (int ks = 0; ks < kKT / 8; ++ks) {
        const uint32_t ox = 2 * ks * lboX, oa = 2 * ks * lboA;
        const uint64_t dxh = smem_desc(xh + ox, lboX, 128), dxl = smem_desc(xl + ox, lboX, 128);
        const uint64_t dah = smem_desc(ah + oa, lboA, 128), dal = smem_desc(al + oa, lboA, 128);
        const uint32_t acc0 = (it > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(dxh), "l"(dah), "r"(idesc), "r"(acc0));
        asm volatile(
            "{\n.reg .pred p;\nsetp.eq.u32 p, 1, 1;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %4, %5, %3, p;\n}\n" ::"r"(tmem),
            "l"(dxh), "l"(dal), "r"(idesc), "l"(dxl), "l"(dah));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar[s])));
    }
  }
  quiesce(mbar, abort_flag, abort_it, nloc);
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool ok = !abort_flag && nloc > 0;
  if (!ok && tid == 0 && abort_flag) atomicExch(&g_tc_timeout, 1);
  // epilogue: warp w reads TMEM lanes 32 (w & 3) .. + 31 (stacked rows R), the two warps
  // of a quarter take alternate 8-column chunks of the nm columns
  const int quarter = warp & 3;
  const int row = 32 * quarter + (tid & 31);
  float *out = g.part + ((((long long)z * gridDim.y + a) * g.ntiles + tile) * 128 + row) * nm;
  for (int c0 = 8 * (warp >> 2); c0 < nm; c0 += 16) {
    uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (ok) {
      const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
    }
    float4 *o = reinterpret_cast<float4 *>(out + c0);
    if (ok) {
      o[0] = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]),
                         __uint_as_float(r[3]));
      o[1] = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]),
                         __uint_as_float(r[7]));
    } else {
      o[0] = o[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(g.tmem_cols));
}

// C[b*sC + m*ldcm + n*ldcn] = sum_z (part[z][a][t][rr][m], part[z][a][t][rr][M+m]) with
// b = a + j amod, stacked row R = j N + n = 128 t + rr (the transposed form's partials).
__global__ void tc_reduce_t_kernel(const float *__restrict__ part, float2 *__restrict__ C, int M,
                                   int N, int amod, int nj, int ntiles, int nm, int nsplit,
                                   long long sC, long long ldcm, long long ldcn) {
  const long long total = (long long)amod * nj * M * N;
  const long long zstride = (long long)amod * ntiles * 128 * nm;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / ((long long)M * N);
    const int rem = (int)(e - b * M * N);
    const int m = rem / N, n = rem - m * N;
    const int a = (int)(b % amod), j = (int)(b / amod);
    const int R = j * N + n, t = R >> 7, rr = R & 127;
    const float *p = part + ((((long long)a * ntiles + t) * 128) + rr) * nm;
    float re = 0.f, im = 0.f;
#pragma unroll 8
    for (int zz = 0; zz < nsplit; ++zz) {
      re += p[(long long)zz * zstride + m];
      im += p[(long long)zz * zstride + M + m];
    }
    C[b * sC + m * ldcm + n * ldcn] = make_float2(re, im);
  }
}

// C[b*sC + m*ldcm + n*ldcn] = sum_z (part[z][a][t][m][col], part[z][a][t][M+m][col])
// with b = a + j amod and stacked row R = j N + n = t nt + col.
__global__ void tc_reduce_kernel(const float *__restrict__ part, float2 *__restrict__ C, int M,
                                 int N, int amod, int nj, int ntiles, int nt, int nsplit,
                                 long long sC, long long ldcm, long long ldcn) {
  const long long total = (long long)amod * nj * M * N;
  const long long zstride = (long long)amod * ntiles * 128 * nt;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / ((long long)M * N);
    const int rem = (int)(e - b * M * N);
    const int m = rem / N, n = rem - m * N;
    const int a = (int)(b % amod), j = (int)(b / amod);
    const int R = j * N + n, t = R / nt, col = R - t * nt;
    const float *p = part + (((long long)a * ntiles + t) * 128) * nt + col;
    float re = 0.f, im = 0.f;
#pragma unroll 8
    for (int zz = 0; zz < nsplit; ++zz) {
      re += p[(long long)zz * zstride + (long long)m * nt];
      im += p[(long long)zz * zstride + (long long)(M + m) * nt];
    }
    C[b * sC + m * ldcm + n * ldcn] = make_float2(re, im);
  }
}

// ---------------------------------------------------------------------------------
// Update GEMMs:  Out[b][r][n] = sg_b (In[b][r][n] + alpha sum_k A[b][r][k] B[b % bmod][k][n])
//
// computed transposed, so that one TMEM lane is one output column n: the MMA's M = 128
// columns of B (rows (b.x, b.y) per complex k), its N = 2R rows built from A with
// Re row 2r = (a.x, -a.y) and Im row 2r+1 = (a.y, a.x) per complex k, so that
// D[n][2r] = Re (A B)[r][n] and D[n][2r+1] = Im (A B)[r][n] sit in neighbouring TMEM
// columns of the same lane.  The epilogue thread of lane n then reads, updates and
// writes row r of column n; a warp covers 32 consecutive n (coalesced).
constexpr int kNnKT = 16;                 // K tile: 16 reals (8 complex) = 64 bytes per row
constexpr int kNnM = 128;                 // output columns per CTA (the MMA's M)

struct NnArgs {
  const float2 *A;
  long long sA, sar, sak;
  const float2 *B;
  long long ldb, sB;
  int bmod;
  const float2 *In;
  float2 *Out;
  long long ldo, sO;
  long long ncol;
  int R, K, nm, nkt;   // output rows, complex K, the MMA's N (2R rounded up to 16), K tiles
  float alpha;
  int neg_from, neg_mod;
  uint32_t tmem_cols;
};

__global__ void __launch_bounds__(kTcThreads, 2) tc_gemm_nn_kernel(const NnArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, abort_it;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ct = blockIdx.x;  // column tile
  const long long b = blockIdx.y;   // batch
  const uint32_t lboA = (kNnM / 8) * 128, lboB = (uint32_t)(g.nm / 8) * 128;
  const uint32_t aTile = kNnM * kNnKT * 4, bTile = (uint32_t)g.nm * kNnKT * 4;
  const uint32_t stage_bytes = 2 * aTile + 2 * bTile;

  // zero both stages once (B-operand rows >= 2R stay zero)
  for (uint32_t i = tid; i < 2 * stage_bytes / 16; i += blockDim.x)
    reinterpret_cast<float4 *>(tc_smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
    abort_it = g.nkt;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(g.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = (1u << 4)                           // D: F32
                         | (2u << 7) | (2u << 10)             // A, B: TF32
                         | ((uint32_t)(g.nm >> 3) << 17)      // N >> 3
                         | ((uint32_t)(kNnM >> 4) << 24);     // M >> 4
  const float2 *Bb = g.B + (b % g.bmod) * g.sB;
  const float2 *Ab = g.A + b * g.sA;
  // staging items: the MMA's A operand has 128 rows x 4 chunks (two per thread, lanes on
  // consecutive columns n: coalesced loads, 16-byte stores at a 16-byte stride); its
  // B operand has R x 4 (row r, chunk) items, each writing rows 2r and 2r+1
  float4 va[2], vb[2];
  auto load_tile = [&](int t) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * kTcThreads;
      const int i = e & (kNnM - 1), c = e >> 7;
      const long long n = ct * kNnM + i;
      const int kc = t * (kNnKT / 2) + 2 * c;
      float2 t0 = make_float2(0.f, 0.f), t1 = t0;
      if (n < g.ncol) {
        if (kc < g.K) t0 = __ldg(Bb + (long long)kc * g.ldb + n);
        if (kc + 1 < g.K) t1 = __ldg(Bb + (long long)(kc + 1) * g.ldb + n);
      }
      va[u] = make_float4(t0.x, t0.y, t1.x, t1.y);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * kTcThreads;
      const int r = e >> 2, c = e & 3;
      const int kc = t * (kNnKT / 2) + 2 * c;
      float2 t0 = make_float2(0.f, 0.f), t1 = t0;
      if (r < g.R) {
        if (kc < g.K) t0 = __ldg(Ab + r * g.sar + kc * g.sak);
        if (kc + 1 < g.K) t1 = __ldg(Ab + r * g.sar + (kc + 1) * g.sak);
      }
      vb[u] = make_float4(t0.x, t0.y, t1.x, t1.y);
    }
  };
  if (g.nkt > 0) load_tile(0);
  for (int it = 0; it < g.nkt; ++it) {
    const int s = it & 1;
    if (it >= 2) {
      if (!mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((it - 2) >> 1) & 1))) {
        abort_flag = 1;
        abort_it = it;
      }
    }
    __syncthreads();
    if (abort_flag) break;
    unsigned char *st = tc_smem + (size_t)s * stage_bytes;
    unsigned char *Ahi = st, *Alo = st + aTile, *Bhi = st + 2 * aTile, *Blo = Bhi + bTile;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * kTcThreads;
      const int i = e & (kNnM - 1), c = e >> 7;
      float4 hi, lo;
      split4(va[u], hi, lo);
      *reinterpret_cast<float4 *>(Ahi + tile_off(i, c, lboA)) = hi;
      *reinterpret_cast<float4 *>(Alo + tile_off(i, c, lboA)) = lo;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * kTcThreads;
      const int r = e >> 2, c = e & 3;
      if (r < g.R) {
        const float4 v = vb[u];
        float4 hi, lo;
        split4(make_float4(v.x, -v.y, v.z, -v.w), hi, lo);  // Re row: (a.x, -a.y)
        *reinterpret_cast<float4 *>(Bhi + tile_off(2 * r, c, lboB)) = hi;
        *reinterpret_cast<float4 *>(Blo + tile_off(2 * r, c, lboB)) = lo;
        split4(make_float4(v.y, v.x, v.w, v.z), hi, lo);    // Im row: (a.y, a.x)
        *reinterpret_cast<float4 *>(Bhi + tile_off(2 * r + 1, c, lboB)) = hi;
        *reinterpret_cast<float4 *>(Blo + tile_off(2 * r + 1, c, lboB)) = lo;
      }
    }
    if (it + 1 < g.nkt) load_tile(it + 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi),
                     bl = smem_u32(Blo);
#pragma unroll
      for (int ks = 0; ks < kNnKT / 8; ++ks) {
        const uint32_t oa = 2 * ks * lboA, ob = 2 * ks * lboB;
        const uint64_t dah = smem_desc(ah + oa, lboA, 128), dal = smem_desc(al + oa, lboA, 128);
        const uint64_t dbh = smem_desc(bh + ob, lboB, 128), dbl = smem_desc(bl + ob, lboB, 128);
        const uint32_t acc0 = (it > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
        asm volatile(
            "{\n.reg .pred p;\nsetp.eq.u32 p, 1, 1;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %4, %5, %3, p;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbl), "r"(idesc), "l"(dal), "l"(dbh));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar[s])));
    }
  }
  quiesce(mbar, abort_flag, abort_it, g.nkt);
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool ok = !abort_flag;
  if (abort_flag && tid == 0) atomicExch(&g_tc_timeout, 1);
  // epilogue: warp w reads lane quarter w & 3 (32 consecutive columns n); the two warps
  // of a quarter take alternate 16-column TMEM blocks (8 output rows each)
  const int quarter = warp & 3;
  const long long n = ct * kNnM + 32 * quarter + lane;
  const bool nv = n < g.ncol;
  const float sg = (b % g.neg_mod) >= g.neg_from ? -1.f : 1.f;
  const float2 *inb = g.In + b * g.sO + n;
  float2 *outb = g.Out + b * g.sO + n;
  for (int j0 = 16 * (warp >> 2); j0 < 2 * g.R; j0 += 32) {
    const int r0 = j0 >> 1;
    float2 iv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      iv[u] = (nv && r0 + u < g.R) ? inb[(long long)(r0 + u) * g.ldo] : make_float2(0.f, 0.f);
    if (!ok) break;  // TMEM is read only after the last commit's barrier completed
    uint32_t v[16];
    const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)j0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (ok && nv) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (r0 + u >= g.R) break;
        const float re = __uint_as_float(v[2 * u]), im = __uint_as_float(v[2 * u + 1]);
        outb[(long long)(r0 + u) * g.ldo] =
            make_float2(sg * (iv[u].x + g.alpha * re), sg * (iv[u].y + g.alpha * im));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(g.tmem_cols));
}

// 64 < M <= 128: the transposed form (tc_gemm_tnt_kernel), same contract as tc_gemm_tn.
bool tc_gemm_tn_transposed(Context &ctx, DevBuf &partbuf, const float2 *A, long long lda,
                           long long sA, int amod, const float2 *B, long long ldb, long long sB,
                           float2 *C, long long sC, long long ldcm, long long ldcn, int M, int N,
                           long long K, int batch) {
  TcArgs g{};
  g.A = A;
  g.lda = lda;
  g.sA = sA;
  g.amod = amod;
  g.B = B;
  g.ldb = ldb;
  g.sB = sB;
  g.M = M;
  g.N = N;
  g.K = K;
  g.nj = batch / amod;
  g.ntot = g.nj * N;
  g.ntiles = (g.ntot + 127) / 128;
  g.nt = 128;
  g.nm = (2 * M + 15) / 16 * 16;
  g.nkt = (int)((K + kKT / 2 - 1) / (kKT / 2));
  const int ctas = amod * g.ntiles;
  const size_t per_split = (size_t)amod * g.ntiles * 128 * g.nm * sizeof(float);
  const long long fit = (long long)(partbuf.bytes / per_split);
  if (fit < 1) return false;
  long long ns = std::max(1, std::min(g.nkt, (4 * 152 + ctas - 1) / ctas));
  ns = std::min(ns, fit);
  g.kt_per_split = (int)((g.nkt + ns - 1) / ns);
  g.nsplit = (g.nkt + g.kt_per_split - 1) / g.kt_per_split;
  g.tmem_cols = 32;
  while (g.tmem_cols < (uint32_t)g.nm) g.tmem_cols *= 2;
  g.part = partbuf.as<float>();
  // no more CTAs per SM than the 512 TMEM columns hold (ask for enough shared memory that
  // one more would not fit), so that no CTA waits in tcgen05.alloc
  const int cap = (int)(512 / g.tmem_cols);
  const size_t smem = std::max(2 * (2 * (size_t)128 * kKT * 4 + 2 * (size_t)g.nm * kKT * 4),
                               (size_t)(233472 / (cap + 1)));
  TDLZ_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_tnt_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(g.ntiles, amod, g.nsplit);
  tc_gemm_tnt_kernel<<<grid, kTcThreads, smem, ctx.stream>>>(g);
  TDLZ_LAUNCH_CHECK();
  const long long total = (long long)batch * M * N;
  tc_reduce_t_kernel<<<blocks_for(total), 256, 0, ctx.stream>>>(g.part, C, M, N, amod, g.nj,
                                                                 g.ntiles, g.nm, g.nsplit, sC,
                                                                 ldcm, ldcn);
  TDLZ_LAUNCH_CHECK();
  return true;
}

// ---------------------------------------------------------------------------------
// Update GEMM from operand images: the bulk-copy / TMA form of tc_gemm_nn_kernel.
//
// The MMA operands of every K tile are kept in global memory already split into TF32
// hi and lo parts and laid out as the canonical K-major shared-memory tiles the MMA
// reads (core matrices of 8 rows x 16 bytes, chunks 16 rows-groups apart):
//   A operand: 128 columns n of the constant matrix B[g][k][n] (the occupied k+q
//              states, the projectors), built once per ground state (nn_aimg_kernel);
//   B operand: the 2R rows (Re, Im) built from A[b][r][k], per call (nn_bimg_kernel).
// A CTA then only moves bytes and issues MMAs: one thread copies the K tiles into a
// ring of S shared-memory stages with 1-D bulk copies (cp.async.bulk) and issues the
// MMAs of each stage as it lands; a stage is refilled once the MMAs that read it have
// committed.  Meanwhile the other threads prefetch the CTA's In tile into L2 for the
// epilogue (or, optionally, one tensor copy, cp.async.bulk.tensor over the 3-D map
// [batch][R][2 ncol], brings it into shared memory at launch).  Values, MMA order and
// epilogue arithmetic are those of tc_gemm_nn_kernel, so the result is the same bit
// for bit.
constexpr uint32_t kAImgTile = 2 * 128 * 16 * 4;  // A-operand image of one K tile, hi + lo
constexpr int kNnMaxStages = 8;

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// tiled tensor copy of the box at (x, y, z) of a 3-D map (x in elements of dimension 0)
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], "
      "[%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// img[(g nct + ct) nkt + kt][hl][c][nl] (16-byte entries) = TF32 split (hl = 0: hi,
// 1: lo) of (B[g][k][n], B[g][k + 1][n]) with k = 8 kt + 2 c, n = 128 ct + nl; zero
// outside K x ncol.  Consecutive threads take consecutive columns (coalesced).
__global__ void nn_aimg_kernel(const float2 *__restrict__ B, long long ldb, long long sB, int G,
                               int K, long long ncol, int nct, int nkt, float4 *__restrict__ img) {
  const long long total = (long long)G * nct * nkt * 512;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int nl = (int)(e & 127), c = (int)((e >> 7) & 3);
    const long long tile = e >> 9;
    const int kt = (int)(tile % nkt);
    const long long gc = tile / nkt;
    const int ct = (int)(gc % nct);
    const long long g = gc / nct;
    const long long n = (long long)ct * 128 + nl;
    const int k0 = 8 * kt + 2 * c;
    float2 t0 = make_float2(0.f, 0.f), t1 = t0;
    if (n < ncol) {
      const float2 *col = B + g * sB + n;
      if (k0 < K) t0 = col[(long long)k0 * ldb];
      if (k0 + 1 < K) t1 = col[(long long)(k0 + 1) * ldb];
    }
    float4 hi, lo;
    split4(make_float4(t0.x, t0.y, t1.x, t1.y), hi, lo);
    float4 *o = img + tile * 1024 + c * 128 + nl;
    o[0] = hi;
    o[512] = lo;
  }
}

// img[b nkt + kt][hl][c][row] (16-byte entries, nm rows): rows 2r and 2r + 1 hold the
// TF32 split of (a0.x, -a0.y, a1.x, -a1.y) and (a0.y, a0.x, a1.y, a1.x) with
// a0 = A[b][r][k0], a1 = A[b][r][k0 + 1], k0 = 8 kt + 2 c (zero beyond K); rows >= 2R
// are zero.
__global__ void nn_bimg_kernel(const float2 *__restrict__ A, long long sA, long long sar,
                               long long sak, int R, int K, int nkt, int nm, long long batch,
                               float4 *__restrict__ img) {
  const int half = nm / 2;
  const long long total = batch * nkt * 4 * half;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int rp = (int)(e % half);
    long long t = e / half;
    const int c = (int)(t & 3);
    t >>= 2;  // b nkt + kt
    const int kt = (int)(t % nkt);
    const long long b = t / nkt;
    float4 *o = img + t * (8LL * nm) + (long long)c * nm + 2 * rp;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (rp >= R) {
      o[0] = o[1] = o[4 * nm] = o[4 * nm + 1] = z4;
      continue;
    }
    const int k0 = 8 * kt + 2 * c;
    const float2 *row = A + b * sA + (long long)rp * sar;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0;
    if (k0 < K) a0 = row[(long long)k0 * sak];
    if (k0 + 1 < K) a1 = row[(long long)(k0 + 1) * sak];
    float4 hr, lr, hm, lm;
    split4(make_float4(a0.x, -a0.y, a1.x, -a1.y), hr, lr);  // Re row
    split4(make_float4(a0.y, a0.x, a1.y, a1.x), hm, lm);    // Im row
    o[0] = hr;
    o[1] = hm;
    o[4 * nm] = lr;
    o[4 * nm + 1] = lm;
  }
}

struct NnImgArgs {
  const unsigned char *aimg;  // [G][nct][nkt] A-operand K-tile images (kAImgTile bytes each)
  const unsigned char *bimg;  // [batch][nkt] B-operand K-tile images (128 nm bytes each)
  const float2 *In;           // read in the epilogue where the tensor copy is not used
  float2 *Out;
  long long ldo, sO, ncol;
  int R, nm, nkt, nct, G, nj, S, in_tma;
  float alpha;
  int neg_from, neg_mod;
  uint32_t tmem_cols, in_bytes, stage_bytes;
};

// One CTA per (batch b, 128-column tile); the CTAs of the batches b = g + j G that share
// an A-operand image are consecutive in launch order (j fastest), so that the image is
// read from L2 after the first of them.
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_nn_img_kernel(const __grid_constant__ CUtensorMap tm_in, const NnImgArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t full[kNnMaxStages], empty[kNnMaxStages], inbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, n_commit;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  long long L = blockIdx.x;
  const int j = (int)(L % g.nj);
  L /= g.nj;
  const int ct = (int)(L % g.nct);
  const long long gi = L / g.nct;
  const long long b = gi + (long long)j * g.G;
  const uint32_t bop = 128u * (uint32_t)g.nm;
  const int S = g.S;
  unsigned char *in_s = tc_smem;               // [R][256 floats] In tile (tensor copy)
  unsigned char *ring = tc_smem + g.in_bytes;  // S stages: A image, then B image
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&inbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
    n_commit = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(g.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const float2 *inb = g.In + b * g.sO;
  if (!g.in_tma) {
    // In is read in the epilogue: start pulling this tile's rows into L2 now
    for (int e = tid; e < g.R * 8; e += kTcThreads) {
      const long long n0 = (long long)ct * 128 + (e & 7) * 16;
      if (n0 < g.ncol)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(inb + (long long)(e >> 3) * g.ldo + n0));
    }
  }
  if (tid == 0) {
    const unsigned char *abase = g.aimg + (gi * g.nct + ct) * g.nkt * (long long)kAImgTile;
    const unsigned char *bbase = g.bimg + b * g.nkt * (long long)bop;
    auto issue = [&](int t) {
      const int s = t % S;
      const uint32_t bar = smem_u32(&full[s]);
      const uint32_t dst = smem_u32(ring + (size_t)s * g.stage_bytes);
      mbar_expect_tx(bar, kAImgTile + bop);
      bulk_g2s(dst, abase + (long long)t * kAImgTile, kAImgTile, bar);
      bulk_g2s(dst + kAImgTile, bbase + (long long)t * bop, bop, bar);
    };
    if (g.in_tma) {
      const uint32_t bar = smem_u32(&inbar);
      mbar_expect_tx(bar, g.in_bytes);
      tma_load_3d(smem_u32(in_s), &tm_in, ct * 256, 0, (int)b, bar);
    }
    int issued = 0;
    while (issued < min(S, g.nkt)) issue(issued++);
    const uint32_t idesc = (1u << 4)                           // D: F32
                           | (2u << 7) | (2u << 10)             // A, B: TF32
                           | ((uint32_t)(g.nm >> 3) << 17)      // N >> 3
                           | ((uint32_t)(kNnM >> 4) << 24);     // M >> 4
    const uint32_t lboA = (kNnM / 8) * 128, lboB = (uint32_t)g.nm * 16;
    bool ok = true;
    int committed = 0;
    for (int it = 0; it < g.nkt; ++it) {
      const int s = it % S;
      if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((it / S) & 1))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = smem_u32(ring + (size_t)s * g.stage_bytes), al = ah + kAImgTile / 2;
      const uint32_t bh = ah + kAImgTile, bl = bh + bop / 2;
#pragma unroll
      for (int ks = 0; ks < kNnKT / 8; ++ks) {
        const uint32_t oa = 2 * ks * lboA, ob = 2 * ks * lboB;
        const uint64_t dah = smem_desc(ah + oa, lboA, 128), dal = smem_desc(al + oa, lboA, 128);
        const uint64_t dbh = smem_desc(bh + ob, lboB, 128), dbl = smem_desc(bl + ob, lboB, 128);
        const uint32_t acc0 = (it > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
        asm volatile(
            "{\n.reg .pred p;\nsetp.eq.u32 p, 1, 1;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %4, %5, %3, p;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbl), "r"(idesc), "l"(dal), "l"(dbh));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&empty[s])));
      committed = it + 1;
      // refill the stage of the previous tile once its MMAs have committed (the stage
      // of this tile is still being read); issued == it - 1 + S here
      if (it >= 1 && issued < g.nkt) {
        const int p = it - 1;
        if (!mbar_wait(smem_u32(&empty[p % S]), (uint32_t)((p / S) & 1))) {
          ok = false;
          break;
        }
        issue(issued++);
      }
    }
    // quiesce: every copy issued lands, and the last commit (which covers every MMA
    // issued before it) completes, before TMEM is read or the CTA's memory released.
    // The last S copies issued are the newest of their stages, so their phases are
    // unambiguous; waits after an expiry ignore test injections.
    if (!ok)
      for (int u = max(0, issued - S); u < issued; ++u)
        mbar_wait_raw(smem_u32(&full[u % S]), (uint32_t)((u / S) & 1));
    if (committed > 0) {
      const int last = committed - 1;
      const uint32_t bar = smem_u32(&empty[last % S]), par = (uint32_t)((last / S) & 1);
      if (ok && !mbar_wait(bar, par)) ok = false;
      if (!ok) mbar_wait_raw(bar, par);
    }
    if (g.in_tma) {
      const uint32_t bar = smem_u32(&inbar);
      if (ok && !mbar_wait(bar, 0)) ok = false;
      if (!ok) mbar_wait_raw(bar, 0);
    }
    abort_flag = ok ? 0 : 1;
    n_commit = committed;
  }
  __syncthreads();
  const bool ok = !abort_flag && n_commit == g.nkt;
  if (tid == 0 && abort_flag) atomicExch(&g_tc_timeout, 1);
  if (ok) {
    // completed phases: these waits return at once and order the MMAs' TMEM writes and
    // the tensor copy's shared-memory writes before this thread's reads
    const int last = g.nkt - 1;
    mbar_wait_raw(smem_u32(&empty[last % S]), (uint32_t)((last / S) & 1));
    if (g.in_tma) mbar_wait_raw(smem_u32(&inbar), 0);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  // epilogue (as tc_gemm_nn_kernel): warp w reads lane quarter w & 3 (32 consecutive
  // columns n); the two warps of a quarter take alternate 16-column TMEM blocks
  const int quarter = warp & 3;
  const int nl = 32 * quarter + lane;
  const long long n = (long long)ct * kNnM + nl;
  const bool nv = n < g.ncol;
  const float sg = (b % g.neg_mod) >= g.neg_from ? -1.f : 1.f;
  const float2 *inrow = inb + n;
  float2 *outb = g.Out + b * g.sO + n;
  for (int j0 = 16 * (warp >> 2); j0 < 2 * g.R; j0 += 32) {
    const int r0 = j0 >> 1;
    if (!ok) break;  // TMEM is read only after the last commit's barrier completed
    float2 iv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      iv[u] = make_float2(0.f, 0.f);
      if (r0 + u < g.R) {
        if (g.in_tma)
          iv[u] = *reinterpret_cast<const float2 *>(in_s + (size_t)(r0 + u) * 1024 + nl * 8);
        else if (nv)
          iv[u] = inrow[(long long)(r0 + u) * g.ldo];
      }
    }
    uint32_t v[16];
    const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)j0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (nv) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (r0 + u >= g.R) break;
        const float re = __uint_as_float(v[2 * u]), im = __uint_as_float(v[2 * u + 1]);
        outb[(long long)(r0 + u) * g.ldo] =
            make_float2(sg * (iv[u].x + g.alpha * re), sg * (iv[u].y + g.alpha * im));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(g.tmem_cols));
}

// ---------------------------------------------------------------------------------
// Host side of the tensor-copy GEMMs.

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// FP32 tensor map of `rank` dimensions (dims[0] contiguous; strides[i] in bytes between
// consecutive elements of dimension i + 1) with the given box and zero fill outside;
// false where the base or a stride is not 16-byte aligned or the encoder refuses it
bool encode_map(CUtensorMap &m, int rank, const void *base, const uint64_t *dims,
                const uint64_t *strides, const uint32_t *box) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn || reinterpret_cast<uintptr_t>(base) % 16) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    bx[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) {
      if (strides[i] % 16) return false;
      st[i] = strides[i];
    }
  }
  return fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void *>(base), d,
            st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// CTAs per SM the image GEMM sizes its shared memory for (TDLZ_NN_CTAS=1, 2 or 3; default
// 3): fewer CTAs keep more K tiles in flight each
int nn_img_ctas_per_sm() {
  const char *e = std::getenv("TDLZ_NN_CTAS");
  return (e && e[0] >= '1' && e[0] <= '3') ? e[0] - '0' : 3;
}

// whether the image GEMM fetches its In tile with a tensor copy where it can
// (TDLZ_NN_IN_TMA=1); by default it is read in the epilogue after an L2 prefetch, which
// leaves the shared memory to a deeper ring (at C2 shapes 122 against 131 us per launch)
bool nn_img_in_tma() {
  const char *e = std::getenv("TDLZ_NN_IN_TMA");
  return e && e[0] == '1';
}

}  // namespace

bool tc_gemm_tn(Context &ctx, DevBuf &partbuf, const float2 *A, long long lda, long long sA,
                int amod, const float2 *B, long long ldb, long long sB, float2 *C, long long sC,
                long long ldcm, long long ldcn, int M, int N, long long K, int batch) {
  if (M > 128 || M < 1 || N < 1 || K < 1 || amod < 1 || batch % amod != 0) return false;
  if (2 * M > 128)
    return tc_gemm_tn_transposed(ctx, partbuf, A, lda, sA, amod, B, ldb, sB, C, sC, ldcm, ldcn,
                                 M, N, K, batch);
  TcArgs g;
  g.A = A;
  g.lda = lda;
  g.sA = sA;
  g.amod = amod;
  g.B = B;
  g.ldb = ldb;
  g.sB = sB;
  g.M = M;
  g.N = N;
  g.K = K;
  g.nj = batch / amod;
  g.ntot = g.nj * N;
  g.ntiles = (g.ntot + 255) / 256;
  g.nt = ((g.ntot + g.ntiles - 1) / g.ntiles + 15) / 16 * 16;
  g.nkt = (int)((K + kKT / 2 - 1) / (kKT / 2));
  const int ctas = amod * g.ntiles;
  // about two waves of two CTAs per SM, within the split-K scratch
  const size_t per_split = (size_t)amod * g.ntiles * 128 * g.nt * sizeof(float);
  const long long fit = (long long)(partbuf.bytes / per_split);
  if (fit < 1) return false;
  long long ns = std::max(1, std::min(g.nkt, (4 * 152 + ctas - 1) / ctas));
  ns = std::min(ns, fit);
  g.kt_per_split = (int)((g.nkt + ns - 1) / ns);
  g.nsplit = (g.nkt + g.kt_per_split - 1) / g.kt_per_split;
  g.tmem_cols = 32;
  while (g.tmem_cols < (uint32_t)g.nt) g.tmem_cols *= 2;
  g.part = partbuf.as<float>();
  const size_t smem = 2 * (2 * (size_t)kATile + 2 * (size_t)g.nt * kKT * 4);
  TDLZ_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_tn_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(g.ntiles, amod, g.nsplit);
  tc_gemm_tn_kernel<<<grid, kTcThreads, smem, ctx.stream>>>(g);
  TDLZ_LAUNCH_CHECK();
  const long long total = (long long)batch * M * N;
  tc_reduce_kernel<<<blocks_for(total), 256, 0, ctx.stream>>>(g.part, C, M, N, amod, g.nj,
                                                               g.ntiles, g.nt, g.nsplit, sC,
                                                               ldcm, ldcn);
  TDLZ_LAUNCH_CHECK();
  return true;
}

bool tc_gemm_nn(Context &ctx, const float2 *A, long long sA, long long sar, long long sak,
                const float2 *B, long long ldb, long long sB, int bmod, const float2 *In,
                float2 *Out, long long ldo, long long sO, int rows, long long ncol, int K,
                float alpha, int batch, int neg_from, int neg_mod) {
  if (rows < 1 || K < 1 || ncol < 1 || batch < 1 || bmod < 1 || neg_mod < 1) return false;
  if (2 * rows > 256) {
    // more rows than the MMA's N holds (the V_NL update with 2 N_b > 128 rows): row
    // blocks of at most 128, each an independent launch on its own rows of A, In and Out
    for (int r0 = 0; r0 < rows; r0 += 128) {
      const int nr = std::min(128, rows - r0);
      if (!tc_gemm_nn(ctx, A + (long long)r0 * sar, sA, sar, sak, B, ldb, sB, bmod,
                      In + (long long)r0 * ldo, Out + (long long)r0 * ldo, ldo, sO, nr, ncol, K,
                      alpha, batch, neg_from, neg_mod))
        return false;
    }
    return true;
  }
  NnArgs g;
  g.A = A;
  g.sA = sA;
  g.sar = sar;
  g.sak = sak;
  g.B = B;
  g.ldb = ldb;
  g.sB = sB;
  g.bmod = bmod;
  g.In = In;
  g.Out = Out;
  g.ldo = ldo;
  g.sO = sO;
  g.ncol = ncol;
  g.R = rows;
  g.K = K;
  g.nm = (2 * rows + 15) / 16 * 16;
  g.nkt = (K + kNnKT / 2 - 1) / (kNnKT / 2);
  g.alpha = alpha;
  g.neg_from = neg_from;
  g.neg_mod = neg_mod;
  g.tmem_cols = 32;
  while (g.tmem_cols < (uint32_t)g.nm) g.tmem_cols *= 2;
  const size_t stage = 2 * (size_t)kNnM * kNnKT * 4 + 2 * (size_t)g.nm * kNnKT * 4;
  // no more CTAs per SM than the 512 TMEM columns hold: ask for enough shared memory
  // that one more would not fit either (228 KB per SM, 1 KB reserved per CTA)
  const int cap = (int)(512 / g.tmem_cols);
  const size_t smem = std::max(2 * stage, (size_t)(233472 / (cap + 1)));
  TDLZ_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_nn_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)((ncol + kNnM - 1) / kNnM), (unsigned)batch);
  tc_gemm_nn_kernel<<<grid, kTcThreads, smem, ctx.stream>>>(g);
  TDLZ_LAUNCH_CHECK();
  return true;
}

void tc_image_build(Context &ctx, TcImage &im, const float2 *B, long long ldb, long long sB,
                    int G, int K, long long ncol) {
  TDLZ_REQUIRE(G >= 1 && K >= 1 && ncol >= 1, TDLZ_ERR_ARG, "operand image: empty matrix");
  (void)tensor_map_encoder();  // resolve the encoder now, outside any stream capture
  im.G = G;
  im.K = K;
  im.ncol = ncol;
  im.nct = (int)((ncol + kNnM - 1) / kNnM);
  im.nkt = (K + kNnKT / 2 - 1) / (kNnKT / 2);
  const long long tiles = (long long)G * im.nct * im.nkt;
  im.buf.alloc((size_t)tiles * kAImgTile);
  nn_aimg_kernel<<<blocks_for(tiles * 512), 256, 0, ctx.stream>>>(B, ldb, sB, G, K, ncol, im.nct,
                                                                  im.nkt, im.buf.as<float4>());
  TDLZ_LAUNCH_CHECK();
}

bool tc_gemm_nn_img(Context &ctx, const TcImage &im, DevBuf &scratch, const float2 *A,
                    long long sA, long long sar, long long sak, const float2 *In, float2 *Out,
                    long long ldo, long long sO, int rows, float alpha, int batch, int neg_from,
                    int neg_mod) {
  const int G = im.G, nkt = im.nkt;
  if (!im.buf.p || rows < 1 || batch < 1 || G < 1 || batch % G != 0 || neg_mod < 1) return false;
  const bool tma_ok = nn_img_in_tma() && reinterpret_cast<uintptr_t>(In) % 16 == 0 &&
                      ldo % 2 == 0 && sO % 2 == 0 && tensor_map_encoder() != nullptr;
  // CTAs per SM: as asked, but no more than the 512 TMEM columns hold (the accumulator of
  // 2R <= 256 columns is rounded up to a power of two)
  int cps = nn_img_ctas_per_sm();
  {
    uint32_t cols = 32;
    while (cols < (uint32_t)((2 * std::min(rows, 128) + 15) / 16 * 16)) cols *= 2;
    cps = std::min(cps, (int)(512 / cols));
  }
  const long long budget = 233472 / cps - 2048;  // per-CTA reserve + static
  auto stages = [&](int R, bool tma) {
    const int nm = (2 * R + 15) / 16 * 16;
    const long long in_b = tma ? (long long)R * 1024 : 0;
    return (int)std::min<long long>(std::min<long long>(nkt, kNnMaxStages),
                                    (budget - in_b) / (kAImgTile + 128LL * nm));
  };
  // row blocks of at most 128 rows: as few as leave a ring of two stages (all K tiles
  // where there are fewer)
  int R = 0;
  for (int nblk = (rows + 127) / 128; nblk <= rows; ++nblk) {
    const int r = (rows + nblk - 1) / nblk;
    if (stages(r, tma_ok) >= std::min(2, nkt)) {
      R = r;
      break;
    }
  }
  if (R == 0) return false;
  {
    const int nm = (2 * R + 15) / 16 * 16;
    if (scratch.bytes < (size_t)batch * nkt * 128 * nm) return false;
  }
  for (int r0 = 0; r0 < rows; r0 += R) {
    const int nr = std::min(R, rows - r0);
    NnImgArgs g{};
    g.aimg = im.buf.as<unsigned char>();
    g.bimg = scratch.as<unsigned char>();
    g.In = In + (long long)r0 * ldo;
    g.Out = Out + (long long)r0 * ldo;
    g.ldo = ldo;
    g.sO = sO;
    g.ncol = im.ncol;
    g.R = nr;
    g.nm = (2 * nr + 15) / 16 * 16;
    g.nkt = nkt;
    g.nct = im.nct;
    g.G = G;
    g.nj = batch / G;
    g.alpha = alpha;
    g.neg_from = neg_from;
    g.neg_mod = neg_mod;
    g.tmem_cols = 32;
    while (g.tmem_cols < (uint32_t)g.nm) g.tmem_cols *= 2;
    alignas(64) CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    {
      const uint64_t dims[3] = {2 * (uint64_t)im.ncol, (uint64_t)nr, (uint64_t)batch};
      const uint64_t str[2] = {(uint64_t)ldo * 8, (uint64_t)sO * 8};
      const uint32_t box[3] = {256, (uint32_t)nr, 1};
      g.in_tma = tma_ok && encode_map(map, 3, g.In, dims, str, box);
    }
    g.in_bytes = g.in_tma ? (uint32_t)nr * 1024 : 0;
    g.S = stages(nr, g.in_tma);
    g.stage_bytes = kAImgTile + 128u * (uint32_t)g.nm;
    nn_bimg_kernel<<<blocks_for((long long)batch * nkt * 2 * g.nm), 256, 0, ctx.stream>>>(
        A + (long long)r0 * sar, sA, sar, sak, nr, im.K, nkt, g.nm, batch, scratch.as<float4>());
    TDLZ_LAUNCH_CHECK();
    // no more CTAs per SM than the 512 TMEM columns hold: ask for enough shared memory
    // that one more would not fit either
    const int cap = (int)(512 / g.tmem_cols);
    const size_t smem = std::max((size_t)g.in_bytes + (size_t)g.S * g.stage_bytes,
                                 (size_t)(233472 / (cap + 1)));
    TDLZ_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_nn_img_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long nblocks = (long long)im.nct * batch;
    tc_gemm_nn_img_kernel<<<(unsigned)nblocks, kTcThreads, smem, ctx.stream>>>(map, g);
    TDLZ_LAUNCH_CHECK();
  }
  return true;
}

void tc_gemm_inject_timeout(int n) {
  TDLZ_CUDA_TRY(cudaMemcpyToSymbol(g_tc_inject, &n, sizeof(int)));
}

void tc_gemm_check() {
  int flag = 0;
  TDLZ_CUDA_TRY(cudaMemcpyFromSymbol(&flag, g_tc_timeout, sizeof(int)));
  if (flag) {
    int zero = 0;
    TDLZ_CUDA_TRY(cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int)));
    throw Error{TDLZ_ERR_TIMEOUT, "tensor-core GEMM: an mbarrier wait ran out (results invalid)"};
  }
}

}  // namespace tdlz
