// Fused plane-by-plane real-space stages of the Liouvillian.
//
// After the inverse Z pass over the sphere's sticks (pipeline.cu; stick buffer
// i1t[row][j3][stick]) every remaining transform of a band-side acts on one z plane
// at a time, and so do the pointwise stages.  Two passes, each one CTA per
// (vector, z plane, chunk of band-sides), looping over the chunk one band-side at a
// time:
//
//   A (density)   inverse Y lines over the sphere's planes (shared memory), inverse
//                 X lines (registers), then the response densities
//                 rho'_a += w t_a U^+ sigma_a x  (Eqs. charge_dens_resp_q,
//                 spin_dens_resp_q; t = (1,-1,-1,-1) on the Y side) summed in
//                 registers over the chunk; one partial density per chunk reaches HBM.
//   B (products)  the same inverse lines again, t = [v_loc + s B.sigma] x + W^s U
//                 (W^X = v'_0 + v'.sigma, W^Y = v'_0 - v'.sigma; the D and K blocks
//                 after Eq. Liouvillian_BR_q) in registers, forward X lines keeping
//                 the sphere's planes, forward Y lines keeping its sticks, written
//                 back into i1t in place for the forward Z pass.
//
// x(r) never reaches HBM: pass B recomputes the inverse lines of a band-side plane
// instead of reading a stored grid (storing would move a write and a read of every
// band-side's full grid, ~15 GB per pass on the 36x36x96 workload).  Per band-side
// plane a pass reads its sticks and its U slab plane; the potential plane of the
// CTA's vector is read once per CTA.
//
// Lines over lanes: a line of length N = NL * N2 is split over NL neighbouring lanes
// (four-step).  Inverse (decimation in time): lane n1 holds x[n1 + NL n2], transforms
// over n2 in registers, multiplies by w_N^(n1 k2) and a cross-lane NL-point DFT leaves
// it holding the block X[N2 kb + k2] (kb = bit-reversed n1 for NL = 4, n1 for NL = 5).
// Forward (decimation in frequency) runs the same steps in reverse order from that
// block layout and leaves lane n1 holding X[n1 + NL m2].  In the X phase the lanes
// (column c, spinor row sp, n1) sit at 2 NL c' + NL sp + n1 of a warp, so the two
// spinor components of a point are one shuffle apart, and each thread owns the same
// points of the plane for the whole chunk.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <functional>

#include "planes.cuh"
#include "regfft.cuh"

namespace tdlz {

namespace {

struct PlTables {
  const int *pl_n;   // [nk] planes per k
  const int *pl_of;  // [nk][N] plane index of j1 or -1
  const int *st_id;  // [nk][npm][N] stick index of (plane, j2) or -1
  int nsm, npm, n3, nk, nb;
  long long nnp;     // plane stride of the U slabs and potential planes
};

PlTables tables_of(const QSlot &s) {
  PlTables tb;
  tb.pl_n = s.pl_n.as<int>();
  tb.pl_of = s.pl_of.as<int>();
  tb.st_id = s.st_id.as<int>();
  tb.nsm = s.nstick_max;
  tb.npm = s.nplane_max;
  tb.n3 = s.fft[2];
  tb.nk = s.nk;
  tb.nb = s.nb;
  tb.nnp = planes_nnp(s);
  return tb;
}

// Split of a line of length N over NL lanes of N2 points (NL = 2, or 3 for odd N);
// columns and lines per warp; warps per band-side (all columns of both spinor rows).
template <int N> struct Lay {
  static constexpr int NL = N % 2 == 0 ? 2 : 3;
  static constexpr int N2 = N / NL;
  static constexpr int CPW = 32 / (2 * NL);  // columns per warp in the X phase
  static constexpr int GPW = 32 / NL;        // lines per warp in the Y phases
  static constexpr int WPB = (N + CPW - 1) / CPW;
  static constexpr int THREADS = 32 * WPB;
  static constexpr int NM = (N2 + 1) / 2;   // points of a lane's block it owns
  static_assert(N2 * NL == N, "line split");
};
// CTAs per SM the FP32 register budget is sized for (FP64 is bound by its arithmetic
// rate, not by occupancy)
template <class T, int N> constexpr int min_ctas() {
  return sizeof(T) == 8 ? 1 : Lay<N>::THREADS <= 160 ? 3 : Lay<N>::THREADS <= 288 ? 2 : 1;
}

// Per-lane constants of the lane-split line transforms: the lane's position n1 in its
// group (it holds block n1 of a line after an inverse transform), and for NL = 3 the
// source lanes and coefficients of the cross-lane 3-point DFT.
template <class T, int N> struct LaneCtx {
  int n1;
  T s2;          // NL = 2: sign of the own value in the cross-lane butterfly
  int src[3];    // NL = 3: source lane of offset d in the group
  cx<T> cw[3];   // NL = 3: w_3^((n1 + d) % 3 * n1)
};

template <class T, int N>
__device__ __forceinline__ LaneCtx<T, N> lane_ctx(int lane, const RegTw<T, 3> &tw3) {
  using L = Lay<N>;
  LaneCtx<T, N> c;
  c.n1 = lane % L::NL;
  c.s2 = c.n1 ? T(-1) : T(1);
  if constexpr (L::NL == 3) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int a = (c.n1 + d) % 3;
      c.src[d] = lane - c.n1 + a;
      c.cw[d] = tw3.w[(a * c.n1) % 3];
    }
  }
  return c;
}

template <class T> __device__ __forceinline__ cx<T> shfl_idx(cx<T> v, int src) {
  cx<T> r;
  r.x = __shfl_sync(0xffffffffu, v.x, src);
  r.y = __shfl_sync(0xffffffffu, v.y, src);
  return r;
}
template <class T> __device__ __forceinline__ cx<T> shfl_xor(cx<T> v, int m) {
  cx<T> r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return r;
}

// Cross-lane NL-point DFT of every register; lane n1 holds input n1 and ends with
// output n1.  NL = 2: (a0 + a1, a0 - a1).  NL = 3: each lane forms its own output.
template <class T, int N, int M, bool INV>
__device__ __forceinline__ void cross_lanes(cx<T> (&a)[M], const LaneCtx<T, N> &c) {
  if constexpr (Lay<N>::NL == 2) {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const cx<T> p = shfl_xor<T>(a[k], 1);
      a[k] = mk<T>(fma(c.s2, a[k].x, p.x), fma(c.s2, a[k].y, p.y));
    }
  } else {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const cx<T> x = a[k];
      const cx<T> v1 = shfl_idx<T>(x, c.src[1]), v2 = shfl_idx<T>(x, c.src[2]);
      cx<T> w0 = c.cw[0], w1 = c.cw[1], w2 = c.cw[2];
      if (!INV) {
        w0.y = -w0.y;
        w1.y = -w1.y;
        w2.y = -w2.y;
      }
      cx<T> acc = cmul<T>(w0, x);
      cfma<T>(acc, w1, v1);
      cfma<T>(acc, w2, v2);
      a[k] = acc;
    }
  }
}

// four-step factor w_N^(n1 k) of the lane (1 for n1 = 0), DIR < 0 conjugated
template <class T, int N, int DIR>
__device__ __forceinline__ cx<T> lane_tw(const RegTw<T, N> &twn, int n1, int k) {
  cx<T> w;
  if constexpr (Lay<N>::NL == 2) {
    const cx<T> t = twn.w[k % N];
    w = n1 ? t : mk<T>(T(1), T(0));
  } else {
    const cx<T> t1 = twn.w[k % N], t2 = twn.w[(2 * k) % N];
    w = n1 == 0 ? mk<T>(T(1), T(0)) : n1 == 1 ? t1 : t2;
  }
  if (DIR < 0) w.y = -w.y;
  return w;
}

// Inverse line (DIT): a[n2] = x[n1 + NL n2] in, a[k2] = X[N2 n1 + k2] out.
template <class T, int N>
__device__ __forceinline__ void line_inverse(cx<T> (&a)[Lay<N>::N2], const LaneCtx<T, N> &c,
                                             const RegTw<T, Lay<N>::N2> &tw2,
                                             const RegTw<T, N> &twn) {
  constexpr int N2 = Lay<N>::N2;
  RegPlan<N2>::template run<T, +1>(a, tw2);
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) a[k2] = cmul<T>(a[k2], lane_tw<T, N, +1>(twn, c.n1, k2));
  cross_lanes<T, N, N2, true>(a, c);
}

// Forward line (DIF): a[b] = t[N2 n1 + b] in, a[m2] = X[n1 + NL m2] out.
template <class T, int N>
__device__ __forceinline__ void line_forward(cx<T> (&a)[Lay<N>::N2], const LaneCtx<T, N> &c,
                                             const RegTw<T, Lay<N>::N2> &tw2,
                                             const RegTw<T, N> &twn) {
  constexpr int N2 = Lay<N>::N2;
  cross_lanes<T, N, N2, false>(a, c);
#pragma unroll
  for (int b = 1; b < N2; ++b) a[b] = cmul<T>(a[b], lane_tw<T, N, -1>(twn, c.n1, b));
  RegPlan<N2>::template run<T, -1>(a, tw2);
}

// Twiddles of one line length: the per-lane register part, the four-step factors and
// the cross-lane 3-point DFT.
template <class T, int N> struct LineTw {
  RegTw<T, Lay<N>::N2> tw2;
  RegTw<T, N> twn;
  RegTw<T, 3> tw3;
};
template <class T, int N> LineTw<T, N> line_tw() {
  LineTw<T, N> t;
  t.tw2 = regtw<T, Lay<N>::N2>();
  t.twn = regtw<T, N>();
  t.tw3 = regtw<T, 3>();
  return t;
}

// 16-byte asynchronous global -> shared copies (no registers, no wait loop: the
// issuing thread waits with cp.async.wait_group, the block with a barrier)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// One stage: the sticks of plane j3 of both spinor rows of band-side bs -> st[spin][nsm]
// and, with SU, their U slab planes -> u[spin][nnp] (u = st + 2 nsm).
__host__ __device__ constexpr long long stage_elems(long long nsm, long long nnp, bool su) {
  return 2 * (nsm + (su ? nnp : 0));
}
template <class T, bool SU>
__device__ __forceinline__ void stage_copy(cx<T> *st, const cx<T> *__restrict__ i1t,
                                           const cx<T> *__restrict__ us, const PlTables &tb,
                                           long long row0, long long urow0, int j3) {
  constexpr int E = 16 / (int)sizeof(cx<T>);  // complex elements per 16-byte chunk
  const int cs = tb.nsm / E;
  const long long rstride = (long long)tb.n3 * tb.nsm;
  for (int e = threadIdx.x; e < 2 * cs; e += blockDim.x) {
    const int spp = e >= cs, ch = e - spp * cs;
    cp_async16(st + spp * tb.nsm + ch * E,
               i1t + (row0 + spp) * rstride + (long long)j3 * tb.nsm + ch * E);
  }
  if constexpr (SU) {
    const int cu = (int)(tb.nnp / E);
    const long long uplane = (long long)tb.n3 * tb.nnp;
    cx<T> *u = st + 2 * tb.nsm;
    for (int e = threadIdx.x; e < 2 * cu; e += blockDim.x) {
      const int spp = e >= cu, ch = e - spp * cu;
      cp_async16(u + spp * tb.nnp + ch * E,
                 us + (urow0 + spp) * uplane + (long long)j3 * tb.nnp + ch * E);
    }
  }
}

// Inverse Y lines of one band-side (both spinor rows, every plane of its k): staged
// sticks st -> Yi[spin][plane][YP].  Every lane of a warp with a line takes part in
// the warp's rounds (shuffles).
template <class T, int N>
__device__ __forceinline__ void inverse_y_lines(const cx<T> *st, cx<T> *Yi, const PlTables &tb,
                                                int k, int npl, const LaneCtx<T, N> &c,
                                                const LineTw<T, N> &tw) {
  using L = Lay<N>;
  constexpr int YP = N + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane / L::NL;
  const int nw = blockDim.x >> 5, nyl = 2 * tb.npm;
  const int per_round = nw * L::GPW, rounds = (nyl + per_round - 1) / per_round;
  for (int r = 0; r < rounds; ++r) {
    if (r * per_round + warp * L::GPW >= nyl) break;  // no line for this warp (uniform)
    const int line = r * per_round + warp * L::GPW + g;
    const int spp = line >= tb.npm, p = line - spp * tb.npm;  // line < 2 npm when ok
    const bool ok = g < L::GPW && line < nyl && p < npl;
    const int *sd = tb.st_id + ((long long)k * tb.npm + (ok ? p : 0)) * N + c.n1;
    const cx<T> *src = st + (ok ? spp : 0) * tb.nsm;
    cx<T> a[L::N2];
#pragma unroll
    for (int n2 = 0; n2 < L::N2; ++n2) {
      const int sidx = ok ? __ldg(sd + L::NL * n2) : -1;
      a[n2] = sidx >= 0 ? src[sidx] : czero<T>();
    }
    line_inverse<T, N>(a, c, tw.tw2, tw.twn);
    if (ok) {
      cx<T> *o = Yi + (spp * tb.npm + p) * YP + L::N2 * c.n1;
#pragma unroll
      for (int k2 = 0; k2 < L::N2; ++k2) o[k2] = a[k2];
    }
  }
}

// Exchange with the pair lane (the other spinor row of the column) for the owned
// points: lane sp owns k2 = 2m + sp of its block; it sends the value at the partner's
// point and receives the partner's value at its own.  Returns the partner's value.
template <class T, int N, int M>
__device__ __forceinline__ cx<T> pair_swap(const cx<T> (&a)[M], int m, int sp, int partner) {
  const int e0 = 2 * m, e1 = 2 * m + 1 < M ? 2 * m + 1 : 2 * m;
  const cx<T> send = sp ? a[e0] : a[e1];
  return Lay<N>::NL == 2 ? shfl_xor<T>(send, 2) : shfl_idx<T>(send, partner);
}

// ------------------------------------------------------------------ pass A
template <class T, int N>
__global__ void __launch_bounds__(Lay<N>::THREADS, (min_ctas<T, N>()))
    plane_density_kernel(const cx<T> *__restrict__ i1t, const cx<T> *__restrict__ us,
                         const T *__restrict__ wk, cx<T> *__restrict__ part, PlTables tb,
                         int nvec, int chunk_len, const LineTw<T, N> tw) {
  using L = Lay<N>;
  constexpr int N2 = L::N2, NN = N * N, YP = N + 1, NM = L::NM;
  extern __shared__ float4 pl_smem[];
  cx<T> *Yi = reinterpret_cast<cx<T> *>(pl_smem);  // [2][npm][YP]
  cx<T> *stg = Yi + 2 * tb.npm * YP;                 // 2 stages: sticks [2][nsm], U [2][nnp]
  const long long sz = stage_elems(tb.nsm, tb.nnp, true);
  const int v = blockIdx.x % nvec, ch = blockIdx.x / nvec, j3 = blockIdx.y;
  const long long nbs1 = 2LL * tb.nk * tb.nb, rows1 = 2 * nbs1;
  const long long bsb = (long long)ch * chunk_len;
  const long long bse = bsb + chunk_len < nbs1 ? bsb + chunk_len : nbs1;
  const long long vrow = (long long)v * rows1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LaneCtx<T, N> lc = lane_ctx<T, N>(lane, tw.tw3);
  // X-phase role: column col of spinor row sp, block n1; the pair lane holds the other row
  const int cq = lane / (2 * L::NL), sp = (lane / L::NL) & 1;
  const int col = warp * L::CPW + cq;
  const bool xv = cq < L::CPW && col < N;
  const int partner = L::NL == 2 ? (lane ^ 2) : (!xv ? lane : sp ? lane - 3 : lane + 3);
  const int colc = xv ? col : 0;
  cx<T> acc[NM][4];
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int a_ = 0; a_ < 4; ++a_) acc[m][a_] = czero<T>();
  if (bsb < bse) stage_copy<T, true>(stg, i1t, us, tb, vrow + 2 * bsb, 2 * bsb, j3);
  cp_async_commit();
  // band-side bs = (side nk + k) nb + n, advanced incrementally
  int n = (int)(bsb % tb.nb), k = (int)((bsb / tb.nb) % tb.nk);
  int side = (int)(bsb / ((long long)tb.nk * tb.nb));
  int it = 0;
  for (long long bs = bsb; bs < bse; ++bs, ++it) {
    const cx<T> *st = stg + (it & 1) * sz;
    if (bs + 1 < bse)
      stage_copy<T, true>(stg + ((it + 1) & 1) * sz, i1t, us, tb, vrow + 2 * (bs + 1),
                          2 * (bs + 1), j3);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    const int npl = __ldg(tb.pl_n + k);
    inverse_y_lines<T, N>(st, Yi, tb, k, npl, lc, tw);
    __syncthreads();
    const cx<T> *u0p = st + 2 * tb.nsm + colc, *u1p = u0p + tb.nnp;  // staged U planes
    cx<T> a[N2];
    {
      const int *po = tb.pl_of + (long long)k * N + lc.n1;
      const cx<T> *src = Yi + sp * tb.npm * YP + colc;
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        const int p = xv ? __ldg(po + L::NL * n2) : -1;
        a[n2] = p >= 0 ? src[p * YP] : czero<T>();
      }
    }
    line_inverse<T, N>(a, lc, tw.tw2, tw.twn);
    const T w = wk[k], wt = side == 0 ? w : -w;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const cx<T> recv = pair_swap<T, N, N2>(a, m, sp, partner);
      const int e0 = 2 * m, e1 = 2 * m + 1 < N2 ? 2 * m + 1 : 2 * m;
      const cx<T> own = sp ? a[e1] : a[e0];
      const cx<T> x0 = sp ? recv : own, x1 = sp ? own : recv;
      const int k2 = 2 * m + sp;
      const int i = (N2 * lc.n1 + (k2 < N2 ? k2 : 0)) * N;
      const cx<T> u0 = u0p[i], u1 = u1p[i];
      const cx<T> p00 = cmulc<T>(u0, x0), p01 = cmulc<T>(u0, x1);
      const cx<T> p10 = cmulc<T>(u1, x0), p11 = cmulc<T>(u1, x1);
      const cx<T> d = csub<T>(p10, p01);  // m_y: i (p10 - p01)
      acc[m][0] = cadd<T>(acc[m][0], cscale<T>(cadd<T>(p00, p11), w));
      acc[m][1] = cadd<T>(acc[m][1], cscale<T>(cadd<T>(p01, p10), wt));
      acc[m][2] = cadd<T>(acc[m][2], cscale<T>(mk<T>(-d.y, d.x), wt));
      acc[m][3] = cadd<T>(acc[m][3], cscale<T>(csub<T>(p00, p11), wt));
    }
    if (++n == tb.nb) {
      n = 0;
      if (++k == tb.nk) {
        k = 0;
        ++side;
      }
    }
    __syncthreads();  // Yi and this stage's sticks are rewritten by the next iteration
  }
  // this chunk's partial density of plane j3: every point written by its one owner
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    const int k2 = 2 * m + sp;
    if (xv && k2 < N2) {
      const int i = (N2 * lc.n1 + k2) * N + col;
#pragma unroll
      for (int a_ = 0; a_ < 4; ++a_)
        part[(((long long)ch * nvec + v) * 4 + a_) * tb.n3 * NN + (long long)j3 * NN + i] =
            acc[m][a_];
    }
  }
}

// rho[v][a][i*n3 + j3] = sum_c part[c][v][a][j3][i] in fixed order
template <class T>
__global__ void plane_reduce_kernel(const cx<T> *__restrict__ part, cx<T> *__restrict__ rho,
                                    int nchunk, long long nn, int n3, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    cx<T> s = part[e];
    for (int c = 1; c < nchunk; ++c) s = cadd<T>(s, part[(long long)c * total + e]);
    const long long plane = nn * n3;
    const long long va = e / plane, rem = e - va * plane;
    const long long j3 = rem / nn, i = rem - j3 * nn;
    rho[va * plane + i * n3 + j3] = s;
  }
}

// ------------------------------------------------------------------ potential
// v_a = delta_a0 vH + sum_b f_ab rho_b (f packed 00,01,02,03,11,12,13,22,23,33), written
// with (v_loc, B_z) and (B_x, B_y) as the potential plane pot[v][j3][6][nnp].
template <class T>
__global__ void potential_planes_kernel(const cx<T> *__restrict__ rho, const cx<T> *__restrict__ vh,
                                        const T *__restrict__ f, const T *__restrict__ vloc,
                                        const T *__restrict__ bf, cx<T> *__restrict__ pot,
                                        long long nr, int n3, long long nnp, int use_h,
                                        int use_xc, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long v = e / nr, r = e - v * nr;
    const long long i = r / n3, j3 = r - i * n3;
    cx<T> out[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
    if (use_xc) {
      cx<T> p[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) p[a] = rho[(v * 4 + a) * nr + r];
      T fm[4][4];
      int q = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b) {
          const T val = f[q++ * nr + r];
          fm[a][b] = val;
          fm[b][a] = val;
        }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          out[a].x += fm[a][b] * p[b].x;
          out[a].y += fm[a][b] * p[b].y;
        }
    }
    if (use_h) out[0] = cadd<T>(out[0], vh[v * nr + r]);
    cx<T> *o = pot + (v * n3 + j3) * 6 * nnp + i;
#pragma unroll
    for (int a = 0; a < 4; ++a) o[a * nnp] = out[a];
    o[4 * nnp] = mk<T>(vloc[r], bf[2 * nr + r]);
    o[5 * nnp] = mk<T>(bf[r], bf[nr + r]);
  }
}

// ------------------------------------------------------------------ pass B
// PS: the CTA's potential plane staged in shared memory (else read through L1); SU: the
// U planes staged with the sticks (else loaded into registers before the X lines).
template <class T, int N, bool PS, bool SU>
__global__ void __launch_bounds__(Lay<N>::THREADS, (min_ctas<T, N>()))
    plane_product_fwd_kernel(cx<T> *__restrict__ i1t, const cx<T> *__restrict__ us,
                             const cx<T> *__restrict__ pot, PlTables tb, int nvec,
                             int chunk_len, const LineTw<T, N> tw) {
  using L = Lay<N>;
  constexpr int N2 = L::N2, NN = N * N, YP = N + 1, NM = L::NM;
  extern __shared__ float4 pl_smem[];
  cx<T> *Yi = reinterpret_cast<cx<T> *>(pl_smem);  // [2][npm][YP] inverse Y lines
  cx<T> *Yf = Yi + 2 * tb.npm * YP;                  // [2][npm][YP] forward X lines
  cx<T> *stg = Yf + 2 * tb.npm * YP;                 // 2 stages: sticks, U when SU
  const long long sz = stage_elems(tb.nsm, tb.nnp, SU);
  cx<T> *P = stg + 2 * sz;                           // [6][NN] when PS
  const int v = blockIdx.x % nvec, ch = blockIdx.x / nvec, j3 = blockIdx.y;
  const long long nbs1 = 2LL * tb.nk * tb.nb, rows1 = 2 * nbs1;
  const long long bsb = (long long)ch * chunk_len;
  const long long bse = bsb + chunk_len < nbs1 ? bsb + chunk_len : nbs1;
  const long long vrow = (long long)v * rows1;
  const long long uplane = (long long)tb.n3 * tb.nnp, rstride = (long long)tb.n3 * tb.nsm;
  if (bsb < bse) stage_copy<T, SU>(stg, i1t, us, tb, vrow + 2 * bsb, 2 * bsb, j3);
  cp_async_commit();
  const cx<T> *pg = pot + ((long long)v * tb.n3 + j3) * 6 * tb.nnp;
  if constexpr (PS) {
    for (int e = threadIdx.x; e < 6 * NN; e += blockDim.x) {
      const int cc = e / NN, i = e - cc * NN;
      P[e] = pg[cc * tb.nnp + i];
    }
  }
  const cx<T> *pp = PS ? P : pg;
  const long long pst = PS ? (long long)NN : tb.nnp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LaneCtx<T, N> lc = lane_ctx<T, N>(lane, tw.tw3);
  const int cq = lane / (2 * L::NL), sp = (lane / L::NL) & 1;
  const int col = warp * L::CPW + cq;
  const bool xv = cq < L::CPW && col < N;
  const int partner = L::NL == 2 ? (lane ^ 2) : (!xv ? lane : sp ? lane - 3 : lane + 3);
  const int colc = xv ? col : 0;
  // band-side bs = (side nk + k) nb + n, advanced incrementally
  int n = (int)(bsb % tb.nb), k = (int)((bsb / tb.nb) % tb.nk);
  int side = (int)(bsb / ((long long)tb.nk * tb.nb));
  int it = 0;
  for (long long bs = bsb; bs < bse; ++bs, ++it) {
    const cx<T> *st = stg + (it & 1) * sz;
    if (bs + 1 < bse)
      stage_copy<T, SU>(stg + ((it + 1) & 1) * sz, i1t, us, tb, vrow + 2 * (bs + 1),
                        2 * (bs + 1), j3);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    const int npl = __ldg(tb.pl_n + k);
    inverse_y_lines<T, N>(st, Yi, tb, k, npl, lc, tw);
    // U of both rows at the owned points (j1 = N2 n1 + k2, k2 = sp, sp + 2, ...)
    cx<T> u[NM][2];
    if constexpr (!SU) {
      const cx<T> *ub = us + (2 * bs * tb.n3 + j3) * tb.nnp + colc;
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const int k2 = 2 * m + sp;
        const bool ok = xv && k2 < N2;
        const int i = (N2 * lc.n1 + (k2 < N2 ? k2 : 0)) * N;
        u[m][0] = ok ? __ldg(ub + i) : czero<T>();
        u[m][1] = ok ? __ldg(ub + uplane + i) : czero<T>();
      }
    }
    __syncthreads();
    const int *po = tb.pl_of + (long long)k * N + lc.n1;
    cx<T> a[N2];
    {
      const cx<T> *src = Yi + sp * tb.npm * YP + colc;
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        const int p = xv ? __ldg(po + L::NL * n2) : -1;
        a[n2] = p >= 0 ? src[p * YP] : czero<T>();
      }
    }
    line_inverse<T, N>(a, lc, tw.tw2, tw.twn);
    {
      // both rows of [v_loc + s B.sigma] x + W^s U at the owned points, then the pair
      // swaps so that each lane holds its own row at every point of its block:
      //   t0 = (vl + s Bz) x0 + s(Bx - i By) x1 + (v0 + s v3) u0 + s(v1 - i v2) u1
      //   t1 = s(Bx + i By) x0 + (vl - s Bz) x1 + s(v1 + i v2) u0 + (v0 - s v3) u1
      const T s = side == 0 ? T(1) : T(-1);
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const cx<T> recv = pair_swap<T, N, N2>(a, m, sp, partner);
        const int e0 = 2 * m, e1 = 2 * m + 1 < N2 ? 2 * m + 1 : 2 * m;
        const cx<T> own = sp ? a[e1] : a[e0];
        const cx<T> x0 = sp ? recv : own, x1 = sp ? own : recv;
        const int k2 = 2 * m + sp;
        const int i = (N2 * lc.n1 + (k2 < N2 ? k2 : 0)) * N + colc;
        const cx<T> v0 = pp[i], v1 = pp[pst + i], v2 = pp[2 * pst + i], v3 = pp[3 * pst + i];
        const cx<T> lz = pp[4 * pst + i], bxy = pp[5 * pst + i];
        cx<T> u0, u1;
        if constexpr (SU) {
          const cx<T> *uq = st + 2 * tb.nsm + i;
          u0 = uq[0];
          u1 = uq[tb.nnp];
        } else {
          u0 = u[m][0];
          u1 = u[m][1];
        }
        const T sbx = s * bxy.x, sby = s * bxy.y, sbz = s * lz.y;
        cx<T> t0 = cscale<T>(x0, lz.x + sbz);
        cfma<T>(t0, mk<T>(sbx, -sby), x1);
        cfma<T>(t0, mk<T>(v0.x + s * v3.x, v0.y + s * v3.y), u0);
        cfma<T>(t0, mk<T>(s * (v1.x + v2.y), s * (v1.y - v2.x)), u1);
        cx<T> t1 = cscale<T>(x1, lz.x - sbz);
        cfma<T>(t1, mk<T>(sbx, sby), x0);
        cfma<T>(t1, mk<T>(s * (v1.x - v2.y), s * (v1.y + v2.x)), u0);
        cfma<T>(t1, mk<T>(v0.x - s * v3.x, v0.y - s * v3.y), u1);
        // keep this row's product; send the partner's row, receive this row at the
        // partner's point
        const cx<T> mine = sp ? t1 : t0, theirs = sp ? t0 : t1;
        const cx<T> back = Lay<N>::NL == 2 ? shfl_xor<T>(theirs, 2) : shfl_idx<T>(theirs, partner);
        // (odd N2: the last pair has one point, 2m, owned by row 0; row 1 takes it back)
        if (sp) {
          a[e0] = back;
          if (e1 != e0) a[e1] = mine;
        } else {
          a[e0] = mine;
          if (e1 != e0) a[e1] = back;
        }
      }
    }
    line_forward<T, N>(a, lc, tw.tw2, tw.twn);
    if (xv) {
      cx<T> *dst = Yf + sp * tb.npm * YP + col;
#pragma unroll
      for (int m2 = 0; m2 < N2; ++m2) {
        const int p = __ldg(po + L::NL * m2);
        if (p >= 0) dst[p * YP] = a[m2];
      }
    }
    __syncthreads();
    // forward Y lines keep the sphere's sticks, written back in place
    {
      const int g = lane / L::NL, nw = blockDim.x >> 5, nyl = 2 * tb.npm;
      const int per_round = nw * L::GPW, rounds = (nyl + per_round - 1) / per_round;
      for (int r = 0; r < rounds; ++r) {
        if (r * per_round + warp * L::GPW >= nyl) break;  // no line for this warp (uniform)
        const int line = r * per_round + warp * L::GPW + g;
        const int spp = line >= tb.npm, p = line - spp * tb.npm;  // line < 2 npm when ok
        const bool ok = g < L::GPW && line < nyl && p < npl;
        const cx<T> *src = Yf + ((ok ? spp : 0) * tb.npm + (ok ? p : 0)) * YP + N2 * lc.n1;
        cx<T> y[N2];
#pragma unroll
        for (int b = 0; b < N2; ++b) y[b] = ok ? src[b] : czero<T>();
        line_forward<T, N>(y, lc, tw.tw2, tw.twn);
        if (ok) {
          const int *sd = tb.st_id + ((long long)k * tb.npm + p) * N + lc.n1;
          cx<T> *dst = i1t + (vrow + 2 * bs + spp) * rstride + (long long)j3 * tb.nsm;
#pragma unroll
          for (int m2 = 0; m2 < N2; ++m2) {
            const int sidx = __ldg(sd + L::NL * m2);
            if (sidx >= 0) dst[sidx] = y[m2];
          }
        }
      }
    }
    if (++n == tb.nb) {
      n = 0;
      if (++k == tb.nk) {
        k = 0;
        ++side;
      }
    }
    __syncthreads();  // Yi, Yf and this stage's sticks are rewritten by the next iteration
  }
}

// ------------------------------------------------------------------ U slabs
template <class T>
__global__ void u_slab_kernel(const double2 *__restrict__ ur, cx<T> *__restrict__ us,
                              long long nn, int n3, long long nnp, long long nr,
                              long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long plane = (long long)n3 * nnp;
    const long long row = e / plane, rem = e - row * plane;
    const long long j3 = rem / nnp, i = rem - j3 * nnp;
    cx<T> o = czero<T>();
    if (i < nn) {
      const double2 u = ur[row * nr + i * n3 + j3];
      o = mk<T>((T)u.x, (T)u.y);
    }
    us[e] = o;
  }
}

template <class T>
__global__ void grid_from_slab_kernel(const double2 *__restrict__ us, cx<T> *__restrict__ ur,
                                      long long nn, int n3, long long nnp, long long nr,
                                      long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / nr, r = e - row * nr;
    const long long i = r / n3, j3 = r - i * n3;
    const double2 u = us[(row * n3 + j3) * nnp + i];
    ur[e] = mk<T>((T)u.x, (T)u.y);
  }
}

// -------------------------------------------------------------- dispatch
int threads_of(int n) {
  switch (n) {
    case 12: return Lay<12>::THREADS;
    case 16: return Lay<16>::THREADS;
    case 24: return Lay<24>::THREADS;
    case 36: return Lay<36>::THREADS;
    case 45: return Lay<45>::THREADS;
    case 48: return Lay<48>::THREADS;
    default: return 0;
  }
}

template <class T> size_t smem_density(const QSlot &s) {
  return ((size_t)2 * s.nplane_max * (s.fft[0] + 1) +
          2 * stage_elems(s.nstick_max, planes_nnp(s), true)) *
         sizeof(cx<T>);
}
// pass B launch shapes (equal results; the autotuner picks one), coded 2 * (U planes
// staged) + (potential plane in shared memory)
template <class T> size_t smem_product(const QSlot &s, int code) {
  const long long nn = (long long)s.fft[0] * s.fft[1];
  const bool ps = code & 1, su = code & 2;
  return ((size_t)4 * s.nplane_max * (s.fft[0] + 1) +
          2 * stage_elems(s.nstick_max, planes_nnp(s), su) + (ps ? 6 * nn : 0)) *
         sizeof(cx<T>);
}

constexpr size_t kSmemLimit = 227 * 1024;

template <class K> void set_smem(K kernel, size_t bytes) {
  TDLZ_CUDA_TRY(
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

int device_sms() {
  int dev = 0, n = 0;
  TDLZ_CUDA_TRY(cudaGetDevice(&dev));
  TDLZ_CUDA_TRY(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return n > 0 ? n : 1;
}

// Chunks of band-sides per (vector, plane) so that the grid covers about four CTAs per
// SM (a function of the shape and the device only).
int chunks_for(const QSlot &s, int nvec) {
  const long long nbs1 = 2LL * s.nk * s.nb;
  const long long base = (long long)nvec * s.fft[2];
  long long want = (4LL * device_sms() + base - 1) / base;
  want = std::max(1LL, std::min(want, nbs1));
  return (int)want;
}
int chunk_len_for(const QSlot &s, int nchunk) {
  const long long nbs1 = 2LL * s.nk * s.nb;
  return (int)((nbs1 + nchunk - 1) / nchunk);
}

#define TDLZ_PLANES_SWITCH(n, CALL)                                                     \
  switch (n) {                                                                          \
    case 12: CALL(12); break;                                                           \
    case 16: CALL(16); break;                                                           \
    case 24: CALL(24); break;                                                           \
    case 36: CALL(36); break;                                                           \
    case 45: CALL(45); break;                                                           \
    case 48: if constexpr (sizeof(T) == 4) { CALL(48); } break;                         \
    default: TDLZ_REQUIRE(false, TDLZ_ERR_STATE, "plane stages: unsupported grid length"); \
  }

}  // namespace

long long planes_nnp(const QSlot &s) {
  const long long nn = (long long)s.fft[0] * s.fft[1];
  return (nn + 1) & ~1LL;
}

template <class T> bool planes_supported(const QSlot &s) {
  const int n = s.fft[0];
  if (s.fft[1] != n || !reg_fft_length(n) || threads_of(n) == 0) return false;
  if (sizeof(T) == 8 && n > 45) return false;
  // register plan of the z lines (pipeline.cu z_plan)
  const int n3 = s.fft[2];
  const bool zok = reg_fft_length(n3) ||
                   (n3 % 4 == 0 && (n3 / 4 == 24 || n3 / 4 == 36 || n3 / 4 == 48));
  if (!zok) return false;
  return smem_density<T>(s) <= kSmemLimit && smem_product<T>(s, 0) <= kSmemLimit;
}

int planes_density_chunks(const QSlot &s, int nvec, size_t) { return chunks_for(s, nvec); }

template <class T> void planes_build_u(Context &ctx, QSlot &s, const double2 *ur, DevBuf &us) {
  const long long nn = (long long)s.fft[0] * s.fft[1], nnp = planes_nnp(s);
  const long long total = s.rows() * s.fft[2] * nnp;
  us.alloc((size_t)total * sizeof(cx<T>));
  u_slab_kernel<T><<<blocks_for(total), 256, 0, ctx.stream>>>(ur, us.as<cx<T>>(), nn, s.fft[2],
                                                              nnp, s.nr, total);
  TDLZ_LAUNCH_CHECK();
}

template <class T>
void planes_grid_from_slabs(Context &ctx, QSlot &s, const double2 *us, DevBuf &ur) {
  const long long nn = (long long)s.fft[0] * s.fft[1], total = s.rows() * s.nr;
  ur.alloc((size_t)total * sizeof(cx<T>));
  grid_from_slab_kernel<T><<<blocks_for(total), 256, 0, ctx.stream>>>(
      us, ur.as<cx<T>>(), nn, s.fft[2], planes_nnp(s), s.nr, total);
  TDLZ_LAUNCH_CHECK();
}

template <class T>
void planes_density(Context &ctx, QSlot &s, const cx<T> *i1t, const cx<T> *us, const T *wk,
                    cx<T> *part, cx<T> *rho, int nvec) {
  const PlTables tb = tables_of(s);
  const int n = s.fft[0];
  const int nchunk = chunks_for(s, nvec), len = chunk_len_for(s, nchunk);
  const size_t sm = smem_density<T>(s);
  const dim3 grid((unsigned)(nvec * nchunk), (unsigned)s.fft[2]);
#define TDLZ_PL_DENS(NV)                                                                  \
  {                                                                                       \
    auto kern = plane_density_kernel<T, NV>;                                              \
    set_smem(kern, sm);                                                                   \
    kern<<<grid, Lay<NV>::THREADS, sm, ctx.stream>>>(i1t, us, wk, part, tb, nvec, len,    \
                                                     line_tw<T, NV>());                   \
  }
  TDLZ_PLANES_SWITCH(n, TDLZ_PL_DENS)
#undef TDLZ_PL_DENS
  TDLZ_LAUNCH_CHECK();
  const long long nn = (long long)n * s.fft[1];
  const long long total = (long long)nvec * 4 * s.nr;
  plane_reduce_kernel<T><<<blocks_for(total), 256, 0, ctx.stream>>>(part, rho, nchunk, nn,
                                                                    s.fft[2], total);
  TDLZ_LAUNCH_CHECK();
}

template <class T>
void planes_potential(Context &ctx, QSlot &s, const cx<T> *rho, const cx<T> *vh, const T *fxc,
                      const T *vloc, const T *bf, cx<T> *pot, int nvec, bool use_h,
                      bool use_xc) {
  const long long total = (long long)nvec * s.nr;
  potential_planes_kernel<T><<<blocks_for(total), 256, 0, ctx.stream>>>(
      rho, vh, fxc, vloc, bf, pot, s.nr, s.fft[2], planes_nnp(s), use_h ? 1 : 0, use_xc ? 1 : 0,
      total);
  TDLZ_LAUNCH_CHECK();
}

template <class T>
void planes_product_forward(Context &ctx, QSlot &s, cx<T> *i1t, const cx<T> *us,
                            const cx<T> *pot, int nvec, const std::function<void()> &refill) {
  const PlTables tb = tables_of(s);
  const int n = s.fft[0];
  std::vector<int> cands;
  for (int c : {2, 1, 0})
    if (smem_product<T>(s, c) <= kSmemLimit) cands.push_back(c);
  TDLZ_REQUIRE(!cands.empty(), TDLZ_ERR_STATE, "plane stages: shared memory");
  char key[160];
  snprintf(key, sizeof(key), "plane_product/%s/n=%d/n3=%d/nsm=%d/npm=%d/nbs=%lld/nvec=%d",
           sizeof(T) == 4 ? "f32" : "f64", n, s.fft[2], s.nstick_max, s.nplane_max,
           2LL * s.nk * s.nb, nvec);
  const int nchunk = chunks_for(s, nvec), len = chunk_len_for(s, nchunk);
  const dim3 grid((unsigned)(nvec * nchunk), (unsigned)s.fft[2]);
  ctx.tuner.pick(
      ctx.stream, key, cands, cands[0],
      [&](int code) {
        const size_t sm = smem_product<T>(s, code);
#define TDLZ_PL_PROD(NV)                                                                  \
  {                                                                                       \
    auto kern = code == 2   ? plane_product_fwd_kernel<T, NV, false, true>                \
                : code == 1 ? plane_product_fwd_kernel<T, NV, true, false>                \
                            : plane_product_fwd_kernel<T, NV, false, false>;              \
    set_smem(kern, sm);                                                                   \
    kern<<<grid, Lay<NV>::THREADS, sm, ctx.stream>>>(i1t, us, pot, tb, nvec, len,         \
                                                     line_tw<T, NV>());                   \
  }
        TDLZ_PLANES_SWITCH(n, TDLZ_PL_PROD)
#undef TDLZ_PL_PROD
        TDLZ_LAUNCH_CHECK();
      },
      refill);
}

template bool planes_supported<float>(const QSlot &);
template bool planes_supported<double>(const QSlot &);
template void planes_build_u<float>(Context &, QSlot &, const double2 *, DevBuf &);
template void planes_build_u<double>(Context &, QSlot &, const double2 *, DevBuf &);
template void planes_grid_from_slabs<float>(Context &, QSlot &, const double2 *, DevBuf &);
template void planes_grid_from_slabs<double>(Context &, QSlot &, const double2 *, DevBuf &);
template void planes_density<float>(Context &, QSlot &, const float2 *, const float2 *,
                                    const float *, float2 *, float2 *, int);
template void planes_density<double>(Context &, QSlot &, const double2 *, const double2 *,
                                     const double *, double2 *, double2 *, int);
template void planes_potential<float>(Context &, QSlot &, const float2 *, const float2 *,
                                      const float *, const float *, const float *, float2 *, int,
                                      bool, bool);
template void planes_potential<double>(Context &, QSlot &, const double2 *, const double2 *,
                                       const double *, const double *, const double *, double2 *,
                                       int, bool, bool);
template void planes_product_forward<float>(Context &, QSlot &, float2 *, const float2 *,
                                            const float2 *, int, const std::function<void()> &);
template void planes_product_forward<double>(Context &, QSlot &, double2 *, const double2 *,
                                             const double2 *, int,
                                             const std::function<void()> &);

}  // namespace tdlz
