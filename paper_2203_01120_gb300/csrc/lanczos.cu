// Lanczos recursions of Sec. 2.5 on the GPU.
//
// The vectors live in HBM in the precision of the Liouvillian (complex double
// for TDLZ_FP64, complex float for TDLZ_MIXED); every scalar (dot products,
// alpha, beta, gamma, z, signs) is FP64 and stays on the device, so a step is a
// fixed sequence of launches with no host round trip:
//   L application(s) -> dots (alpha, z) -> scalar A -> three-term update fused
//   with the dots of the new residual -> scalar B (beta, gamma, breakdown) ->
//   rescale.
// Dot products are deterministic: a fixed grid of blocks each sums a fixed
// contiguous range in FP64, and one block adds the partials in a fixed order.
//
// Flavours:
//  NH   q1 = p1 = v/||v||; a = L q, b = L^H p; alpha = p^H a;
//       r = a - alpha q - gamma q',  t = b - conj(alpha) p - conj(beta) p';
//       c = t^H r, beta' = sqrt|c|, gamma' = c / beta', q = r/beta', p = t/conj(gamma').
//       The left vectors are stored as p~ = J p: then L^H p = J L p~, so one plain L
//       pass over [q.., p~..] gives a and b~ = J b, the recursion for t~ = J t has the
//       same form, and p^H a = p~^H J a, t^H r = t~^H J r (no sign-flip passes).
//  PH   J metric: c0 = v^H J v, q1 = v/sqrt|c0|, s1 = sign c0; a = L q;
//       alpha = s Re(q^H J a); r = a - alpha q - gamma q'; c = r^H J r,
//       beta' = sqrt|c|, s' = sign c, gamma' = s s' beta'.
//  PHM  metric M = J L (positive definite when D + K > 0): alpha = (Lq)^H J (Lq);
//       r = Lq - alpha q - beta q'; w = L r; c = r^H J w; beta' = sqrt c;
//       q = r/beta', Lq = w/beta' (the product of the step is the one on r).
#include <cmath>
#include <cstring>

#include "lanczos.cuh"
#include "tc_gemm.cuh"

namespace tdlz {

namespace {

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;
constexpr double kBreakdownTol = 1e-14;

struct Pair {
  const void *a;
  const void *b;
  int jsign;  // 1: weight -1 on the Y half
};
struct Pairs {
  Pair p[5];
  int n;
};

// Partial sums are stored kPStride values per block: alpha's dot and up to four z dots.
constexpr int kPStride = 5;


// Block-level deterministic sum of NV complex values per thread into
// out[blockIdx][0..NV) (row stride kPStride).
template <int NV>
__device__ void block_sum_store(double2 (&v)[NV], double2 *out) {
  static_assert(NV <= kPStride, "partial row");
  __shared__ double2 sh[kRedThreads];
  for (int q = 0; q < NV; ++q) {
    sh[threadIdx.x] = v[q];
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        sh[threadIdx.x].x += sh[threadIdx.x + s].x;
        sh[threadIdx.x].y += sh[threadIdx.x + s].y;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) out[(long long)blockIdx.x * kPStride + q] = sh[0];
    __syncthreads();
  }
}

// partial[blk][i] = sum_{e in blk range} conj(a_i[e]) b_i[e] (J-weighted if requested)
// Products are formed in the vectors' precision T and summed in T over runs of
// kRun elements per thread before each run is added to an FP64 accumulator (on
// this part FP64 arithmetic is ~1/64 of the FP32 rate, so the mixed path keeps
// the per-element work in FP32 and only the reduction in FP64).
constexpr int kRun = 16;
constexpr int kUnroll = 4;  // independent elements per thread per iteration (loads in flight)
template <class T, int NP>
__global__ void __launch_bounds__(kRedThreads)
    dots_kernel(Pairs pr, long long n, long long half, double2 *partial) {
  double2 acc[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) acc[i] = make_double2(0.0, 0.0);
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  const cx<T> *A[NP], *B[NP];
  T sgn[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    A[i] = reinterpret_cast<const cx<T> *>(pr.p[i].a);
    B[i] = reinterpret_cast<const cx<T> *>(pr.p[i].b);
    sgn[i] = pr.p[i].jsign ? T(-1) : T(1);
  }
  const long long bd = blockDim.x;
  long long e = b0 + threadIdx.x;
  // runs of kRun elements summed in T, each run added to the FP64 accumulators
  while (e < b1) {
    T rx[NP], ry[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) rx[i] = ry[i] = T(0);
    for (int it = 0; it < kRun / kUnroll && e < b1; ++it) {
      cx<T> av[kUnroll][NP], bv[kUnroll][NP];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const long long eu = e + u * bd;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          av[u][i] = eu < b1 ? A[i][eu] : czero<T>();
          bv[u][i] = eu < b1 ? B[i][eu] : czero<T>();
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const bool neg = e + u * bd >= half;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const T sg = neg ? sgn[i] : T(1);
          rx[i] += sg * (av[u][i].x * bv[u][i].x + av[u][i].y * bv[u][i].y);
          ry[i] += sg * (av[u][i].x * bv[u][i].y - av[u][i].y * bv[u][i].x);
        }
      }
      e += kUnroll * bd;
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      acc[i].x += (double)rx[i];
      acc[i].y += (double)ry[i];
    }
  }
  block_sum_store<NP>(acc, partial);
}

// Sum the partials of nv values in fixed order; result into out[nv].
__device__ void reduce_partials(const double2 *partial, int nblk, int nv, double2 *out) {
  __shared__ double2 sh[kRedThreads];
  for (int q = 0; q < nv; ++q) {
    double2 s = {0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      s.x += partial[(long long)b * kPStride + q].x;
      s.y += partial[(long long)b * kPStride + q].y;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = kRedThreads / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        sh[threadIdx.x].x += sh[threadIdx.x + st].x;
        sh[threadIdx.x].y += sh[threadIdx.x + st].y;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
    __syncthreads();
  }
}

__device__ __forceinline__ bool finite2(double2 v) { return isfinite(v.x) && isfinite(v.y); }

// ---------------------------------------------------------------- scalars
// Stage A: alpha and z from the dots (d0 = alpha source, d1..nz = q^H u^l).
__global__ void scalar_a_kernel(const double2 *partial, int nblk, ChainScalars *cs,
                                ChainCoeffs cf, int flavor, int nz) {
  __shared__ double2 d[kPStride];
  reduce_partials(partial, nblk, 1 + nz, d);
  if (threadIdx.x != 0) return;
  if (cs->stopped) return;
  int j = cs->step;
  double2 alpha;
  if (flavor == TDLZ_NONHERMITIAN)
    alpha = d[0];
  else if (flavor == TDLZ_PSEUDOHERMITIAN)
    alpha = make_double2(cs->s * d[0].x, 0.0);
  else
    alpha = make_double2(d[0].x, 0.0);
  cs->alpha = alpha;
  cf.alpha[j] = alpha;
  bool finite = finite2(alpha);
  for (int l = 0; l < nz; ++l) {
    cf.z[(long long)l * cf.cap + j] = d[1 + l];
    finite = finite && finite2(d[1 + l]);
  }
  if (!finite) {
    cs->status = TDLZ_ERR_NUMERIC;
    cs->stopped = 1;
    cs->steps_done = j;  // step j has no valid alpha or z: the chain ends before it
  }
}

// Stage B: beta, gamma, signs and rescale factors from c (d0) and norms (d1, d2).
__global__ void scalar_b_kernel(const double2 *partial, int nblk, ChainScalars *cs,
                                ChainCoeffs cf, int flavor) {
  __shared__ double2 d[kPStride];
  reduce_partials(partial, nblk, 3, d);
  if (threadIdx.x != 0) return;
  if (cs->stopped) {
    cs->scale_q = make_double2(0, 0);
    cs->scale_p = make_double2(0, 0);
    return;
  }
  int j = cs->step;
  double2 c = d[0];
  double nr2 = d[1].x, nt2 = d[2].x;
  bool stop = false;
  int status = TDLZ_OK;
  double beta = 0.0;
  double2 gamma = make_double2(0, 0);
  if (flavor == TDLZ_NONHERMITIAN) {
    double ac = hypot(c.x, c.y);
    if (!(ac >= kBreakdownTol * sqrt(nr2 * nt2)) || ac == 0.0) {
      stop = true;
      status = isfinite(ac) ? TDLZ_ERR_BREAKDOWN : TDLZ_ERR_NUMERIC;
    } else {
      beta = sqrt(ac);
      gamma = make_double2(c.x / beta, c.y / beta);
      cs->scale_q = make_double2(1.0 / beta, 0.0);
      // p' = t / conj(gamma) = t * gamma / |gamma|^2
      double g2 = gamma.x * gamma.x + gamma.y * gamma.y;
      cs->scale_p = make_double2(gamma.x / g2, gamma.y / g2);
    }
  } else if (flavor == TDLZ_PSEUDOHERMITIAN) {
    double cr = c.x;
    if (!(fabs(cr) >= kBreakdownTol * nr2) || nr2 == 0.0) {
      stop = true;
      status = isfinite(cr) ? TDLZ_ERR_BREAKDOWN : TDLZ_ERR_NUMERIC;
    } else {
      beta = sqrt(fabs(cr));
      double sn = cr >= 0 ? 1.0 : -1.0;
      gamma = make_double2(cs->s * sn * beta, 0.0);
      cs->s = sn;
      cs->scale_q = make_double2(1.0 / beta, 0.0);
    }
  } else {  // PHM: c = r^H J L r, norms ||r||^2, ||L r||^2
    double cr = c.x;
    if (!(cr > kBreakdownTol * sqrt(nr2 * nt2))) {
      stop = true;
      status = (cr < 0.0 && isfinite(cr)) ? TDLZ_ERR_NUMERIC
                                          : (isfinite(cr) ? TDLZ_ERR_BREAKDOWN : TDLZ_ERR_NUMERIC);
    } else {
      beta = sqrt(cr);
      gamma = make_double2(beta, 0.0);
      cs->scale_q = make_double2(1.0 / beta, 0.0);
      cs->scale_p = make_double2(1.0 / beta, 0.0);
    }
  }
  if (stop) {
    cs->stopped = 1;
    cs->status = status;
    cs->steps_done = j + 1;
    cs->scale_q = make_double2(0, 0);
    cs->scale_p = make_double2(0, 0);
    return;
  }
  cf.beta[j] = beta;
  cf.gamma[j] = gamma;
  cs->beta_prev = beta;
  cs->gamma_prev = gamma;
  cs->step = j + 1;
  cs->steps_done = j + 1;
}

// Initial normalisation: c0 = d0 (J-norm, norm or M-norm of v).
__global__ void scalar_init_kernel(const double2 *partial, int nblk, ChainScalars *cs,
                                   int flavor) {
  __shared__ double2 d[kPStride];
  reduce_partials(partial, nblk, 1, d);
  if (threadIdx.x != 0) return;
  double c0 = d[0].x;
  cs->step = 0;
  cs->steps_done = 0;
  cs->stopped = 0;
  cs->status = TDLZ_OK;
  cs->beta_prev = 0.0;
  cs->gamma_prev = make_double2(0, 0);
  cs->alpha = make_double2(0, 0);
  double n0;
  if (flavor == TDLZ_PSEUDOHERMITIAN) {
    n0 = sqrt(fabs(c0));
    cs->s = c0 >= 0 ? 1.0 : -1.0;
  } else if (flavor == TDLZ_NONHERMITIAN) {
    n0 = sqrt(c0);
    cs->s = 1.0;
  } else {
    n0 = c0 > 0 ? sqrt(c0) : 0.0;
    cs->s = 1.0;
  }
  cs->n0 = n0;
  if (!(n0 > 0.0) || !isfinite(n0)) {
    cs->stopped = 1;
    cs->status = (flavor == TDLZ_PSEUDOHERMITIAN_POSDEF && c0 < 0) ? TDLZ_ERR_NUMERIC
                                                                   : TDLZ_ERR_BREAKDOWN;
    cs->scale_q = make_double2(0, 0);
    cs->scale_p = make_double2(0, 0);
    return;
  }
  cs->scale_q = make_double2(1.0 / n0, 0.0);
  cs->scale_p = make_double2(1.0 / n0, 0.0);
}

// ------------------------------------------------------------ vector ops
// x *= *scale (complex, read on the device)
template <class T>
__global__ void scale_kernel(cx<T> *x, const double2 *scale, long long n) {
  double2 s = *scale;
  T sr = (T)s.x, si = (T)s.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cx<T> v = x[i];
    x[i] = mk<T>(v.x * sr - v.y * si, v.x * si + v.y * sr);
  }
}

// r = a - alpha q - g q'  (written over q'); partial dots of (r, r)_J, (r, r).
// NH also: t~ = b~ - conj(alpha) p~ - conj(beta) p~' (over p~'); dots (t~, r)_J = (t, r),
// (r, r), (t~, t~) = (t, t).
template <class T>
__global__ void __launch_bounds__(kRedThreads)
    update_kernel(const cx<T> *a, const cx<T> *q, cx<T> *qp, const cx<T> *b, const cx<T> *p,
                  cx<T> *pp, const ChainScalars *cs, int flavor, long long n, long long half,
                  double2 *partial) {
  // coefficients in the vectors' precision (FP64 path: exact; mixed: rounded to FP32,
  // an error of the order of the FP32 storage of r itself)
  const double2 a64 = cs->alpha;
  const double2 g64 = (flavor == TDLZ_PSEUDOHERMITIAN_POSDEF) ? make_double2(cs->beta_prev, 0.0)
                                                            : cs->gamma_prev;
  const T ax = (T)a64.x, ay = (T)a64.y, gx = (T)g64.x, gy = (T)g64.y, bp = (T)cs->beta_prev;
  double2 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  const long long bd = blockDim.x;
  const bool nh = flavor == TDLZ_NONHERMITIAN;
  long long e = b0 + threadIdx.x;
  while (e < b1) {
    T s0x = 0, s0y = 0, s1 = 0, s2 = 0;
    for (int it = 0; it < kRun / kUnroll && e < b1; ++it) {
      cx<T> av[kUnroll], qv[kUnroll], qpv[kUnroll], bv[kUnroll], pv[kUnroll], ppv[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const long long eu = e + u * bd;
        const bool in = eu < b1;
        av[u] = in ? a[eu] : czero<T>();
        qv[u] = in ? q[eu] : czero<T>();
        qpv[u] = in ? qp[eu] : czero<T>();
        if (nh) {
          bv[u] = in ? b[eu] : czero<T>();
          pv[u] = in ? p[eu] : czero<T>();
          ppv[u] = in ? pp[eu] : czero<T>();
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const long long eu = e + u * bd;
        if (eu >= b1) break;
        const cx<T> r = mk<T>(av[u].x - (ax * qv[u].x - ay * qv[u].y) - (gx * qpv[u].x - gy * qpv[u].y),
                              av[u].y - (ax * qv[u].y + ay * qv[u].x) - (gx * qpv[u].y + gy * qpv[u].x));
        qp[eu] = r;
        const T rn = r.x * r.x + r.y * r.y;
        if (nh) {
          // t = b - conj(alpha) p - beta p'  (beta real)
          const cx<T> t = mk<T>(bv[u].x - (ax * pv[u].x + ay * pv[u].y) - bp * ppv[u].x,
                                bv[u].y - (ax * pv[u].y - ay * pv[u].x) - bp * ppv[u].y);
          pp[eu] = t;
          const T sg = eu >= half ? T(-1) : T(1);
          s0x += sg * (t.x * r.x + t.y * r.y);
          s0y += sg * (t.x * r.y - t.y * r.x);
          s1 += rn;
          s2 += t.x * t.x + t.y * t.y;
        } else {
          s0x += eu >= half ? -rn : rn;
          s1 += rn;
        }
      }
      e += kUnroll * bd;
    }
    acc[0].x += (double)s0x;
    acc[0].y += (double)s0y;
    acc[1].x += (double)s1;
    acc[2].x += (double)s2;
  }
  block_sum_store<4>(acc, partial);
}

// NH, the M <= 4 chains of one group at once: partial[c][blk][0..NZ] = (p~_c^H J a_c,
// q_c^H u^0, .., q_c^H u^(NZ-1)), each u^l read once for every chain of the group.
struct NhGroupDots {
  const void *p[4], *a[4], *q[4];
  const void *u[4];
};
constexpr int kGroupUnroll = 2;
template <class T, int M, int NZ>
__global__ void __launch_bounds__(kRedThreads)
    nh_group_dots_kernel(NhGroupDots g, long long n, long long half, double2 *partial) {
  constexpr int NA = NZ + 1;
  double2 acc[M][NA];
#pragma unroll
  for (int c = 0; c < M; ++c)
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[c][i] = make_double2(0.0, 0.0);
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  const long long bd = blockDim.x;
  const cx<T> *U[NZ];
#pragma unroll
  for (int l = 0; l < NZ; ++l) U[l] = reinterpret_cast<const cx<T> *>(g.u[l]);
  long long e = b0 + threadIdx.x;
  while (e < b1) {
    T rx[M][NA], ry[M][NA];
#pragma unroll
    for (int c = 0; c < M; ++c)
#pragma unroll
      for (int i = 0; i < NA; ++i) rx[c][i] = ry[c][i] = T(0);
    for (int it = 0; it < kRun / kGroupUnroll && e < b1; ++it) {
      cx<T> uv[kGroupUnroll][NZ], pv[kGroupUnroll][M], av[kGroupUnroll][M], qv[kGroupUnroll][M];
#pragma unroll
      for (int w = 0; w < kGroupUnroll; ++w) {
        const long long ew = e + w * bd;
        const bool in = ew < b1;
#pragma unroll
        for (int l = 0; l < NZ; ++l) uv[w][l] = in ? U[l][ew] : czero<T>();
#pragma unroll
        for (int c = 0; c < M; ++c) {
          pv[w][c] = in ? reinterpret_cast<const cx<T> *>(g.p[c])[ew] : czero<T>();
          av[w][c] = in ? reinterpret_cast<const cx<T> *>(g.a[c])[ew] : czero<T>();
          qv[w][c] = in ? reinterpret_cast<const cx<T> *>(g.q[c])[ew] : czero<T>();
        }
      }
#pragma unroll
      for (int w = 0; w < kGroupUnroll; ++w) {
        const T sg = e + w * bd >= half ? T(-1) : T(1);
#pragma unroll
        for (int c = 0; c < M; ++c) {
          rx[c][0] += sg * (pv[w][c].x * av[w][c].x + pv[w][c].y * av[w][c].y);
          ry[c][0] += sg * (pv[w][c].x * av[w][c].y - pv[w][c].y * av[w][c].x);
#pragma unroll
          for (int l = 0; l < NZ; ++l) {
            rx[c][1 + l] += qv[w][c].x * uv[w][l].x + qv[w][c].y * uv[w][l].y;
            ry[c][1 + l] += qv[w][c].x * uv[w][l].y - qv[w][c].y * uv[w][l].x;
          }
        }
      }
      e += kGroupUnroll * bd;
    }
#pragma unroll
    for (int c = 0; c < M; ++c)
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        acc[c][i].x += (double)rx[c][i];
        acc[c][i].y += (double)ry[c][i];
      }
  }
#pragma unroll
  for (int c = 0; c < M; ++c)
    block_sum_store<NA>(acc[c], partial + (long long)c * gridDim.x * kPStride);
}

// x_v *= *s_v for the nv vectors of a set (the new Lanczos vectors of a group)
struct ScaleSet {
  void *x[32];
  const double2 *s[32];
};
template <class T>
__global__ void scale_set_kernel(ScaleSet ss, long long n) {
  const int v = blockIdx.y;
  cx<T> *x = reinterpret_cast<cx<T> *>(ss.x[v]);
  const double2 sc = *ss.s[v];
  const T sr = (T)sc.x, si = (T)sc.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cx<T> a = x[i];
    x[i] = mk<T>(a.x * sr - a.y * si, a.x * si + a.y * sr);
  }
}

template <class T>
__global__ void jflip_kernel(const cx<T> *x, cx<T> *y, long long n, long long half) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cx<T> v = x[i];
    y[i] = i >= half ? mk<T>(-v.x, -v.y) : v;
  }
}

template <class T>
void launch_dots(Context &ctx, Pairs pr, long long n, long long half, double2 *partial) {
  switch (pr.n) {
    case 1: dots_kernel<T, 1><<<kRedBlocks, kRedThreads, 0, ctx.stream>>>(pr, n, half, partial); break;
    case 2: dots_kernel<T, 2><<<kRedBlocks, kRedThreads, 0, ctx.stream>>>(pr, n, half, partial); break;
    case 3: dots_kernel<T, 3><<<kRedBlocks, kRedThreads, 0, ctx.stream>>>(pr, n, half, partial); break;
    case 4: dots_kernel<T, 4><<<kRedBlocks, kRedThreads, 0, ctx.stream>>>(pr, n, half, partial); break;
    default: dots_kernel<T, 5><<<kRedBlocks, kRedThreads, 0, ctx.stream>>>(pr, n, half, partial); break;
  }
  TDLZ_LAUNCH_CHECK();
}

}  // namespace

template <class T>
void jflip_copy(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *y) {
  long long n = s.br_elems();
  jflip_kernel<T><<<blocks_for(n), 256, 0, ctx.stream>>>(x, y, n, n / 2);
  TDLZ_LAUNCH_CHECK();
}
template void jflip_copy<double>(Context &, QSlot &, const double2 *, double2 *);
template void jflip_copy<float>(Context &, QSlot &, const float2 *, float2 *);

// ================================================================== chains
// Chains on the same q-slot form a group whose vectors are stacked so that one
// Liouvillian pass serves them all (the occupied orbitals are read once per pass).
// Vector slots of a group (m members; each slot holds a block of vectors):
//   NH : 0 [q_1..q_m, p~_1..p~_m]  1 [q'.., p~'..]  2 [a.., b~..]   (one L pass, p~ = J p)
//   PH : 0 [q..]  1 [q'..]  2 [a..]
//   PHM: 0 [q..]  1 [q'.. / r..]  2 [Lq..]  3 [w..]
template <class T>
void ChainSet::init_impl() {
  const size_t c = sizeof(cx<T>);
  red.alloc((size_t)kRedBlocks * kPStride * 16 * sizeof(double2));  // up to 16 chains per group
  for (size_t i = 0; i < chains.size(); ++i) {
    Chain &ch = chains[i];
    int g = -1;
    for (size_t j = 0; j < groups.size(); ++j)
      if (groups[j].qslot == ch.qslot) g = (int)j;
    if (g < 0) {
      groups.push_back(Group{});
      g = (int)groups.size() - 1;
      groups[g].qslot = ch.qslot;
    }
    ch.group = g;
    ch.index = (int)groups[g].members.size();
    groups[g].members.push_back((int)i);
  }
  for (Group &gr : groups) {
    QSlot &s = *ctx->slots[gr.qslot];
    ensure_precision<T>(*ctx, s);
    const long long n = s.br_elems(), half = n / 2;
    const int m = (int)gr.members.size();
    gr.nv = flavor == TDLZ_NONHERMITIAN ? 2 * m : m;
    const int nslot = flavor == TDLZ_PSEUDOHERMITIAN_POSDEF ? 4 : 3;
    gr.vec.alloc((size_t)nslot * gr.nv * n * c);
    TDLZ_CUDA_TRY(cudaMemsetAsync(gr.vec.p, 0, gr.vec.bytes, ctx->stream));
    for (int k = 0; k < nslot; ++k) gr.slot[k] = (char *)gr.vec.p + (size_t)k * gr.nv * n * c;
    for (int mi = 0; mi < m; ++mi) {
      Chain &ch = chains[gr.members[mi]];
      ch.coef.alloc((size_t)cap * (sizeof(double2) * 6 + sizeof(double)));
      TDLZ_CUDA_TRY(cudaMemsetAsync(ch.coef.p, 0, ch.coef.bytes, ctx->stream));
      ch.cf.cap = cap;
      ch.cf.alpha = ch.coef.as<double2>();
      ch.cf.gamma = ch.cf.alpha + cap;
      ch.cf.z = ch.cf.gamma + cap;
      ch.cf.beta = reinterpret_cast<double *>(ch.cf.z + 4 * (size_t)cap);
      ch.sc.alloc(sizeof(ChainScalars));
      TDLZ_CUDA_TRY(cudaMemsetAsync(ch.sc.p, 0, ch.sc.bytes, ctx->stream));
      start_vector<T>(*ctx, s, ch.mu, (cx<T> *)gr.slot[0] + mi * n);
    }
    if (flavor == TDLZ_PSEUDOHERMITIAN_POSDEF)  // w = L v for every member, one pass
      apply_liouvillian<T>(*ctx, s, (cx<T> *)gr.slot[0], (cx<T> *)gr.slot[3], m, 0u);
    double2 *part = red.as<double2>();
    for (int mi = 0; mi < m; ++mi) {
      Chain &ch = chains[gr.members[mi]];
      ChainScalars *cs = ch.sc.as<ChainScalars>();
      cx<T> *Q = (cx<T> *)gr.slot[0] + mi * n;
      Pairs pr{};
      pr.n = 1;
      if (flavor == TDLZ_PSEUDOHERMITIAN_POSDEF)
        pr.p[0] = Pair{Q, (cx<T> *)gr.slot[3] + mi * n, 1};
      else
        pr.p[0] = Pair{Q, Q, flavor == TDLZ_PSEUDOHERMITIAN ? 1 : 0};
      launch_dots<T>(*ctx, pr, n, half, part);
      scalar_init_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, flavor);
      TDLZ_LAUNCH_CHECK();
      scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(Q, &cs->scale_q, n);
      TDLZ_LAUNCH_CHECK();
      if (flavor == TDLZ_PSEUDOHERMITIAN_POSDEF) {
        scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>((cx<T> *)gr.slot[3] + mi * n,
                                                                &cs->scale_q, n);
        TDLZ_LAUNCH_CHECK();
      }
      if (flavor == TDLZ_NONHERMITIAN)  // p~_1 = J q_1
        jflip_copy<T>(*ctx, s, Q, (cx<T> *)gr.slot[0] + (m + mi) * n);
    }
    if (flavor == TDLZ_PSEUDOHERMITIAN_POSDEF) std::swap(gr.slot[2], gr.slot[3]);  // Lq = w / n0
  }
}

template <class T>
void ChainSet::advance_impl(int nsteps) {
  double2 *part = red.as<double2>();
  for (int it = 0; it < nsteps; ++it) {
    for (Group &gr : groups) {
      if (gr.host_step >= cap) continue;
      QSlot &s = *ctx->slots[gr.qslot];
      const long long n = s.br_elems(), half = n / 2;
      const int m = (int)gr.members.size();
      const cx<T> *u = slot_data<T>(s).uvec.template as<cx<T>>();
      cx<T> *S0 = (cx<T> *)gr.slot[0], *S1 = (cx<T> *)gr.slot[1], *S2 = (cx<T> *)gr.slot[2];
      if (flavor == TDLZ_NONHERMITIAN) {
        // a = L q and b~ = L p~ = J L^H p for every member in one pass
        apply_liouvillian<T>(*ctx, s, S0, S2, 2 * m, 0u);
        if (m <= 4) {
          // the group's dots in one pass (u^l read once), then per chain the scalars and
          // the update, then every new vector rescaled in one launch
          ProfScope ps(ctx->prof, ctx->stream, ST_LANCZOS, (15.0 * m + 3.0) * n * sizeof(cx<T>),
                       40.0 * m * n);
          NhGroupDots gd{};
          for (int mi = 0; mi < m; ++mi) {
            gd.q[mi] = S0 + mi * n;
            gd.p[mi] = S0 + (m + mi) * n;
            gd.a[mi] = S2 + mi * n;
          }
          for (int l = 0; l < ncomp; ++l) gd.u[l] = u + l * n;
#define TDLZ_NH_DOTS(MM)                                                                   \
  if (ncomp == 4)                                                                           \
    nh_group_dots_kernel<T, MM, 4><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(gd, n, half, part); \
  else                                                                                      \
    nh_group_dots_kernel<T, MM, 3><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(gd, n, half, part);
          switch (m) {
            case 1: TDLZ_NH_DOTS(1) break;
            case 2: TDLZ_NH_DOTS(2) break;
            case 3: TDLZ_NH_DOTS(3) break;
            default: TDLZ_NH_DOTS(4) break;
          }
#undef TDLZ_NH_DOTS
          TDLZ_LAUNCH_CHECK();
          const long long pstride = (long long)kRedBlocks * kPStride;
          for (int mi = 0; mi < m; ++mi) {
            Chain &ch = chains[gr.members[mi]];
            scalar_a_kernel<<<1, kRedThreads, 0, ctx->stream>>>(
                part + mi * pstride, kRedBlocks, ch.sc.as<ChainScalars>(), ch.cf, flavor, ncomp);
            TDLZ_LAUNCH_CHECK();
          }
          ScaleSet ss{};
          for (int mi = 0; mi < m; ++mi) {
            Chain &ch = chains[gr.members[mi]];
            ChainScalars *cs = ch.sc.as<ChainScalars>();
            cx<T> *Q = S0 + mi * n, *P = S0 + (m + mi) * n, *QP = S1 + mi * n,
                  *PP = S1 + (m + mi) * n, *A = S2 + mi * n, *B = S2 + (m + mi) * n;
            double2 *pc = part + mi * pstride;
            update_kernel<T><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(A, Q, QP, B, P, PP, cs,
                                                                         flavor, n, half, pc);
            TDLZ_LAUNCH_CHECK();
            scalar_b_kernel<<<1, kRedThreads, 0, ctx->stream>>>(pc, kRedBlocks, cs, ch.cf, flavor);
            TDLZ_LAUNCH_CHECK();
            ss.x[mi] = QP;
            ss.s[mi] = &cs->scale_q;
            ss.x[m + mi] = PP;
            ss.s[m + mi] = &cs->scale_p;
          }
          scale_set_kernel<T><<<dim3(blocks_for(n) / 2 + 1, 2 * m), 256, 0, ctx->stream>>>(ss, n);
          TDLZ_LAUNCH_CHECK();
          std::swap(gr.slot[0], gr.slot[1]);
          gr.host_step++;
          continue;
        }
        ProfScope ps(ctx->prof, ctx->stream, ST_LANCZOS, 18.0 * m * n * sizeof(cx<T>),
                     40.0 * m * n);
        for (int mi = 0; mi < m; ++mi) {
          Chain &ch = chains[gr.members[mi]];
          ChainScalars *cs = ch.sc.as<ChainScalars>();
          cx<T> *Q = S0 + mi * n, *P = S0 + (m + mi) * n, *QP = S1 + mi * n,
                *PP = S1 + (m + mi) * n, *A = S2 + mi * n, *B = S2 + (m + mi) * n;
          Pairs pr{};
          pr.n = 1 + ncomp;
          pr.p[0] = Pair{P, A, 1};  // p^H a = p~^H J a
          for (int l = 0; l < ncomp; ++l) pr.p[1 + l] = Pair{Q, u + l * n, 0};
          launch_dots<T>(*ctx, pr, n, half, part);
          scalar_a_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor,
                                                              ncomp);
          TDLZ_LAUNCH_CHECK();
          update_kernel<T><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(A, Q, QP, B, P, PP, cs,
                                                                       flavor, n, half, part);
          TDLZ_LAUNCH_CHECK();
          scalar_b_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor);
          TDLZ_LAUNCH_CHECK();
          scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(QP, &cs->scale_q, n);
          scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(PP, &cs->scale_p, n);
          TDLZ_LAUNCH_CHECK();
        }
        std::swap(gr.slot[0], gr.slot[1]);
      } else if (flavor == TDLZ_PSEUDOHERMITIAN) {
        apply_liouvillian<T>(*ctx, s, S0, S2, m, 0u);
        ProfScope ps(ctx->prof, ctx->stream, ST_LANCZOS, 11.0 * m * n * sizeof(cx<T>),
                     28.0 * m * n);
        for (int mi = 0; mi < m; ++mi) {
          Chain &ch = chains[gr.members[mi]];
          ChainScalars *cs = ch.sc.as<ChainScalars>();
          cx<T> *Q = S0 + mi * n, *QP = S1 + mi * n, *A = S2 + mi * n;
          Pairs pr{};
          pr.n = 1 + ncomp;
          pr.p[0] = Pair{Q, A, 1};
          for (int l = 0; l < ncomp; ++l) pr.p[1 + l] = Pair{Q, u + l * n, 0};
          launch_dots<T>(*ctx, pr, n, half, part);
          scalar_a_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor,
                                                              ncomp);
          TDLZ_LAUNCH_CHECK();
          update_kernel<T><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(
              A, Q, QP, nullptr, nullptr, nullptr, cs, flavor, n, half, part);
          TDLZ_LAUNCH_CHECK();
          scalar_b_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor);
          TDLZ_LAUNCH_CHECK();
          scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(QP, &cs->scale_q, n);
          TDLZ_LAUNCH_CHECK();
        }
        std::swap(gr.slot[0], gr.slot[1]);
      } else {
        cx<T> *S3 = (cx<T> *)gr.slot[3];
        {
          ProfScope ps(ctx->prof, ctx->stream, ST_LANCZOS, 9.0 * m * n * sizeof(cx<T>),
                       24.0 * m * n);
          for (int mi = 0; mi < m; ++mi) {
            Chain &ch = chains[gr.members[mi]];
            ChainScalars *cs = ch.sc.as<ChainScalars>();
            cx<T> *Q = S0 + mi * n, *QP = S1 + mi * n, *LQ = S2 + mi * n;
            Pairs pr{};
            pr.n = 1 + ncomp;
            pr.p[0] = Pair{LQ, LQ, 1};
            for (int l = 0; l < ncomp; ++l) pr.p[1 + l] = Pair{Q, u + l * n, 0};
            launch_dots<T>(*ctx, pr, n, half, part);
            scalar_a_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf,
                                                                flavor, ncomp);
            TDLZ_LAUNCH_CHECK();
            update_kernel<T><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(
                LQ, Q, QP, nullptr, nullptr, nullptr, cs, flavor, n, half, part);
            TDLZ_LAUNCH_CHECK();
          }
        }
        apply_liouvillian<T>(*ctx, s, S1, S3, m, 0u);  // w = L r for every member
        ProfScope ps(ctx->prof, ctx->stream, ST_LANCZOS, 6.0 * m * n * sizeof(cx<T>),
                     12.0 * m * n);
        for (int mi = 0; mi < m; ++mi) {
          Chain &ch = chains[gr.members[mi]];
          ChainScalars *cs = ch.sc.as<ChainScalars>();
          cx<T> *QP = S1 + mi * n, *W = S3 + mi * n;
          Pairs pc{};
          pc.n = 3;
          pc.p[0] = Pair{QP, W, 1};
          pc.p[1] = Pair{QP, QP, 0};
          pc.p[2] = Pair{W, W, 0};
          launch_dots<T>(*ctx, pc, n, half, part);
          scalar_b_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor);
          TDLZ_LAUNCH_CHECK();
          scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(QP, &cs->scale_q, n);
          scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(W, &cs->scale_q, n);
          TDLZ_LAUNCH_CHECK();
        }
        // q' <- q, q <- r/beta, Lq <- w/beta, w <- old Lq
        std::swap(gr.slot[0], gr.slot[1]);
        std::swap(gr.slot[2], gr.slot[3]);
      }
      gr.host_step++;
    }
  }
}

void ChainSet::init() {
  if (precision == TDLZ_FP64)
    init_impl<double>();
  else
    init_impl<float>();
}

void ChainSet::advance_eager(int nsteps) {
  if (nsteps <= 0) return;
  if (precision == TDLZ_FP64)
    advance_impl<double>(nsteps);
  else
    advance_impl<float>(nsteps);
}

ChainSet::~ChainSet() {
  if (gexec) cudaGraphExecDestroy(gexec);
}

std::vector<void *> ChainSet::slot_key() const {
  std::vector<void *> k;
  for (const Group &g : groups)
    for (int i = 0; i < 4; ++i) k.push_back(g.slot[i]);
  return k;
}

// Records two steps of every group into a graph without running them: the host
// bookkeeping that the recording advanced (step counters, launch counter) is put
// back, and the slot pointers are back where they were after two rotations.
void ChainSet::capture_two_steps() {
  if (gexec) {
    cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }
  std::vector<int> steps;
  for (const Group &g : groups) steps.push_back(g.host_step);
  const long long l0 = g_launches.load();
  cudaStream_t st = ctx->stream;
  TDLZ_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  cudaGraph_t graph = nullptr;
  try {
    advance_eager(2);
  } catch (...) {
    cudaStreamEndCapture(st, &graph);
    if (graph) cudaGraphDestroy(graph);
    for (size_t i = 0; i < groups.size(); ++i) groups[i].host_step = steps[i];
    throw;
  }
  TDLZ_CUDA_TRY(cudaStreamEndCapture(st, &graph));
  graph_kernels = g_launches.load() - l0;
  g_launches.fetch_sub(graph_kernels);
  for (size_t i = 0; i < groups.size(); ++i) groups[i].host_step = steps[i];
  cudaError_t e = cudaGraphInstantiate(&gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    gexec = nullptr;
    throw Error{TDLZ_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)};
  }
  graph_key = slot_key();
}

// Steps run eagerly (one launch sequence per step) while the profiler records
// per-stage events or while fewer than four steps are asked for; otherwise one
// eager step (which also sizes every workspace), then pairs of steps replayed
// from the captured graph, then the remainder eagerly.
void ChainSet::advance(int nsteps) {
  NvtxRange range("tdlz/advance");
  if (!use_graphs || ctx->prof.on || nsteps < 4) {
    advance_eager(nsteps);
    return;
  }
  advance_eager(1);
  int done = 1;
  int room = nsteps - done;
  for (const Group &g : groups) room = std::min(room, cap - g.host_step);
  const int pairs = room / 2;
  if (pairs > 0) {
    if (!gexec || graph_key != slot_key()) {
      NvtxRange cap_range("tdlz/capture");
      capture_two_steps();
    }
    NvtxRange replay_range("tdlz/graph_replay");
    for (int p = 0; p < pairs; ++p) {
      TDLZ_CUDA_TRY(cudaGraphLaunch(gexec, ctx->stream));
      g_launches.fetch_add(graph_kernels);
    }
    for (Group &g : groups) g.host_step += 2 * pairs;
    done += 2 * pairs;
  }
  advance_eager(nsteps - done);
}

void ChainSet::read(tdlz_lanczos_result *res) {
  TDLZ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  tc_gemm_check();
  for (size_t c = 0; c < chains.size(); ++c) {
    Chain &ch = chains[c];
    ChainScalars hs;
    TDLZ_CUDA_TRY(cudaMemcpy(&hs, ch.sc.p, sizeof(hs), cudaMemcpyDeviceToHost));
    std::vector<double2> buf((size_t)cap * 6);
    std::vector<double> bet(cap);
    TDLZ_CUDA_TRY(cudaMemcpy(buf.data(), ch.cf.alpha, sizeof(double2) * 6 * cap,
                             cudaMemcpyDeviceToHost));
    TDLZ_CUDA_TRY(cudaMemcpy(bet.data(), ch.cf.beta, sizeof(double) * cap, cudaMemcpyDeviceToHost));
    int done = hs.steps_done;
    if (res->alpha)
      for (int j = 0; j < cap; ++j) {
        double2 v = j < done ? buf[j] : make_double2(0, 0);
        res->alpha[2 * ((size_t)c * cap + j)] = v.x;
        res->alpha[2 * ((size_t)c * cap + j) + 1] = v.y;
      }
    if (res->gamma)
      for (int j = 0; j < cap; ++j) {
        double2 v = j < done ? buf[cap + j] : make_double2(0, 0);
        res->gamma[2 * ((size_t)c * cap + j)] = v.x;
        res->gamma[2 * ((size_t)c * cap + j) + 1] = v.y;
      }
    if (res->z)
      for (int l = 0; l < ncomp; ++l)
        for (int j = 0; j < cap; ++j) {
          double2 v = j < done ? buf[2 * (size_t)cap + (size_t)l * cap + j] : make_double2(0, 0);
          size_t o = 2 * (((size_t)c * ncomp + l) * cap + j);
          res->z[o] = v.x;
          res->z[o + 1] = v.y;
        }
    if (res->beta)
      for (int j = 0; j < cap; ++j) res->beta[(size_t)c * cap + j] = j < done ? bet[j] : 0.0;
    if (res->n0) res->n0[c] = hs.n0;
    if (res->wk) res->wk[c] = ctx->slots[ch.qslot]->wk[0];
    if (res->steps_done) res->steps_done[c] = done;
    if (res->status) res->status[c] = hs.status;
  }
}

// ================================================================ restart
// Image: RestartHeader, then per chain (qslot, mu), per group host_step, then for
// each group its vector slots in logical order, then per chain ChainScalars and
// the coefficient block (cap entries).  A chain set created with the same
// chains, flavour and precision and a capacity >= the saved one accepts it.
namespace {
struct RestartHeader {
  char magic[8];
  int version, flavor, precision, nchain, ngroup, cap, ncomp;
};
constexpr int kRestartVersion = 2;
size_t vec_elem_bytes(int precision) { return precision == TDLZ_FP64 ? 16 : 8; }
int nslots(int flavor) { return flavor == TDLZ_PSEUDOHERMITIAN_POSDEF ? 4 : 3; }
}  // namespace

size_t ChainSet::state_bytes() const {
  size_t b = sizeof(RestartHeader) + chains.size() * 2 * sizeof(int) + groups.size() * sizeof(int);
  for (const Group &g : groups) {
    const QSlot &s = *ctx->slots[g.qslot];
    b += (size_t)nslots(flavor) * g.nv * s.br_elems() * vec_elem_bytes(precision);
  }
  b += chains.size() * (sizeof(ChainScalars) + (size_t)cap * (6 * sizeof(double2) + sizeof(double)));
  return b;
}

void ChainSet::save(void *host, size_t bytes) {
  TDLZ_REQUIRE(bytes >= state_bytes(), TDLZ_ERR_ARG, "restart buffer too small");
  TDLZ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  char *p = static_cast<char *>(host);
  RestartHeader h{};
  std::memcpy(h.magic, "TDLZRST", 8);
  h.version = kRestartVersion;
  h.flavor = flavor;
  h.precision = precision;
  h.nchain = (int)chains.size();
  h.ngroup = (int)groups.size();
  h.cap = cap;
  h.ncomp = ncomp;
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  for (const Chain &c : chains) {
    int qm[2] = {c.qslot, c.mu};
    std::memcpy(p, qm, sizeof(qm));
    p += sizeof(qm);
  }
  for (const Group &g : groups) {
    std::memcpy(p, &g.host_step, sizeof(int));
    p += sizeof(int);
  }
  for (const Group &g : groups) {
    const QSlot &s = *ctx->slots[g.qslot];
    size_t sb = (size_t)g.nv * s.br_elems() * vec_elem_bytes(precision);
    for (int k = 0; k < nslots(flavor); ++k) {
      TDLZ_CUDA_TRY(cudaMemcpy(p, g.slot[k], sb, cudaMemcpyDeviceToHost));
      p += sb;
    }
  }
  const size_t cb = (size_t)cap * (6 * sizeof(double2) + sizeof(double));
  for (const Chain &c : chains) {
    TDLZ_CUDA_TRY(cudaMemcpy(p, c.sc.p, sizeof(ChainScalars), cudaMemcpyDeviceToHost));
    p += sizeof(ChainScalars);
    TDLZ_CUDA_TRY(cudaMemcpy(p, c.coef.p, cb, cudaMemcpyDeviceToHost));
    p += cb;
  }
}

void ChainSet::restore(const void *host, size_t bytes) {
  const char *p = static_cast<const char *>(host);
  TDLZ_REQUIRE(bytes >= sizeof(RestartHeader), TDLZ_ERR_ARG, "restart image truncated");
  RestartHeader h;
  std::memcpy(&h, p, sizeof(h));
  p += sizeof(h);
  TDLZ_REQUIRE(std::memcmp(h.magic, "TDLZRST", 8) == 0 && h.version == kRestartVersion,
               TDLZ_ERR_ARG, "not a tdlz restart image");
  TDLZ_REQUIRE(h.flavor == flavor && h.precision == precision && h.nchain == (int)chains.size() &&
                   h.ngroup == (int)groups.size() && h.ncomp == ncomp,
               TDLZ_ERR_ARG, "restart image was saved from a different chain set");
  TDLZ_REQUIRE(h.cap <= cap, TDLZ_ERR_ARG, "restart image holds more steps than this capacity");
  for (const Chain &c : chains) {
    int qm[2];
    std::memcpy(qm, p, sizeof(qm));
    p += sizeof(qm);
    TDLZ_REQUIRE(qm[0] == c.qslot && qm[1] == c.mu, TDLZ_ERR_ARG,
                 "restart image chains differ (q-slot or mu)");
  }
  size_t need = sizeof(RestartHeader) + chains.size() * 2 * sizeof(int) + groups.size() * sizeof(int);
  for (const Group &g : groups)
    need += (size_t)nslots(flavor) * g.nv * ctx->slots[g.qslot]->br_elems() *
            vec_elem_bytes(precision);
  const size_t cb_old = (size_t)h.cap * (6 * sizeof(double2) + sizeof(double));
  need += chains.size() * (sizeof(ChainScalars) + cb_old);
  TDLZ_REQUIRE(bytes >= need, TDLZ_ERR_ARG, "restart image truncated");
  std::vector<int> steps(groups.size());
  for (size_t i = 0; i < groups.size(); ++i) {
    std::memcpy(&steps[i], p, sizeof(int));
    p += sizeof(int);
  }
  TDLZ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  for (size_t i = 0; i < groups.size(); ++i) {
    Group &g = groups[i];
    size_t sb = (size_t)g.nv * ctx->slots[g.qslot]->br_elems() * vec_elem_bytes(precision);
    for (int k = 0; k < nslots(flavor); ++k) {
      TDLZ_CUDA_TRY(cudaMemcpy(g.slot[k], p, sb, cudaMemcpyHostToDevice));
      p += sb;
    }
    g.host_step = steps[i];
  }
  for (Chain &c : chains) {
    TDLZ_CUDA_TRY(cudaMemcpy(c.sc.p, p, sizeof(ChainScalars), cudaMemcpyHostToDevice));
    p += sizeof(ChainScalars);
    // coefficient block [alpha cap][gamma cap][z 4 cap][beta cap]: copy each part
    const double2 *src = reinterpret_cast<const double2 *>(p);
    TDLZ_CUDA_TRY(cudaMemcpy(c.cf.alpha, src, h.cap * sizeof(double2), cudaMemcpyHostToDevice));
    TDLZ_CUDA_TRY(cudaMemcpy(c.cf.gamma, src + h.cap, h.cap * sizeof(double2),
                             cudaMemcpyHostToDevice));
    for (int l = 0; l < 4; ++l)
      TDLZ_CUDA_TRY(cudaMemcpy(c.cf.z + (size_t)l * cap, src + (size_t)(2 + l) * h.cap,
                               h.cap * sizeof(double2), cudaMemcpyHostToDevice));
    TDLZ_CUDA_TRY(cudaMemcpy(c.cf.beta, reinterpret_cast<const double *>(src + 6 * (size_t)h.cap),
                             h.cap * sizeof(double), cudaMemcpyHostToDevice));
    p += cb_old;
  }
}

}  // namespace tdlz
