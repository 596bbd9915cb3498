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
//  PH   J metric: c0 = v^H J v, q1 = v/sqrt|c0|, s1 = sign c0; a = L q;
//       alpha = s Re(q^H J a); r = a - alpha q - gamma q'; c = r^H J r,
//       beta' = sqrt|c|, s' = sign c, gamma' = s s' beta'.
//  PHM  metric M = J L (positive definite when D + K > 0): alpha = (Lq)^H J (Lq);
//       r = Lq - alpha q - beta q'; w = L r; c = r^H J w; beta' = sqrt c;
//       q = r/beta', Lq = w/beta' (the product of the step is the one on r).
#include <cmath>

#include "lanczos.cuh"

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
  Pair p[4];
  int n;
};

__device__ __forceinline__ double2 load_d(const double2 *p, long long i) { return p[i]; }
__device__ __forceinline__ double2 load_d(const float2 *p, long long i) {
  float2 v = p[i];
  return make_double2(v.x, v.y);
}

// Block-level deterministic sum of nv complex values per thread into out[blockIdx][nv].
template <int NV>
__device__ void block_sum_store(double2 (&v)[NV], double2 *out) {
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
    if (threadIdx.x == 0) out[(long long)blockIdx.x * NV + q] = sh[0];
    __syncthreads();
  }
}

// partial[blk][i] = sum_{e in blk range} conj(a_i[e]) b_i[e] (J-weighted if requested)
template <class T>
__global__ void __launch_bounds__(kRedThreads)
    dots_kernel(Pairs pr, long long n, long long half, double2 *partial) {
  double2 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  long long chunk = (n + gridDim.x - 1) / gridDim.x;
  long long b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  for (long long e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
    double w = e >= half ? -1.0 : 1.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i >= pr.n) break;
      double2 a = load_d(reinterpret_cast<const cx<T> *>(pr.p[i].a), e);
      double2 b = load_d(reinterpret_cast<const cx<T> *>(pr.p[i].b), e);
      double s = pr.p[i].jsign ? w : 1.0;
      acc[i].x += s * (a.x * b.x + a.y * b.y);
      acc[i].y += s * (a.x * b.y - a.y * b.x);
    }
  }
  block_sum_store<4>(acc, partial);
}

// Sum the partials of nv values in fixed order; result into out[nv].
__device__ void reduce_partials(const double2 *partial, int nblk, int nv, double2 *out) {
  __shared__ double2 sh[kRedThreads];
  for (int q = 0; q < nv; ++q) {
    double2 s = {0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      s.x += partial[(long long)b * 4 + q].x;
      s.y += partial[(long long)b * 4 + q].y;
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
// Stage A: alpha and z from the dots (d0 = alpha source, d1..3 = q^H u^l).
__global__ void scalar_a_kernel(const double2 *partial, int nblk, ChainScalars *cs,
                                ChainCoeffs cf, int flavor) {
  __shared__ double2 d[4];
  reduce_partials(partial, nblk, 4, d);
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
  for (int l = 0; l < 3; ++l) cf.z[(long long)l * cf.cap + j] = d[1 + l];
  if (!finite2(alpha) || !finite2(d[1]) || !finite2(d[2]) || !finite2(d[3])) {
    cs->status = TDLZ_ERR_NUMERIC;
    cs->stopped = 1;
    cs->steps_done = j + 1;
  }
}

// Stage B: beta, gamma, signs and rescale factors from c (d0) and norms (d1, d2).
__global__ void scalar_b_kernel(const double2 *partial, int nblk, ChainScalars *cs,
                                ChainCoeffs cf, int flavor) {
  __shared__ double2 d[4];
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
  __shared__ double2 d[4];
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
// NH also: t = b - conj(alpha) p - conj(beta) p' (over p'); dots (t, r), (r, r), (t, t).
template <class T>
__global__ void __launch_bounds__(kRedThreads)
    update_kernel(const cx<T> *a, const cx<T> *q, cx<T> *qp, const cx<T> *b, const cx<T> *p,
                  cx<T> *pp, const ChainScalars *cs, int flavor, long long n, long long half,
                  double2 *partial) {
  double2 alpha = cs->alpha;
  double2 g = (flavor == TDLZ_PSEUDOHERMITIAN_POSDEF) ? make_double2(cs->beta_prev, 0.0)
                                                     : cs->gamma_prev;
  double bp = cs->beta_prev;
  double2 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  long long chunk = (n + gridDim.x - 1) / gridDim.x;
  long long b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  for (long long e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
    double2 av = load_d(a, e), qv = load_d(q, e), qpv = load_d(qp, e);
    double2 r;
    r.x = av.x - (alpha.x * qv.x - alpha.y * qv.y) - (g.x * qpv.x - g.y * qpv.y);
    r.y = av.y - (alpha.x * qv.y + alpha.y * qv.x) - (g.x * qpv.y + g.y * qpv.x);
    cx<T> rs = mk<T>((T)r.x, (T)r.y);
    qp[e] = rs;
    double2 rr = load_d(&rs, 0);  // the stored (rounded) residual
    double w = e >= half ? -1.0 : 1.0;
    if (flavor == TDLZ_NONHERMITIAN) {
      double2 bv = load_d(b, e), pv = load_d(p, e), ppv = load_d(pp, e);
      double2 t;
      // t = b - conj(alpha) p - beta p'  (beta real)
      t.x = bv.x - (alpha.x * pv.x + alpha.y * pv.y) - bp * ppv.x;
      t.y = bv.y - (alpha.x * pv.y - alpha.y * pv.x) - bp * ppv.y;
      cx<T> ts = mk<T>((T)t.x, (T)t.y);
      pp[e] = ts;
      double2 tt = load_d(&ts, 0);
      acc[0].x += tt.x * rr.x + tt.y * rr.y;
      acc[0].y += tt.x * rr.y - tt.y * rr.x;
      acc[1].x += rr.x * rr.x + rr.y * rr.y;
      acc[2].x += tt.x * tt.x + tt.y * tt.y;
    } else {
      acc[0].x += w * (rr.x * rr.x + rr.y * rr.y);
      acc[1].x += rr.x * rr.x + rr.y * rr.y;
    }
  }
  block_sum_store<4>(acc, partial);
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
  dots_kernel<T><<<kRedBlocks, kRedThreads, 0, ctx.stream>>>(pr, n, half, partial);
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
template <class T>
void ChainSet::init_impl() {
  size_t c = sizeof(cx<T>);
  red.alloc((size_t)kRedBlocks * 4 * sizeof(double2));
  for (auto &ch : chains) {
    QSlot &s = *ctx->slots[ch.qslot];
    ensure_precision<T>(*ctx, s);
    long long n = s.br_elems();
    int nvec = flavor == TDLZ_NONHERMITIAN ? 6 : 4;
    ch.vec.alloc((size_t)nvec * n * c);
    TDLZ_CUDA_TRY(cudaMemsetAsync(ch.vec.p, 0, ch.vec.bytes, ctx->stream));
    for (int i = 0; i < nvec; ++i) ch.v[i] = (char *)ch.vec.p + (size_t)i * n * c;
    ch.coef.alloc((size_t)cap * (sizeof(double2) * 5 + sizeof(double)));
    TDLZ_CUDA_TRY(cudaMemsetAsync(ch.coef.p, 0, ch.coef.bytes, ctx->stream));
    ch.cf.cap = cap;
    ch.cf.alpha = ch.coef.as<double2>();
    ch.cf.gamma = ch.cf.alpha + cap;
    ch.cf.z = ch.cf.gamma + cap;
    ch.cf.beta = reinterpret_cast<double *>(ch.cf.z + 3 * (size_t)cap);
    ch.sc.alloc(sizeof(ChainScalars));
    TDLZ_CUDA_TRY(cudaMemsetAsync(ch.sc.p, 0, ch.sc.bytes, ctx->stream));
    // start vector into Q (slot 0)
    cx<T> *Q = (cx<T> *)ch.v[0];
    start_vector<T>(*ctx, s, ch.mu, Q);
    double2 *part = red.as<double2>();
    ChainScalars *cs = ch.sc.as<ChainScalars>();
    long long half = n / 2;
    Pairs pr{};
    if (flavor == TDLZ_PSEUDOHERMITIAN_POSDEF) {
      // v in Q; W = L v in slot 3; c0 = v^H J W
      cx<T> *W = (cx<T> *)ch.v[3];
      apply_liouvillian<T>(*ctx, s, Q, W, false);
      pr.n = 1;
      pr.p[0] = Pair{Q, W, 1};
    } else {
      pr.n = 1;
      pr.p[0] = Pair{Q, Q, flavor == TDLZ_PSEUDOHERMITIAN ? 1 : 0};
    }
    launch_dots<T>(*ctx, pr, n, half, part);
    scalar_init_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, flavor);
    TDLZ_LAUNCH_CHECK();
    scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(Q, &cs->scale_q, n);
    TDLZ_LAUNCH_CHECK();
    if (flavor == TDLZ_PSEUDOHERMITIAN_POSDEF) {
      // Lq = W / n0 lives in slot 2
      std::swap(ch.v[2], ch.v[3]);
      scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>((cx<T> *)ch.v[2], &cs->scale_q, n);
      TDLZ_LAUNCH_CHECK();
    }
    if (flavor == TDLZ_NONHERMITIAN) {
      // P = Q
      TDLZ_CUDA_TRY(cudaMemcpyAsync(ch.v[3], Q, n * c, cudaMemcpyDeviceToDevice, ctx->stream));
    }
  }
}

// Vector slots:  NH: 0 q, 1 q', 2 a, 3 p, 4 p', 5 b
//                PH: 0 q, 1 q', 2 a
//                PHM: 0 q, 1 q' (r), 2 Lq, 3 w
template <class T>
void ChainSet::advance_impl(int nsteps) {
  for (auto &ch : chains) {
    QSlot &s = *ctx->slots[ch.qslot];
    long long n = s.br_elems(), half = n / 2;
    double2 *part = red.as<double2>();
    ChainScalars *cs = ch.sc.as<ChainScalars>();
    SlotData<T> &d = slot_data<T>(s);
    const cx<T> *u = d.uvec.template as<cx<T>>();
    for (int it = 0; it < nsteps; ++it) {
      if (ch.host_step >= cap) break;
      cx<T> *Q = (cx<T> *)ch.v[0], *QP = (cx<T> *)ch.v[1], *A = (cx<T> *)ch.v[2];
      Pairs pr{};
      pr.n = 4;
      if (flavor == TDLZ_NONHERMITIAN) {
        cx<T> *P = (cx<T> *)ch.v[3], *PP = (cx<T> *)ch.v[4], *B = (cx<T> *)ch.v[5];
        apply_liouvillian<T>(*ctx, s, Q, A, false);
        apply_liouvillian<T>(*ctx, s, P, B, true);
        ProfScope ps(ctx->prof, ctx->stream, ST_LANCZOS, 20.0 * n * sizeof(cx<T>), 40.0 * n);
        pr.p[0] = Pair{P, A, 0};
        for (int l = 0; l < 3; ++l) pr.p[1 + l] = Pair{Q, u + l * n, 0};
        launch_dots<T>(*ctx, pr, n, half, part);
        scalar_a_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor);
        TDLZ_LAUNCH_CHECK();
        update_kernel<T><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(A, Q, QP, B, P, PP, cs, flavor,
                                                                     n, half, part);
        TDLZ_LAUNCH_CHECK();
        scalar_b_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor);
        TDLZ_LAUNCH_CHECK();
        scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(QP, &cs->scale_q, n);
        scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(PP, &cs->scale_p, n);
        TDLZ_LAUNCH_CHECK();
        std::swap(ch.v[0], ch.v[1]);
        std::swap(ch.v[3], ch.v[4]);
      } else if (flavor == TDLZ_PSEUDOHERMITIAN) {
        apply_liouvillian<T>(*ctx, s, Q, A, false);
        ProfScope ps(ctx->prof, ctx->stream, ST_LANCZOS, 11.0 * n * sizeof(cx<T>), 28.0 * n);
        pr.p[0] = Pair{Q, A, 1};
        for (int l = 0; l < 3; ++l) pr.p[1 + l] = Pair{Q, u + l * n, 0};
        launch_dots<T>(*ctx, pr, n, half, part);
        scalar_a_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor);
        TDLZ_LAUNCH_CHECK();
        update_kernel<T><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(
            A, Q, QP, nullptr, nullptr, nullptr, cs, flavor, n, half, part);
        TDLZ_LAUNCH_CHECK();
        scalar_b_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor);
        TDLZ_LAUNCH_CHECK();
        scale_kernel<T><<<blocks_for(n), 256, 0, ctx->stream>>>(QP, &cs->scale_q, n);
        TDLZ_LAUNCH_CHECK();
        std::swap(ch.v[0], ch.v[1]);
      } else {
        cx<T> *LQ = A, *W = (cx<T> *)ch.v[3];
        {
          ProfScope ps(ctx->prof, ctx->stream, ST_LANCZOS, 9.0 * n * sizeof(cx<T>), 24.0 * n);
          pr.p[0] = Pair{LQ, LQ, 1};
          for (int l = 0; l < 3; ++l) pr.p[1 + l] = Pair{Q, u + l * n, 0};
          launch_dots<T>(*ctx, pr, n, half, part);
          scalar_a_kernel<<<1, kRedThreads, 0, ctx->stream>>>(part, kRedBlocks, cs, ch.cf, flavor);
          TDLZ_LAUNCH_CHECK();
          update_kernel<T><<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(
              LQ, Q, QP, nullptr, nullptr, nullptr, cs, flavor, n, half, part);
          TDLZ_LAUNCH_CHECK();
        }
        apply_liouvillian<T>(*ctx, s, QP, W, false);
        ProfScope ps(ctx->prof, ctx->stream, ST_LANCZOS, 6.0 * n * sizeof(cx<T>), 12.0 * n);
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
        // q' <- q, q <- r/beta, Lq <- w/beta, w <- old Lq
        std::swap(ch.v[0], ch.v[1]);
        std::swap(ch.v[2], ch.v[3]);
      }
      ch.host_step++;
    }
  }
}

void ChainSet::init() {
  if (precision == TDLZ_FP64)
    init_impl<double>();
  else
    init_impl<float>();
}

void ChainSet::advance(int nsteps) {
  if (precision == TDLZ_FP64)
    advance_impl<double>(nsteps);
  else
    advance_impl<float>(nsteps);
}

void ChainSet::read(tdlz_lanczos_result *res) {
  TDLZ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  for (size_t c = 0; c < chains.size(); ++c) {
    Chain &ch = chains[c];
    ChainScalars hs;
    TDLZ_CUDA_TRY(cudaMemcpy(&hs, ch.sc.p, sizeof(hs), cudaMemcpyDeviceToHost));
    std::vector<double2> buf((size_t)cap * 5);
    std::vector<double> bet(cap);
    TDLZ_CUDA_TRY(cudaMemcpy(buf.data(), ch.cf.alpha, sizeof(double2) * 5 * cap,
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
      for (int l = 0; l < 3; ++l)
        for (int j = 0; j < cap; ++j) {
          double2 v = j < done ? buf[2 * (size_t)cap + (size_t)l * cap + j] : make_double2(0, 0);
          size_t o = 2 * (((size_t)c * 3 + l) * cap + j);
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

}  // namespace tdlz
