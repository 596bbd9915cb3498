// Plane-slab real-space stages of the mixed-precision Liouvillian.
//
// After the Z pass over the sphere's sticks (pipeline.cu, stick buffer in
// [row][j3][stick] order) every remaining transform works on one z plane j3 at a
// time, with the real-space data in z-major slab order [row][j3][j1*n2 + j2]:
//
//   yx inverse:       sticks -> Y lines (shared memory) -> X lines -> x(r) slab
//   density:          rho'_a(r) = sum w t_a U^+ sigma_a x (Eqs. charge_dens_resp_q,
//                     spin_dens_resp_q), pointwise over the slab order
//   product + fwd:    t = [v_loc + s B.sigma] x + W^s U formed while loading each
//                     X line, forward X (keeping the sphere's planes, shared memory),
//                     forward Y (keeping its sticks) -> stick buffer
//
// Compared with separate X and Y passes over a plane buffer in HBM, this removes
// two plane-buffer round trips and one full-grid pass per vector; every kernel
// keeps one line per thread in registers (regfft.cuh) and small per-CTA shared
// memory, so the SMs stay fully occupied.
#include <cmath>

#include "engine.cuh"
#include "regfft.cuh"
#include "slab.cuh"

namespace tdlz {

namespace {

constexpr int kSlabGroups = 8;  // partial density slices (fixed summation order)

struct SlabTables {
  const int *st_n;   // [nk] sticks per k
  const int *pl_n;   // [nk] planes per k
  const int *pl_of;  // [nk][N] plane index of j1 or -1
  const int *st_id;  // [nk][npm][N] stick index of (plane, j2) or -1
  int nsm, npm, n3, nk, nb;
};

__device__ __forceinline__ float2 f2zero() { return make_float2(0.f, 0.f); }

__host__ __device__ constexpr int line_threads(int n) { return ((2 * n + 31) / 32) * 32; }
constexpr int kSlabFwdThreads = 128;
__host__ __device__ inline int even(int n) { return (n + 1) & ~1; }

// Inverse Y then X transforms of a row pair (the two spinor rows of a band-side)
// on plane j3: sticks -> Y lines (shared memory) -> X lines written straight to
// xr[row][j3][j1*N + j2].  One CTA per (row pair, j3); thread t runs line t of
// each phase.
template <int N>
__global__ void __launch_bounds__(line_threads(N))
    slab_yx_inverse_kernel(const float2 *__restrict__ i1t, float2 *__restrict__ xr,
                           SlabTables tb, long long npairs, const RegTw<float, N> tw) {
  extern __shared__ float4 slab_smem_raw[];
  constexpr int YP = N + 1, NN = N * N;
  const int sst = even(tb.nsm);
  float2 *S = reinterpret_cast<float2 *>(slab_smem_raw);  // [2][nsm]
  float2 *Y = S + 2 * sst;                                 // [2][npm][N+1]
  int *sid = reinterpret_cast<int *>(Y + 2 * tb.npm * YP); // [npm][N] stick of (plane, j2)
  int *pof = sid + tb.npm * N;                             // [N] plane of j1
  const long long pr = blockIdx.x + (long long)gridDim.x * blockIdx.z;
  const int j3 = blockIdx.y;
  if (pr >= npairs) return;
  const long long row0 = 2 * pr;
  const int k = (int)((pr / tb.nb) % tb.nk);
  const int nst = __ldg(tb.st_n + k), npl = __ldg(tb.pl_n + k);
  for (int e = threadIdx.x; e < 2 * nst; e += blockDim.x) {
    const int sp = e >= nst, s = e - sp * nst;
    S[sp * sst + s] = i1t[((row0 + sp) * tb.n3 + j3) * tb.nsm + s];
  }
  for (int e = threadIdx.x; e < npl * N; e += blockDim.x)
    sid[e] = __ldg(tb.st_id + (long long)k * tb.npm * N + e);
  for (int e = threadIdx.x; e < N; e += blockDim.x) pof[e] = __ldg(tb.pl_of + (long long)k * N + e);
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * npl; t += blockDim.x) {
    const int sp = t / npl, p = t - sp * npl;
    const int *sd = sid + p * N;
    const float2 *src = S + sp * sst;
    float2 a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int s = sd[j];
      a[j] = s >= 0 ? src[s] : f2zero();
    }
    RegPlan<N>::template run<float, +1>(a, tw);
    float2 *o = Y + (sp * tb.npm + p) * YP;
#pragma unroll
    for (int j = 0; j < N; ++j) o[j] = a[j];
  }
  __syncthreads();
  if (threadIdx.x < 2 * N) {
    const int sp = threadIdx.x / N, j2 = threadIdx.x - sp * N;
    const float2 *src = Y + sp * tb.npm * YP + j2;
    float2 a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int p = pof[j];
      a[j] = p >= 0 ? src[p * YP] : f2zero();
    }
    RegPlan<N>::template run<float, +1>(a, tw);
    float2 *dst = xr + ((row0 + sp) * tb.n3 + j3) * NN + j2;
#pragma unroll
    for (int j = 0; j < N; ++j) dst[j * N] = a[j];
  }
}

// Products and forward X, Y transforms of one band-side (both spinor rows) on
// plane j3, sticks written to i1t.  All threads first form
//   t0 = a00 x0 + a01 x1 + c00 u0 + c01 u1,  t1 = a10 x0 + a11 x1 + c10 u0 + c11 u1
// pointwise over the plane (coalesced loads of xr, the U slab and the coefficient
// planes) into shared memory; then thread (spin sp, column j2) transforms its X
// line and keeps the sphere's planes, and the Y lines keep the sphere's sticks.
template <int N>
__global__ void __launch_bounds__(kSlabFwdThreads)
    slab_product_fwd_kernel(const float2 *__restrict__ xr, const float2 *__restrict__ us,
                            const float2 *__restrict__ coef, float2 *__restrict__ i1t,
                            SlabTables tb, int nvec, const RegTw<float, N> tw) {
  extern __shared__ float4 slab_smem_raw[];
  constexpr int YP = N + 1, NN = N * N;
  const int sst = even(tb.nsm);
  float2 *X = reinterpret_cast<float2 *>(slab_smem_raw);   // [2][NN]
  float2 *S = X + 2 * NN;                                   // [2][nsm]
  float2 *Y = S + 2 * sst;                                  // [2][npm][N+1]
  int *sid = reinterpret_cast<int *>(Y + 2 * tb.npm * YP);  // [npm][N]
  int *pof = sid + tb.npm * N;                              // [N]
  const long long nbs1 = 2LL * tb.nk * tb.nb;
  // the vectors of one band-side are neighbouring CTAs: they share the U slab in L2
  const long long blk = blockIdx.x + (long long)gridDim.x * blockIdx.z;
  const long long bs1 = blk / nvec;
  if (bs1 >= nbs1) return;
  const int vec = (int)(blk - bs1 * nvec);
  const int j3 = blockIdx.y;
  const int side = (int)(bs1 / ((long long)tb.nk * tb.nb));
  const int k = (int)((bs1 / tb.nb) % tb.nk);
  const int npl = __ldg(tb.pl_n + k), nst = __ldg(tb.st_n + k);
  const long long row0 = 2 * (vec * nbs1 + bs1);
  for (int e = threadIdx.x; e < npl * N; e += blockDim.x)
    sid[e] = __ldg(tb.st_id + (long long)k * tb.npm * N + e);
  for (int e = threadIdx.x; e < N; e += blockDim.x) pof[e] = __ldg(tb.pl_of + (long long)k * N + e);
  {
    const long long nr = (long long)tb.n3 * NN, o = (long long)j3 * NN;
    const float2 *x0p = xr + row0 * nr + o, *x1p = x0p + nr;
    const float2 *u0p = us + (bs1 * 2) * nr + o, *u1p = u0p + nr;
    // coefficient planes of this vector and side: (a00, a11), a01, c00, c01, c10, c11
    const float2 *cp = coef + ((long long)vec * 2 + side) * 6 * nr + o;
#pragma unroll 2
    for (int i = threadIdx.x; i < NN; i += blockDim.x) {
      const float2 x0 = x0p[i], x1 = x1p[i];
      const float2 u0 = __ldg(u0p + i), u1 = __ldg(u1p + i);
      const float2 d = __ldg(cp + i), f = __ldg(cp + nr + i);
      const float2 c00 = __ldg(cp + 2 * nr + i), c01 = __ldg(cp + 3 * nr + i);
      const float2 c10 = __ldg(cp + 4 * nr + i), c11 = __ldg(cp + 5 * nr + i);
      float2 t0 = make_float2(d.x * x0.x, d.x * x0.y);
      cfma<float>(t0, f, x1);
      cfma<float>(t0, c00, u0);
      cfma<float>(t0, c01, u1);
      float2 t1 = make_float2(d.y * x1.x, d.y * x1.y);
      cfma<float>(t1, make_float2(f.x, -f.y), x0);
      cfma<float>(t1, c10, u0);
      cfma<float>(t1, c11, u1);
      X[i] = t0;
      X[NN + i] = t1;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
    const int sp = t / N, j2 = t - sp * N;
    const float2 *src = X + sp * NN + j2;
    float2 a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = src[j * N];
    RegPlan<N>::template run<float, -1>(a, tw);
    float2 *out = Y + sp * tb.npm * YP + j2;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int p = pof[j];
      if (p >= 0) out[p * YP] = a[j];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * npl; t += blockDim.x) {
    const int sp = t / npl, p = t - sp * npl;
    const float2 *src = Y + (sp * tb.npm + p) * YP;
    float2 a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = src[j];
    RegPlan<N>::template run<float, -1>(a, tw);
    const int *sd = sid + p * N;
    float2 *out = S + sp * sst;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int s = sd[j];
      if (s >= 0) out[s] = a[j];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * nst; e += blockDim.x) {
    const int sp = e >= nst, s = e - sp * nst;
    i1t[((row0 + sp) * tb.n3 + j3) * tb.nsm + s] = S[sp * sst + s];
  }
}

// rho'_a for nvec stacked vectors, pointwise over the slab order: block row y sums
// the (side, k) pairs [y*ppg, (y+1)*ppg) into part[y][v][a][e] (e = j3*NN + i);
// t = (1, -1, -1, -1) on the Y side.  U is read once per point and band-side and
// contracted with every vector of the pass.
template <int NV>
__global__ void __launch_bounds__(256)
    slab_density_kernel(const float2 *__restrict__ us, const float2 *__restrict__ xr,
                        const float *__restrict__ wk, float2 *__restrict__ part, int nk, int nb,
                        long long nr, int nvec, int v0, int ppg) {
  const long long rows1 = 4LL * nk * nb;
  const int pb = blockIdx.y * ppg, pe = min(2 * nk, pb + ppg);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nr;
       e += (long long)gridDim.x * blockDim.x) {
    float2 acc[NV][4];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[v][a] = f2zero();
    for (int pair = pb; pair < pe; ++pair) {
      const int side = pair / nk, k = pair - side * nk;
      const float w = __ldg(wk + k), wt = side == 0 ? w : -w;
      float2 s[NV][4];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int a = 0; a < 4; ++a) s[v][a] = f2zero();
      for (int n = 0; n < nb; ++n) {
        const long long row = ((long long)pair * nb + n) * 2;
        const float2 u0 = __ldg(us + row * nr + e), u1 = __ldg(us + (row + 1) * nr + e);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const long long rv = row + (long long)(v0 + v) * rows1;
          const float2 x0 = xr[rv * nr + e], x1 = xr[(rv + 1) * nr + e];
          const float2 p00 = cmulc<float>(u0, x0), p01 = cmulc<float>(u0, x1);
          const float2 p10 = cmulc<float>(u1, x0), p11 = cmulc<float>(u1, x1);
          s[v][0] = cadd<float>(s[v][0], cadd<float>(p00, p11));
          s[v][1] = cadd<float>(s[v][1], cadd<float>(p01, p10));
          const float2 d = csub<float>(p10, p01);  // m_y: i (p10 - p01)
          s[v][2] = cadd<float>(s[v][2], make_float2(-d.y, d.x));
          s[v][3] = cadd<float>(s[v][3], csub<float>(p00, p11));
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        acc[v][0] = cadd<float>(acc[v][0], cscale<float>(s[v][0], w));
#pragma unroll
        for (int a = 1; a < 4; ++a) acc[v][a] = cadd<float>(acc[v][a], cscale<float>(s[v][a], wt));
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int a = 0; a < 4; ++a)
        part[(((long long)blockIdx.y * nvec + v0 + v) * 4 + a) * nr + e] = acc[v][a];
  }
}

// rho[v][a][r] = sum_g part[g][v][a][j3][i] in fixed order, r = i * n3 + j3.
__global__ void slab_reduce_kernel(const float2 *__restrict__ part, float2 *__restrict__ rho,
                                   int ngroup, long long nn, int n3, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    float2 s = part[e];
    for (int g = 1; g < ngroup; ++g) s = cadd<float>(s, part[(long long)g * total + e]);
    const long long plane = nn * n3;
    const long long va = e / plane, rem = e - va * plane;
    const long long j3 = rem / nn, i = rem - j3 * nn;
    rho[va * plane + i * n3 + j3] = s;
  }
}

// Product coefficients of each stacked vector and side, as six planes in slab
// order, coef[v][side][c][j3][i] (complex):
//   c = 0: (a00, a11)  a00 = vl + s bz, a11 = vl - s bz (two reals)
//   c = 1: a01 = s (bx - i by)      (a10 = conj(a01))
//   c = 2, 3: c00 = v0 + s v3, c01 = s (v1 - i v2)
//   c = 4, 5: c10 = s (v1 + i v2), c11 = v0 - s v3
// so that t0 = a00 x0 + a01 x1 + c00 u0 + c01 u1 and t1 = a10 x0 + a11 x1 + c10 u0 + c11 u1.
__global__ void slab_coef_kernel(const float2 *__restrict__ vp, const float *__restrict__ vloc,
                                 const float *__restrict__ bf, float2 *__restrict__ coef,
                                 long long nn, int n3, long long nr, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long vs = e / nr, rem = e - vs * nr;  // rem = j3 * nn + i
    const long long j3 = rem / nn, i = rem - j3 * nn;
    const long long v = vs >> 1;
    const float s = (vs & 1) ? -1.f : 1.f;
    const long long r = i * n3 + j3;
    const float vl = vloc[r], bx = bf[r], by = bf[nr + r], bz = bf[2 * nr + r];
    const float2 *vv = vp + v * 4 * nr;
    const float2 v0 = vv[r], v1 = vv[nr + r], v2 = vv[2 * nr + r], v3 = vv[3 * nr + r];
    float2 *o = coef + vs * 6 * nr + rem;
    o[0] = make_float2(vl + s * bz, vl - s * bz);
    o[nr] = make_float2(s * bx, -s * by);
    o[2 * nr] = make_float2(v0.x + s * v3.x, v0.y + s * v3.y);
    o[3 * nr] = make_float2(s * (v1.x + v2.y), s * (v1.y - v2.x));
    o[4 * nr] = make_float2(s * (v1.x - v2.y), s * (v1.y + v2.x));
    o[5 * nr] = make_float2(v0.x - s * v3.x, v0.y - s * v3.y);
  }
}

// U slab from the FP64 real-space orbitals: us[bs][sp][j3][i] = ur[bs][sp][i * n3 + j3].
__global__ void slab_u_kernel(const double2 *__restrict__ ur, float2 *__restrict__ us,
                              long long nn, int n3, long long nr, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long plane = nn * n3;
    const long long row = e / plane, rem = e - row * plane;
    const long long j3 = rem / nn, i = rem - j3 * nn;
    const double2 u = ur[row * nr + i * n3 + j3];
    us[e] = make_float2((float)u.x, (float)u.y);
  }
}

SlabTables tables_of(const QSlot &s) {
  SlabTables tb;
  tb.st_n = s.st_n.as<int>();
  tb.pl_n = s.pl_n.as<int>();
  tb.pl_of = s.pl_of.as<int>();
  tb.st_id = s.st_id.as<int>();
  tb.nsm = s.nstick_max;
  tb.npm = s.nplane_max;
  tb.n3 = s.fft[2];
  tb.nk = s.nk;
  tb.nb = s.nb;
  return tb;
}

// per-CTA shared memory (bytes): sticks and Y lines of both spinor rows, and the
// stick / plane tables of the CTA's k point
size_t smem_pair(const QSlot &s) {
  return 2 * ((size_t)even(s.nstick_max) + (size_t)s.nplane_max * (s.fft[0] + 1)) *
             sizeof(float2) +
         ((size_t)s.nplane_max + 1) * s.fft[0] * sizeof(int);
}
// the product + forward kernel also holds both spinor planes of products
size_t smem_forward(const QSlot &s) {
  return smem_pair(s) + 2 * (size_t)s.fft[0] * s.fft[1] * sizeof(float2);
}

constexpr size_t kSmemLimit = 227 * 1024;

template <class K>
void set_smem_attr(K kernel, size_t bytes) {
  TDLZ_CUDA_TRY(
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// grid (x, y = n3, z) covering `count` CTAs along x with x <= 65535 * 1024
dim3 plane_grid(long long count, int n3) {
  long long z = 1, x = count;
  while (x > 2147483647LL / 2) {
    z *= 2;
    x = (count + z - 1) / z;
  }
  return dim3((unsigned)x, (unsigned)n3, (unsigned)z);
}

#define TDLZ_SLAB_SWITCH(n, CALL)                                                      \
  switch (n) {                                                                         \
    case 12: CALL(12); break;                                                          \
    case 16: CALL(16); break;                                                          \
    case 24: CALL(24); break;                                                          \
    case 36: CALL(36); break;                                                          \
    case 45: CALL(45); break;                                                          \
    case 48: CALL(48); break;                                                          \
    default: TDLZ_REQUIRE(false, TDLZ_ERR_STATE, "slab path: unsupported grid length"); \
  }

}  // namespace

bool slab_supported(const QSlot &s) {
  const int n = s.fft[0];
  if (s.fft[1] != n || !reg_fft_length(n)) return false;
  return smem_forward(s) <= kSmemLimit;
}

void slab_build_u(Context &ctx, QSlot &s, const double2 *ur, DevBuf &us) {
  const long long nn = (long long)s.fft[0] * s.fft[1];
  const long long total = s.rows() * s.nr;
  us.alloc((size_t)total * sizeof(float2));
  slab_u_kernel<<<blocks_for(total), 256, 0, ctx.stream>>>(ur, us.as<float2>(), nn, s.fft[2],
                                                           s.nr, total);
  TDLZ_LAUNCH_CHECK();
}

void slab_inverse_yx(Context &ctx, QSlot &s, const float2 *i1t, float2 *xr, int nvec) {
  const SlabTables tb = tables_of(s);
  const long long npairs = s.rows() * nvec / 2;
  const size_t sm = smem_pair(s);
  const dim3 grid = plane_grid(npairs, s.fft[2]);
#define TDLZ_SLAB_INV(NV)                                                                   \
  set_smem_attr(slab_yx_inverse_kernel<NV>, sm);                                            \
  slab_yx_inverse_kernel<NV><<<grid, line_threads(NV), sm, ctx.stream>>>(i1t, xr, tb, npairs, \
                                                                         regtw<float, NV>());
  TDLZ_SLAB_SWITCH(s.fft[0], TDLZ_SLAB_INV)
#undef TDLZ_SLAB_INV
  TDLZ_LAUNCH_CHECK();
}

int slab_density_groups(const QSlot &s) { return std::min(kSlabGroups, 2 * s.nk); }

void slab_density(Context &ctx, QSlot &s, const float2 *xr, const float2 *us, const float *wk,
                  float2 *part, float2 *rho, int nvec) {
  const int npair = 2 * s.nk;
  const int ng0 = slab_density_groups(s);
  const int ppg = (npair + ng0 - 1) / ng0;
  const int ng = (npair + ppg - 1) / ppg;
  const dim3 grid(blocks_for(s.nr), ng);
  for (int v0 = 0; v0 < nvec; v0 += 3) {
    const int nv = std::min(3, nvec - v0);
    if (nv == 1)
      slab_density_kernel<1><<<grid, 256, 0, ctx.stream>>>(us, xr, wk, part, s.nk, s.nb, s.nr,
                                                           nvec, v0, ppg);
    else if (nv == 2)
      slab_density_kernel<2><<<grid, 256, 0, ctx.stream>>>(us, xr, wk, part, s.nk, s.nb, s.nr,
                                                           nvec, v0, ppg);
    else
      slab_density_kernel<3><<<grid, 256, 0, ctx.stream>>>(us, xr, wk, part, s.nk, s.nb, s.nr,
                                                           nvec, v0, ppg);
    TDLZ_LAUNCH_CHECK();
  }
  const long long nn = (long long)s.fft[0] * s.fft[1];
  const long long total = (long long)nvec * 4 * s.nr;
  slab_reduce_kernel<<<blocks_for(total), 256, 0, ctx.stream>>>(part, rho, ng, nn, s.fft[2],
                                                                total);
  TDLZ_LAUNCH_CHECK();
}

void slab_product_forward(Context &ctx, QSlot &s, const float2 *xr, const float2 *us,
                          const float2 *vpot, const float *vloc, const float *bf, float2 *coef,
                          float2 *i1t, int nvec) {
  const SlabTables tb = tables_of(s);
  const long long nn = (long long)s.fft[0] * s.fft[1];
  const long long total = (long long)nvec * 2 * s.nr;
  slab_coef_kernel<<<blocks_for(total), 256, 0, ctx.stream>>>(vpot, vloc, bf, coef, nn,
                                                              s.fft[2], s.nr, total);
  TDLZ_LAUNCH_CHECK();
  const size_t sm = smem_forward(s);
  const dim3 grid = plane_grid((long long)nvec * 2 * s.nk * s.nb, s.fft[2]);
#define TDLZ_SLAB_FWD(NV)                                                               \
  set_smem_attr(slab_product_fwd_kernel<NV>, sm);                                       \
  slab_product_fwd_kernel<NV><<<grid, kSlabFwdThreads, sm, ctx.stream>>>(xr, us, coef, i1t,  \
                                                                          tb, nvec,     \
                                                                          regtw<float, NV>());
  TDLZ_SLAB_SWITCH(s.fft[0], TDLZ_SLAB_FWD)
#undef TDLZ_SLAB_FWD
  TDLZ_LAUNCH_CHECK();
}

}  // namespace tdlz
