// Pruned, fused plane-wave <-> real-space transforms of the Liouvillian.
//
// A k+q sphere touches only a fraction of the FFT box: its (m1, m2) "sticks"
// (~20% of the z-lines at C2) and its m1 "planes" (~50% of the x-planes).  The
// inverse transform therefore runs
//   Z: sticks only, reading the sphere coefficients directly (no zeroed grid, no
//      separate scatter),
//   Y: only the planes that hold sticks, lines assembled from the stick buffer,
//   X: every column, lines assembled from the plane buffer -> x(r),
// and the forward transform mirrors it:
//   X: every column, with [v_loc + s B.sigma] x + W^s U formed while loading
//      (the product stage is fused), keeping only the sphere's planes,
//   Y: keeping only the sphere's sticks,
//   Z: writing only sphere coefficients, fused with + (|k+q+G|^2/2 - e_n) x.
// Each pass runs the Stockham line transform of fft.cu's axis kernel on a tile
// of TL lines held in shared memory as [position][TL + 1].
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "pipeline.cuh"
#include "regfft.cuh"

// Launch KERNEL<T, N>(args) for the register-line lengths; sets ok = false otherwise.
// (rt: threads per CTA, a variable in the calling scope)
#define TDLZ_REG_LAUNCH(n, KERNEL, grid, ...)                                          \
  switch (n) {                                                                       \
    case 12: KERNEL<T, 12><<<grid, rt, 0, st>>>(__VA_ARGS__, regtw<T, 12>()); break; \
    case 16: KERNEL<T, 16><<<grid, rt, 0, st>>>(__VA_ARGS__, regtw<T, 16>()); break; \
    case 24: KERNEL<T, 24><<<grid, rt, 0, st>>>(__VA_ARGS__, regtw<T, 24>()); break; \
    case 36: KERNEL<T, 36><<<grid, rt, 0, st>>>(__VA_ARGS__, regtw<T, 36>()); break; \
    case 45: KERNEL<T, 45><<<grid, rt, 0, st>>>(__VA_ARGS__, regtw<T, 45>()); break; \
    case 48: KERNEL<T, 48><<<grid, rt, 0, st>>>(__VA_ARGS__, regtw<T, 48>()); break; \
    default: ok = false;                                                             \
  }

namespace tdlz {

namespace {

struct St {
  int nrad;
  int radix[8];
};

St stages(const AxisPlan &a) {
  St s;
  s.nrad = a.nrad;
  for (int i = 0; i < 8; ++i) s.radix[i] = a.radix[i];
  return s;
}

template <class T>
__device__ __forceinline__ cx<T> twr(const cx<T> *tw, int t, int dir) {
  cx<T> w = tw[t];
  if (dir < 0) w.y = -w.y;
  return w;
}

// Stockham transform of TL lines of length n held at in[j * P + l]; returns the
// buffer (in or out) that holds the result.  Called by all threads of the block.
template <class T, int TL>
__device__ cx<T> *tile_fft(cx<T> *in, cx<T> *out, int n, const St &st, const cx<T> *tw,
                           int dir) {
  constexpr int P = TL + 1;
  cx<T> w3 = czero<T>(), w5a = czero<T>(), w5b = czero<T>();
  if (n % 3 == 0) w3 = twr<T>(tw, n / 3, dir);
  if (n % 5 == 0) {
    w5a = twr<T>(tw, n / 5, dir);
    w5b = twr<T>(tw, (2 * n) / 5, dir);
  }
  int ns = 1;
  for (int s = 0; s < st.nrad; ++s) {
    const int R = st.radix[s];
    const int nR = n / R;
    const int tstride = n / (ns * R);
    for (int b = threadIdx.x; b < nR * TL; b += blockDim.x) {
      const int j = b / TL;
      const int l = b - j * TL;
      const int k = j % ns;
      cx<T> v[5];
#pragma unroll
      for (int r = 0; r < 5; ++r)
        if (r < R) v[r] = in[(j + r * nR) * P + l];
      if (k != 0) {
#pragma unroll
        for (int r = 1; r < 5; ++r)
          if (r < R) v[r] = cmul<T>(v[r], twr<T>(tw, (r * k * tstride) % n, dir));
      }
      if (R == 2) {
        cx<T> a = v[0];
        v[0] = cadd<T>(a, v[1]);
        v[1] = csub<T>(a, v[1]);
      } else if (R == 4) {
        cx<T> a = cadd<T>(v[0], v[2]), bb = csub<T>(v[0], v[2]);
        cx<T> c = cadd<T>(v[1], v[3]), d = csub<T>(v[1], v[3]);
        cx<T> e = dir > 0 ? mk<T>(-d.y, d.x) : mk<T>(d.y, -d.x);
        v[0] = cadd<T>(a, c);
        v[2] = csub<T>(a, c);
        v[1] = cadd<T>(bb, e);
        v[3] = csub<T>(bb, e);
      } else if (R == 3) {
        cx<T> sm = cadd<T>(v[1], v[2]), df = csub<T>(v[1], v[2]);
        cx<T> m = mk<T>(v[0].x + w3.x * sm.x, v[0].y + w3.x * sm.y);
        cx<T> rr = mk<T>(-w3.y * df.y, w3.y * df.x);
        v[0] = cadd<T>(v[0], sm);
        v[1] = cadd<T>(m, rr);
        v[2] = csub<T>(m, rr);
      } else {
        cx<T> a1 = cadd<T>(v[1], v[4]), b1 = csub<T>(v[1], v[4]);
        cx<T> a2 = cadd<T>(v[2], v[3]), b2 = csub<T>(v[2], v[3]);
        T c1 = w5a.x, s1 = w5a.y, c2 = w5b.x, s2 = w5b.y;
        cx<T> m1 = mk<T>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
        cx<T> m2 = mk<T>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
        cx<T> p1 = mk<T>(-(s1 * b1.y + s2 * b2.y), s1 * b1.x + s2 * b2.x);
        cx<T> p2 = mk<T>(-(s2 * b1.y - s1 * b2.y), s2 * b1.x - s1 * b2.x);
        v[0] = cadd<T>(v[0], cadd<T>(a1, a2));
        v[1] = cadd<T>(m1, p1);
        v[4] = csub<T>(m1, p1);
        v[2] = cadd<T>(m2, p2);
        v[3] = csub<T>(m2, p2);
      }
      const int ob = (j / ns) * ns * R + k;
#pragma unroll
      for (int r = 0; r < 5; ++r)
        if (r < R) out[(ob + r * ns) * P + l] = v[r];
    }
    __syncthreads();
    cx<T> *t = in;
    in = out;
    out = t;
    ns *= R;
  }
  return in;
}

__device__ __forceinline__ long long row_of_block() {
  return blockIdx.y + (long long)gridDim.y * blockIdx.z;
}

// ---------------------------------------------------------------- inverse
// Z pass: sticks of row `row`, tile of TL sticks; sphere coefficients gathered.
// TR = false writes the stick buffer as [row][stick][j3], TR = true as
// [row][j3][stick] (the layout of the slab-fused stages).
template <class T, int TL, bool TR = false>
__global__ void __launch_bounds__(256)
    inv_z_kernel(const cx<T> *__restrict__ x, cx<T> *__restrict__ i1, const int *__restrict__ nst,
                 const int *__restrict__ smap, int nk, int nb, int npwx, int nsm, int n3, T scale,
                 long long rows, St st, const cx<T> *__restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int P = TL + 1;
  long long row = row_of_block();
  if (row >= rows) return;
  int k = (int)((row / (2 * nb)) % nk);
  int s0 = blockIdx.x * TL;
  int nl = min(TL, nst[k] - s0);
  if (nl <= 0) return;
  cx<T> *b0 = reinterpret_cast<cx<T> *>(smem_raw), *b1 = b0 + n3 * P;
  const int *mp = smap + ((long long)k * nsm + s0) * n3;
  const cx<T> *xr = x + row * npwx;
  for (int e = threadIdx.x; e < n3 * TL; e += blockDim.x) {
    int l = e / n3, j = e - l * n3;
    cx<T> v = czero<T>();
    if (l < nl) {
      int g = mp[l * n3 + j];
      if (g >= 0) v = cscale<T>(xr[g], scale);
    }
    b0[j * P + l] = v;
  }
  __syncthreads();
  cx<T> *res = tile_fft<T, TL>(b0, b1, n3, st, tw, +1);
  if (TR) {
    cx<T> *o = i1 + row * n3 * (long long)nsm + s0;
    for (int e = threadIdx.x; e < n3 * TL; e += blockDim.x) {
      int j = e / TL, l = e - j * TL;
      if (l < nl) o[(long long)j * nsm + l] = res[j * P + l];
    }
  } else {
    cx<T> *o = i1 + (row * nsm + s0) * n3;
    for (int e = threadIdx.x; e < n3 * TL; e += blockDim.x) {
      int l = e / n3, j = e - l * n3;
      if (l < nl) o[(long long)l * n3 + j] = res[j * P + l];
    }
  }
}

// Y pass: plane p of row, tile of TL consecutive j3; lines assembled from sticks.
template <class T, int TL>
__global__ void __launch_bounds__(256)
    inv_y_kernel(const cx<T> *__restrict__ i1, cx<T> *__restrict__ i2, const int *__restrict__ npl,
                 const int *__restrict__ sid, int nk, int nb, int nsm, int npm, int n2, int n3,
                 long long rows, St st, const cx<T> *__restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int P = TL + 1;
  long long rp = row_of_block();  // (row, plane) flattened
  if (rp >= rows * npm) return;
  long long row = rp / npm;
  int p = (int)(rp - row * npm);
  int k = (int)((row / (2 * nb)) % nk);
  if (p >= npl[k]) return;
  int j0 = blockIdx.x * TL;
  int nl = min(TL, n3 - j0);
  cx<T> *b0 = reinterpret_cast<cx<T> *>(smem_raw), *b1 = b0 + n2 * P;
  const int *sd = sid + ((long long)k * npm + p) * n2;
  const cx<T> *src = i1 + row * nsm * (long long)n3;
  for (int e = threadIdx.x; e < n2 * TL; e += blockDim.x) {
    int j = e / TL, l = e - j * TL;
    cx<T> v = czero<T>();
    int s = sd[j];
    if (s >= 0 && l < nl) v = src[(long long)s * n3 + j0 + l];
    b0[j * P + l] = v;
  }
  __syncthreads();
  cx<T> *res = tile_fft<T, TL>(b0, b1, n2, st, tw, +1);
  cx<T> *o = i2 + ((row * npm + p) * n2) * (long long)n3 + j0;
  for (int e = threadIdx.x; e < n2 * TL; e += blockDim.x) {
    int j = e / TL, l = e - j * TL;
    if (l < nl) o[(long long)j * n3 + l] = res[j * P + l];
  }
}

// X pass: every (j2, j3) column tile; lines assembled from planes -> x(r).
template <class T, int TL>
__global__ void __launch_bounds__(256)
    inv_x_kernel(const cx<T> *__restrict__ i2, cx<T> *__restrict__ xr, const int *__restrict__ plof,
                 int nk, int nb, int npm, int n1, long long n23, long long nr, long long rows, St st,
                 const cx<T> *__restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int P = TL + 1;
  long long row = row_of_block();
  if (row >= rows) return;
  int k = (int)((row / (2 * nb)) % nk);
  long long c0 = (long long)blockIdx.x * TL;
  int nl = (int)min((long long)TL, n23 - c0);
  cx<T> *b0 = reinterpret_cast<cx<T> *>(smem_raw), *b1 = b0 + n1 * P;
  const int *po = plof + (long long)k * n1;
  const cx<T> *src = i2 + row * npm * n23 + c0;
  for (int e = threadIdx.x; e < n1 * TL; e += blockDim.x) {
    int j = e / TL, l = e - j * TL;
    cx<T> v = czero<T>();
    int p = po[j];
    if (p >= 0 && l < nl) v = src[(long long)p * n23 + l];
    b0[j * P + l] = v;
  }
  __syncthreads();
  cx<T> *res = tile_fft<T, TL>(b0, b1, n1, st, tw, +1);
  cx<T> *o = xr + row * nr + c0;
  for (int e = threadIdx.x; e < n1 * TL; e += blockDim.x) {
    int j = e / TL, l = e - j * TL;
    if (l < nl) o[(long long)j * n23 + l] = res[j * P + l];
  }
}

// ---------------------------------------------------------------- forward
// X pass with the local products: band-side bs (both spinor rows), column tile.
template <class T, int TL>
__global__ void __launch_bounds__(256)
    fwd_x_product_kernel(const cx<T> *__restrict__ xr, const cx<T> *__restrict__ ur,
                         const T *__restrict__ vloc, const T *__restrict__ bf,
                         const cx<T> *__restrict__ v, cx<T> *__restrict__ i2,
                         const int *__restrict__ npl, const int *__restrict__ plj, int nk, int nb,
                         int npm, int n1, long long n23, long long nr, long long nbs, St st,
                         const cx<T> *__restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int P = TL + 1;
  long long bs = row_of_block();  // band-side over all stacked vectors
  if (bs >= nbs) return;
  const long long nbs1 = 2LL * nk * nb;  // band-sides per vector
  const long long vec = bs / nbs1, bs1 = bs - vec * nbs1;
  int k = (int)((bs1 / nb) % nk);
  int side = (int)(bs1 / ((long long)nk * nb));
  T s = side == 0 ? T(1) : T(-1);
  v += vec * 4 * nr;     // this vector's HXC potential
  ur += 2 * bs1 * nr;    // its occupied orbitals (shared by all vectors)
  long long c0 = (long long)blockIdx.x * TL;
  int nl = (int)min((long long)TL, n23 - c0);
  cx<T> *a0 = reinterpret_cast<cx<T> *>(smem_raw), *a1 = a0 + n1 * P;
  cx<T> *q0 = a1 + n1 * P, *q1 = q0 + n1 * P;
  long long r0 = 2 * bs;
  for (int e = threadIdx.x; e < n1 * TL; e += blockDim.x) {
    int j = e / TL, l = e - j * TL;
    cx<T> t0 = czero<T>(), t1 = czero<T>();
    if (l < nl) {
      long long r = (long long)j * n23 + c0 + l;
      T vl = vloc[r], bx = bf[r], by = bf[nr + r], bz = bf[2 * nr + r];
      cx<T> v0 = v[r], v1 = v[nr + r], v2 = v[2 * nr + r], v3 = v[3 * nr + r];
      cx<T> x0 = xr[r0 * nr + r], x1 = xr[(r0 + 1) * nr + r];
      cx<T> u0 = ur[r], u1 = ur[nr + r];
      cx<T> h01 = mk<T>(s * bx, -s * by), h10 = mk<T>(s * bx, s * by);
      t0 = cscale<T>(x0, vl + s * bz);
      cfma<T>(t0, h01, x1);
      t1 = cscale<T>(x1, vl - s * bz);
      cfma<T>(t1, h10, x0);
      cx<T> w00 = mk<T>(v0.x + s * v3.x, v0.y + s * v3.y);
      cx<T> w11 = mk<T>(v0.x - s * v3.x, v0.y - s * v3.y);
      cx<T> w01 = mk<T>(s * (v1.x + v2.y), s * (v1.y - v2.x));
      cx<T> w10 = mk<T>(s * (v1.x - v2.y), s * (v1.y + v2.x));
      cfma<T>(t0, w00, u0);
      cfma<T>(t0, w01, u1);
      cfma<T>(t1, w10, u0);
      cfma<T>(t1, w11, u1);
    }
    a0[j * P + l] = t0;
    q0[j * P + l] = t1;
  }
  __syncthreads();
  cx<T> *ra = tile_fft<T, TL>(a0, a1, n1, st, tw, -1);
  cx<T> *rb = tile_fft<T, TL>(q0, q1, n1, st, tw, -1);
  int np_ = npl[k];
  const int *pj = plj + (long long)k * npm;
  for (int e = threadIdx.x; e < np_ * TL; e += blockDim.x) {
    int p = e / TL, l = e - p * TL;
    if (l >= nl) continue;
    int j = pj[p];
    i2[((r0 * npm) + p) * n23 + c0 + l] = ra[j * P + l];
    i2[(((r0 + 1) * npm) + p) * n23 + c0 + l] = rb[j * P + l];
  }
}

// Y pass: plane p, tile of TL j3; keeps only the sphere's sticks.
template <class T, int TL>
__global__ void __launch_bounds__(256)
    fwd_y_kernel(const cx<T> *__restrict__ i2, cx<T> *__restrict__ i1, const int *__restrict__ npl,
                 const int *__restrict__ sid, int nk, int nb, int nsm, int npm, int n2, int n3,
                 long long rows, St st, const cx<T> *__restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int P = TL + 1;
  long long rp = row_of_block();  // (row, plane) flattened
  if (rp >= rows * npm) return;
  long long row = rp / npm;
  int p = (int)(rp - row * npm);
  int k = (int)((row / (2 * nb)) % nk);
  if (p >= npl[k]) return;
  int j0 = blockIdx.x * TL;
  int nl = min(TL, n3 - j0);
  cx<T> *b0 = reinterpret_cast<cx<T> *>(smem_raw), *b1 = b0 + n2 * P;
  const cx<T> *src = i2 + ((row * npm + p) * n2) * (long long)n3 + j0;
  for (int e = threadIdx.x; e < n2 * TL; e += blockDim.x) {
    int j = e / TL, l = e - j * TL;
    b0[j * P + l] = l < nl ? src[(long long)j * n3 + l] : czero<T>();
  }
  __syncthreads();
  cx<T> *res = tile_fft<T, TL>(b0, b1, n2, st, tw, -1);
  const int *sd = sid + ((long long)k * npm + p) * n2;
  cx<T> *o = i1 + row * nsm * (long long)n3 + j0;
  for (int e = threadIdx.x; e < n2 * TL; e += blockDim.x) {
    int j = e / TL, l = e - j * TL;
    int s = sd[j];
    if (s >= 0 && l < nl) o[(long long)s * n3 + l] = res[j * P + l];
  }
}

// Z pass: sticks; writes sphere coefficients + (kin - e) x.  TR as in inv_z_kernel.
template <class T, int TL, bool TR = false>
__global__ void __launch_bounds__(256)
    fwd_z_gather_kernel(const cx<T> *__restrict__ i1, const cx<T> *__restrict__ x,
                        cx<T> *__restrict__ h, const int *__restrict__ nst,
                        const int *__restrict__ smap, const T *__restrict__ kin,
                        const T *__restrict__ evals, int nk, int nb, int npwx, int nsm, int n3,
                        T scale, long long rows, St st, const cx<T> *__restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int P = TL + 1;
  long long row = row_of_block();
  if (row >= rows) return;
  int k = (int)((row / (2 * nb)) % nk);
  int s0 = blockIdx.x * TL;
  int nl = min(TL, nst[k] - s0);
  if (nl <= 0) return;
  cx<T> *b0 = reinterpret_cast<cx<T> *>(smem_raw), *b1 = b0 + n3 * P;
  if (TR) {
    const cx<T> *src = i1 + row * n3 * (long long)nsm + s0;
    for (int e = threadIdx.x; e < n3 * TL; e += blockDim.x) {
      int j = e / TL, l = e - j * TL;
      b0[j * P + l] = l < nl ? src[(long long)j * nsm + l] : czero<T>();
    }
  } else {
    const cx<T> *src = i1 + (row * nsm + s0) * n3;
    for (int e = threadIdx.x; e < n3 * TL; e += blockDim.x) {
      int l = e / n3, j = e - l * n3;
      b0[j * P + l] = l < nl ? src[(long long)l * n3 + j] : czero<T>();
    }
  }
  __syncthreads();
  cx<T> *res = tile_fft<T, TL>(b0, b1, n3, st, tw, -1);
  const int *mp = smap + ((long long)k * nsm + s0) * n3;
  T e_n = evals[(row / 2) % (2LL * nk * nb)];
  const T *kk = kin + (long long)k * npwx;
  const cx<T> *xrow = x + row * npwx;
  cx<T> *hrow = h + row * npwx;
  for (int e = threadIdx.x; e < n3 * TL; e += blockDim.x) {
    int l = e / n3, j = e - l * n3;
    if (l >= nl) continue;
    int g = mp[l * n3 + j];
    if (g < 0) continue;
    cx<T> r = res[j * P + l];
    cx<T> xv = xrow[g];
    T d = kk[g] - e_n;
    hrow[g] = mk<T>(r.x * scale + d * xv.x, r.y * scale + d * xv.y);
  }
}

constexpr int kZThreads = 128;

// ----------------------------------------------- register z lines (four-step)
// A z line of length N = N1 * N2 is split over N1 neighbouring lanes: lane n1
// transforms x[n1 + N1 n2] over n2 (N2 points, registers), multiplies by
// w_N^(n1 k2), and the N1-point transforms across the lanes (warp shuffles) leave
// lane n1 holding X[N2 k1 + k2] for one k1 and every k2:
//   X[N2 k1 + k2] = sum_n1 w_N1^(n1 k1) w_N^(n1 k2) sum_n2 x[n1 + N1 n2] w_N2^(n2 k2).
// For N1 = 4 the cross-lane transform is two radix-2 exchanges (even/odd n1, then
// the halves), which leaves lane n1 with k1 = {0, 2, 1, 3}[n1].
template <class T, int N1, int N2, int DIR>
__device__ __forceinline__ int zline_fft(cx<T> (&a)[N2], int n1, const RegTw<T, N2> &tw2,
                                         const RegTw<T, N1 * N2> &twn) {
  constexpr int N = N1 * N2;
  RegPlan<N2>::template run<T, DIR>(a, tw2);
  if constexpr (N1 == 1) {
    return 0;
  } else {
    static_assert(N1 == 4, "cross-lane radix");
#pragma unroll
    for (int k2 = 1; k2 < N2; ++k2) {
      cx<T> w = twn.w[(n1 * k2) % N];
      if (DIR < 0) w.y = -w.y;
      a[k2] = cmul<T>(a[k2], w);
    }
    const bool hi2 = (n1 & 2) != 0, odd = (n1 & 1) != 0;
    // (A0 + A2, A1 + A3, A0 - A2, A1 - A3) on lanes 0..3
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      cx<T> p;
      p.x = __shfl_xor_sync(0xffffffffu, a[k2].x, 2);
      p.y = __shfl_xor_sync(0xffffffffu, a[k2].y, 2);
      a[k2] = hi2 ? csub<T>(p, a[k2]) : cadd<T>(a[k2], p);
    }
    // X[c + 2d] = E_c + (-1)^d w4^c O_c : lane 0 -> X0, 1 -> X2, 2 -> X1, 3 -> X3
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      cx<T> p;
      p.x = __shfl_xor_sync(0xffffffffu, a[k2].x, 1);
      p.y = __shfl_xor_sync(0xffffffffu, a[k2].y, 1);
      cx<T> o = odd ? a[k2] : p;  // O_c
      const cx<T> e = odd ? p : a[k2];
      if (hi2) o = DIR > 0 ? mk<T>(-o.y, o.x) : mk<T>(o.y, -o.x);  // w4^1 O_1
      a[k2] = odd ? csub<T>(e, o) : cadd<T>(e, o);
    }
    return n1 == 0 ? 0 : n1 == 1 ? 2 : n1 == 2 ? 1 : 3;
  }
}

// Shared-memory staging of the register Z passes (FP32, four lanes per line).  Each
// lane ends its transform holding X[N2 k1 + j] for its own k1.  The inverse pass
// writes a warp's LW = 8 lines of the [row][stick][j3] buffer as one contiguous block
// (full 32-byte sectors instead of 8-byte stores strided over four lanes); the forward
// pass transposes so that lane n1 holds X[n1 + 4 j] and the four lanes of a line
// scatter to consecutive plane waves (the k+q spheres are stored stick by stick).
// Position p = N2 k1 + j of line l sits at l S + k1 (N2 + 1) + j; with S = 4 (N2 + 1)
// (= 4 mod 16 for N2 = 0 mod 4) both the per-lane accesses and the block copies are
// free of bank conflicts.
template <class T, int N1, int N2, bool TR> struct ZStage {
  static constexpr bool on = sizeof(T) == 4 && N1 == 4 && N2 <= 36 && !TR;
  static constexpr int LW = 32 / N1, S = N1 * (N2 + 1);
  static constexpr int IT = LW * N1 * N2 / 32;  // block elements per lane (= N2)
};

// Inverse Z pass in registers: sphere coefficients gathered straight into the
// lanes' registers, sticks written as [row][stick][j3] (TR = false) or
// [row][j3][stick] (TR = true).
template <class T, int N1, int N2, bool TR>
__global__ void __launch_bounds__(kZThreads)
    inv_z_reg_kernel(const cx<T> *__restrict__ x, cx<T> *__restrict__ i1,
                     const int *__restrict__ nst, const int *__restrict__ smap, int nk, int nb,
                     int npwx, int nsm, T scale, long long rows, const int4 *__restrict__ runs,
                     const RegTw<T, N2> tw2, const RegTw<T, N1 * N2> twn) {
  constexpr int N = N1 * N2, LPB = kZThreads / N1;
  const long long row = row_of_block();
  if (row >= rows) return;
  const int k = (int)((row / (2 * nb)) % nk);
  const int line = blockIdx.x * LPB + threadIdx.x / N1, n1 = threadIdx.x % N1;
  const bool valid = line < __ldg(nst + k);
  const cx<T> *xrow = x + row * npwx;
  cx<T> a[N2];
  bool filled = false;
  cx<T> *ws = nullptr;
  if constexpr (ZStage<T, N1, N2, TR>::on) {
    using Z = ZStage<T, N1, N2, TR>;
    __shared__ cx<T> zs[kZThreads / 32][Z::LW * Z::S];
    __shared__ int4 zd[kZThreads / 32][Z::LW + 1];
    ws = zs[threadIdx.x >> 5];
    if (runs) {
      // the warp's sticks are consecutive, so their plane waves are one contiguous run
      // of x: read it coalesced into the lines' natural j3 slots (zeros elsewhere)
      const int lane = threadIdx.x & 31, ll = lane / N1;
      const int l0 = blockIdx.x * LPB + (threadIdx.x >> 5) * Z::LW;
      const int nv = min(max(__ldg(nst + k) - l0, 0), Z::LW);
      int4 *wd = zd[threadIdx.x >> 5];
      if (lane <= nv) wd[lane] = __ldg(runs + (long long)k * (nsm + 1) + l0 + lane);
      for (int e = lane; e < Z::LW * Z::S; e += 32) ws[e] = czero<T>();
      __syncwarp();
      if (nv > 0) {
        const int g1 = wd[nv].x;
        for (int e = wd[0].x + lane; e < g1; e += 32) {
          int l = 0;
#pragma unroll
          for (int t = 1; t < Z::LW; ++t) l += (t < nv && e >= wd[t].x) ? 1 : 0;
          const int4 d = wd[l];
          const int rho = e - d.x;
          const int z = rho < d.y ? d.z + rho : d.w + (rho - d.y);
          if ((unsigned)z < (unsigned)N) ws[l * Z::S + z] = cscale<T>(xrow[e], scale);
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < N2; ++j) a[j] = ws[ll * Z::S + n1 + N1 * j];
      __syncwarp();
      filled = true;
    }
  }
  if (!filled) {
    const int *mp = smap + ((long long)k * nsm + (valid ? line : 0)) * N;
#pragma unroll
    for (int j = 0; j < N2; ++j) {
      const int g = valid ? __ldg(mp + n1 + N1 * j) : -1;
      a[j] = g >= 0 ? cscale<T>(xrow[g], scale) : czero<T>();
    }
  }
  const int k1 = zline_fft<T, N1, N2, +1>(a, n1, tw2, twn);
  if constexpr (ZStage<T, N1, N2, TR>::on) {
    // the warp's lines through shared memory, then one contiguous block per warp
    using Z = ZStage<T, N1, N2, TR>;
    const int ll = (threadIdx.x & 31) / N1, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < N2; ++j) ws[ll * Z::S + k1 * (N2 + 1) + j] = a[j];
    __syncwarp();
    const int l0 = blockIdx.x * LPB + (threadIdx.x >> 5) * Z::LW;
    const int nv = min(max(__ldg(nst + k) - l0, 0), Z::LW);
    cx<T> *o = i1 + (row * nsm + l0) * N;
#pragma unroll
    for (int i = 0; i < Z::IT; ++i) {
      const int e = lane + 32 * i, l = e / N, p = e - l * N, q = p / N2;
      if (e < nv * N) o[e] = ws[l * Z::S + q * (N2 + 1) + (p - q * N2)];
    }
    return;
  }
  if (!valid) return;
  if (TR) {
    cx<T> *o = i1 + row * N * (long long)nsm + line;
#pragma unroll
    for (int j = 0; j < N2; ++j) o[(long long)(N2 * k1 + j) * nsm] = a[j];
  } else {
    cx<T> *o = i1 + (row * nsm + line) * N + N2 * k1;
#pragma unroll
    for (int j = 0; j < N2; ++j) o[j] = a[j];
  }
}

// Forward Z pass in registers, scattered to the sphere with + (kin - e) x.
template <class T, int N1, int N2, bool TR>
__global__ void __launch_bounds__(kZThreads)
    fwd_z_reg_kernel(const cx<T> *__restrict__ i1, const cx<T> *__restrict__ x,
                     cx<T> *__restrict__ h, const int *__restrict__ nst,
                     const int *__restrict__ smap, const T *__restrict__ kin,
                     const T *__restrict__ evals, int nk, int nb, int npwx, int nsm, T scale,
                     long long rows, const int4 *__restrict__ runs, const RegTw<T, N2> tw2,
                     const RegTw<T, N1 * N2> twn) {
  constexpr int N = N1 * N2, LPB = kZThreads / N1;
  const long long row = row_of_block();
  if (row >= rows) return;
  const int k = (int)((row / (2 * nb)) % nk);
  const int line = blockIdx.x * LPB + threadIdx.x / N1, n1 = threadIdx.x % N1;
  const bool valid = line < __ldg(nst + k);
  const int ln = valid ? line : 0;
  cx<T> a[N2];
  if (TR) {
    const cx<T> *src = i1 + row * N * (long long)nsm + ln;
#pragma unroll
    for (int j = 0; j < N2; ++j) a[j] = valid ? src[(long long)(n1 + N1 * j) * nsm] : czero<T>();
  } else {
    const cx<T> *src = i1 + (row * nsm + ln) * N;
#pragma unroll
    for (int j = 0; j < N2; ++j) a[j] = valid ? src[n1 + N1 * j] : czero<T>();
  }
  const int k1 = zline_fft<T, N1, N2, -1>(a, n1, tw2, twn);
  const T e_n = evals[(row / 2) % (2LL * nk * nb)];
  const T *kk = kin + (long long)k * npwx;
  const cx<T> *xrow = x + row * npwx;
  cx<T> *hrow = h + row * npwx;
  if constexpr (ZStage<T, N1, N2, TR>::on) {
    using Z = ZStage<T, N1, N2, TR>;
    __shared__ cx<T> zs[kZThreads / 32][Z::LW * Z::S];
    __shared__ int4 zd[kZThreads / 32][Z::LW + 1];
    cx<T> *ws = zs[threadIdx.x >> 5];
    const int ll = (threadIdx.x & 31) / N1, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < N2; ++j) ws[ll * Z::S + k1 * (N2 + 1) + j] = a[j];
    if (runs) {
      // the warp's sticks are one contiguous run of plane waves: write it coalesced,
      // each plane wave reading its line's transform at its j3
      const int l0 = blockIdx.x * LPB + (threadIdx.x >> 5) * Z::LW;
      const int nv = min(max(__ldg(nst + k) - l0, 0), Z::LW);
      int4 *wd = zd[threadIdx.x >> 5];
      if (lane <= nv) wd[lane] = __ldg(runs + (long long)k * (nsm + 1) + l0 + lane);
      __syncwarp();
      if (nv == 0) return;
      const int g1 = wd[nv].x;
      for (int e = wd[0].x + lane; e < g1; e += 32) {
        int l = 0;
#pragma unroll
        for (int t = 1; t < Z::LW; ++t) l += (t < nv && e >= wd[t].x) ? 1 : 0;
        const int4 d = wd[l];
        const int rho = e - d.x;
        const int z = min(max(rho < d.y ? d.z + rho : d.w + (rho - d.y), 0), N - 1);
        const int q = z / N2;
        const cx<T> v = ws[l * Z::S + q * (N2 + 1) + (z - q * N2)];
        const cx<T> xv = xrow[e];
        const T dd = kk[e] - e_n;
        hrow[e] = mk<T>(v.x * scale + dd * xv.x, v.y * scale + dd * xv.y);
      }
      return;
    }
    // otherwise transpose through shared memory so that lane n1 holds X[n1 + N1 j]: the
    // four lanes of a line then scatter to consecutive plane waves of the stick
    __syncwarp();
#pragma unroll
    for (int j = 0; j < N2; ++j)
      a[j] = ws[ll * Z::S + (N1 * j / N2) * (N2 + 1) + (N1 * j) % N2 + n1];
    if (!valid) return;
    const int *mp = smap + ((long long)k * nsm + line) * N + n1;
#pragma unroll
    for (int j = 0; j < N2; ++j) {
      const int g = __ldg(mp + N1 * j);
      if (g < 0) continue;
      const cx<T> xv = xrow[g];
      const T d = kk[g] - e_n;
      hrow[g] = mk<T>(a[j].x * scale + d * xv.x, a[j].y * scale + d * xv.y);
    }
    return;
  }
  if (!valid) return;
  const int *mp = smap + ((long long)k * nsm + line) * N + N2 * k1;
#pragma unroll
  for (int j = 0; j < N2; ++j) {
    const int g = __ldg(mp + j);
    if (g < 0) continue;
    const cx<T> xv = xrow[g];
    const T d = kk[g] - e_n;
    hrow[g] = mk<T>(a[j].x * scale + d * xv.x, a[j].y * scale + d * xv.y);
  }
}

// ------------------------------------------- register-line variants (x, y axes)
// One thread per line, the whole line in registers (regfft.cuh); neighbouring
// threads own neighbouring lines, so each load/store of a warp is coalesced.
constexpr int kRegThreads = 128;   // default threads per CTA (tuned: 64, 128, 256)
constexpr int kRegMaxThreads = 256;

template <class T, int N1>
__global__ void __launch_bounds__(kRegMaxThreads)
    inv_x_reg_kernel(const cx<T> *__restrict__ i2, cx<T> *__restrict__ xr,
                     const int *__restrict__ plof, int nk, int nb, int npm, long long n23,
                     long long nr, long long rows, const RegTw<T, N1> tw) {
  long long row = row_of_block();
  if (row >= rows) return;
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n23) return;
  int k = (int)((row / (2 * nb)) % nk);
  const int *po = plof + (long long)k * N1;
  const cx<T> *src = i2 + row * npm * n23 + c;
  cx<T> a[N1];
#pragma unroll
  for (int j = 0; j < N1; ++j) {
    int p = __ldg(po + j);
    a[j] = p >= 0 ? src[(long long)p * n23] : czero<T>();
  }
  RegPlan<N1>::template run<T, +1>(a, tw);
  cx<T> *o = xr + row * nr + c;
#pragma unroll
  for (int j = 0; j < N1; ++j) o[(long long)j * n23] = a[j];
}

template <class T, int N2>
__global__ void __launch_bounds__(kRegMaxThreads)
    inv_y_reg_kernel(const cx<T> *__restrict__ i1, cx<T> *__restrict__ i2,
                     const int *__restrict__ npl, const int *__restrict__ sid, int nk, int nb,
                     int nsm, int npm, int n3, long long rows, const RegTw<T, N2> tw) {
  long long row = row_of_block();
  if (row >= rows) return;
  int k = (int)((row / (2 * nb)) % nk);
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (plane, j3)
  int p = (int)(idx / n3), j3 = (int)(idx - (long long)p * n3);
  if (p >= __ldg(npl + k)) return;
  const int *sd = sid + ((long long)k * npm + p) * N2;
  const cx<T> *src = i1 + row * nsm * (long long)n3 + j3;
  cx<T> a[N2];
#pragma unroll
  for (int j = 0; j < N2; ++j) {
    int s = __ldg(sd + j);
    a[j] = s >= 0 ? src[(long long)s * n3] : czero<T>();
  }
  RegPlan<N2>::template run<T, +1>(a, tw);
  cx<T> *o = i2 + ((row * npm + p) * N2) * (long long)n3 + j3;
#pragma unroll
  for (int j = 0; j < N2; ++j) o[(long long)j * n3] = a[j];
}

// Local products, elementwise and in place over x(r): one thread per (band-side,
// point) handles that band-side for every stacked vector, so U(r) is read once.
//   t0 = [vl + s bz] x0 + s(bx - i by) x1 + (v0 + s v3) u0 + s(v1 - i v2) u1
//   t1 = s(bx + i by) x0 + [vl - s bz] x1 + s(v1 + i v2) u0 + (v0 - s v3) u1
template <class T>
__global__ void __launch_bounds__(256)
    product_group_kernel(cx<T> *__restrict__ xr, const cx<T> *__restrict__ ur,
                         const T *__restrict__ vloc, const T *__restrict__ bf,
                         const cx<T> *__restrict__ v, int nk, int nb, long long nr, int nvec) {
  const long long bs1 = row_of_block();  // band-side of one vector
  const long long nbs1 = 2LL * nk * nb;
  if (bs1 >= nbs1) return;
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nr) return;
  const T s = (bs1 / ((long long)nk * nb)) == 0 ? T(1) : T(-1);
  const cx<T> u0 = ur[2 * bs1 * nr + r], u1 = ur[(2 * bs1 + 1) * nr + r];
  const T vl = vloc[r], bx = bf[r], by = bf[nr + r], bz = bf[2 * nr + r];
  const cx<T> h01 = mk<T>(s * bx, -s * by), h10 = mk<T>(s * bx, s * by);
  for (int vec = 0; vec < nvec; ++vec) {
    const cx<T> *vv = v + (long long)vec * 4 * nr;
    const cx<T> v0 = vv[r], v1 = vv[nr + r], v2 = vv[2 * nr + r], v3 = vv[3 * nr + r];
    const long long r0 = 2 * (vec * nbs1 + bs1);
    cx<T> x0 = xr[r0 * nr + r], x1 = xr[(r0 + 1) * nr + r];
    cx<T> t0 = cscale<T>(x0, vl + s * bz);
    cfma<T>(t0, h01, x1);
    cfma<T>(t0, mk<T>(v0.x + s * v3.x, v0.y + s * v3.y), u0);
    cfma<T>(t0, mk<T>(s * (v1.x + v2.y), s * (v1.y - v2.x)), u1);
    cx<T> t1 = cscale<T>(x1, vl - s * bz);
    cfma<T>(t1, h10, x0);
    cfma<T>(t1, mk<T>(s * (v1.x - v2.y), s * (v1.y + v2.x)), u0);
    cfma<T>(t1, mk<T>(v0.x - s * v3.x, v0.y - s * v3.y), u1);
    xr[r0 * nr + r] = t0;
    xr[(r0 + 1) * nr + r] = t1;
  }
}

// Forward X pass in registers over the products; keeps only the sphere's planes.
template <class T, int N1>
__global__ void __launch_bounds__(kRegMaxThreads)
    fwd_x_reg_kernel(const cx<T> *__restrict__ xr, cx<T> *__restrict__ i2,
                     const int *__restrict__ plof, int nk, int nb, int npm, long long n23,
                     long long nr, long long rows, const RegTw<T, N1> tw) {
  long long row = row_of_block();
  if (row >= rows) return;
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n23) return;
  int k = (int)((row / (2 * nb)) % nk);
  const cx<T> *src = xr + row * nr + c;
  cx<T> a[N1];
#pragma unroll
  for (int j = 0; j < N1; ++j) a[j] = src[(long long)j * n23];
  RegPlan<N1>::template run<T, -1>(a, tw);
  const int *po = plof + (long long)k * N1;
  cx<T> *o = i2 + row * npm * n23 + c;
#pragma unroll
  for (int j = 0; j < N1; ++j) {
    int p = __ldg(po + j);
    if (p >= 0) o[(long long)p * n23] = a[j];
  }
}

template <class T, int N2>
__global__ void __launch_bounds__(kRegMaxThreads)
    fwd_y_reg_kernel(const cx<T> *__restrict__ i2, cx<T> *__restrict__ i1,
                     const int *__restrict__ npl, const int *__restrict__ sid, int nk, int nb,
                     int nsm, int npm, int n3, long long rows, const RegTw<T, N2> tw) {
  long long row = row_of_block();
  if (row >= rows) return;
  int k = (int)((row / (2 * nb)) % nk);
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int p = (int)(idx / n3), j3 = (int)(idx - (long long)p * n3);
  if (p >= __ldg(npl + k)) return;
  const cx<T> *src = i2 + ((row * npm + p) * N2) * (long long)n3 + j3;
  cx<T> a[N2];
#pragma unroll
  for (int j = 0; j < N2; ++j) a[j] = src[(long long)j * n3];
  RegPlan<N2>::template run<T, -1>(a, tw);
  const int *sd = sid + ((long long)k * npm + p) * N2;
  cx<T> *o = i1 + row * nsm * (long long)n3 + j3;
#pragma unroll
  for (int j = 0; j < N2; ++j) {
    int s = __ldg(sd + j);
    if (s >= 0) o[(long long)s * n3] = a[j];
  }
}

// ------------------------------------------- fused Y + X line passes
// One CTA per (row, chunk of kJ3 consecutive z planes) of a square x-y grid: the Y
// lines of the sphere's planes, then the X lines of the whole box, the planes held in
// shared memory between the two, so the plane buffer never reaches HBM.  Every line is
// transformed in one thread's registers by the same plan and in the same order as in
// the separate passes above, so the results are identical to theirs.
// Shared memory yb[p][j2][jj] (p < nplane, j2 < N, jj < kJ3): the plane stride is an
// odd multiple of 8 elements, so the two half-warp phases of a warp's 8-byte accesses
// (lanes (p, jj), p = 0..3) fall on disjoint banks.
constexpr int kJ3 = 8;
template <int N> __host__ __device__ constexpr int yx_pstride() {
  return (N * kJ3) % 16 == 8 ? N * kJ3 : N * kJ3 + 8;
}
template <int N> constexpr int yx_threads() { return 32 * ((N * kJ3 + 63) / 64); }
constexpr int kYXMaxThreads = 192;

template <class T, int N>
__global__ void __launch_bounds__(kYXMaxThreads)
    inv_yx_reg_kernel(const cx<T> *__restrict__ i1, cx<T> *__restrict__ xr,
                      const int *__restrict__ npl, const int *__restrict__ sid,
                      const int *__restrict__ plof, int nk, int nb, int nsm, int npm, int n3,
                      long long nr, long long rows, const RegTw<T, N> tw) {
  extern __shared__ float4 yx_smem[];
  cx<T> *yb = reinterpret_cast<cx<T> *>(yx_smem);
  constexpr int PS = yx_pstride<N>();
  const long long row = row_of_block();
  if (row >= rows) return;  // uniform over the CTA
  const int k = (int)((row / (2 * nb)) % nk);
  const int j3c = blockIdx.x * kJ3;
  const int np = __ldg(npl + k);
  const long long n23 = (long long)N * n3;
  const cx<T> *src = i1 + row * nsm * (long long)n3;
  // Y lines of the sphere's planes: (plane p, z plane j3c + jj)
  for (int t = threadIdx.x; t < np * kJ3; t += blockDim.x) {
    const int p = t / kJ3, jj = t - p * kJ3, j3 = j3c + jj;
    const bool in = j3 < n3;
    const int *sd = sid + ((long long)k * npm + p) * N;
    cx<T> a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int st = __ldg(sd + j);
      a[j] = (in && st >= 0) ? src[(long long)st * n3 + j3] : czero<T>();
    }
    RegPlan<N>::template run<T, +1>(a, tw);
    cx<T> *o = yb + p * PS + jj;
#pragma unroll
    for (int j = 0; j < N; ++j) o[j * kJ3] = a[j];
  }
  __syncthreads();
  // X lines of the box: (j2, z plane j3c + jj)
  const int *po = plof + (long long)k * N;
  cx<T> *dst = xr + row * nr;
  for (int t = threadIdx.x; t < N * kJ3; t += blockDim.x) {
    const int j2 = t / kJ3, jj = t - j2 * kJ3, j3 = j3c + jj;
    cx<T> a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int p = __ldg(po + j);
      a[j] = p >= 0 ? yb[p * PS + j2 * kJ3 + jj] : czero<T>();
    }
    RegPlan<N>::template run<T, +1>(a, tw);
    if (j3 < n3) {
      cx<T> *o = dst + (long long)j2 * n3 + j3;
#pragma unroll
      for (int j = 0; j < N; ++j) o[j * n23] = a[j];
    }
  }
}

// Forward: X lines of the box (keeping the sphere's planes) into shared memory, then
// the Y lines of those planes written to the sphere's sticks.
template <class T, int N>
__global__ void __launch_bounds__(kYXMaxThreads)
    fwd_xy_reg_kernel(const cx<T> *__restrict__ xr, cx<T> *__restrict__ i1,
                      const int *__restrict__ npl, const int *__restrict__ sid,
                      const int *__restrict__ plof, int nk, int nb, int nsm, int npm, int n3,
                      long long nr, long long rows, const RegTw<T, N> tw) {
  extern __shared__ float4 yx_smem[];
  cx<T> *yb = reinterpret_cast<cx<T> *>(yx_smem);
  constexpr int PS = yx_pstride<N>();
  const long long row = row_of_block();
  if (row >= rows) return;  // uniform over the CTA
  const int k = (int)((row / (2 * nb)) % nk);
  const int j3c = blockIdx.x * kJ3;
  const int np = __ldg(npl + k);
  const long long n23 = (long long)N * n3;
  const int *po = plof + (long long)k * N;
  const cx<T> *src = xr + row * nr;
  for (int t = threadIdx.x; t < N * kJ3; t += blockDim.x) {
    const int j2 = t / kJ3, jj = t - j2 * kJ3, j3 = j3c + jj;
    const bool in = j3 < n3;
    const cx<T> *sp = src + (long long)j2 * n3 + j3;
    cx<T> a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = in ? sp[j * n23] : czero<T>();
    RegPlan<N>::template run<T, -1>(a, tw);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int p = __ldg(po + j);
      if (p >= 0) yb[p * PS + j2 * kJ3 + jj] = a[j];
    }
  }
  __syncthreads();
  cx<T> *dst = i1 + row * nsm * (long long)n3;
  for (int t = threadIdx.x; t < np * kJ3; t += blockDim.x) {
    const int p = t / kJ3, jj = t - p * kJ3, j3 = j3c + jj;
    const cx<T> *ys = yb + p * PS + jj;
    cx<T> a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = ys[j * kJ3];
    RegPlan<N>::template run<T, -1>(a, tw);
    if (j3 < n3) {
      const int *sd = sid + ((long long)k * npm + p) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int st = __ldg(sd + j);
        if (st >= 0) dst[(long long)st * n3 + j3] = a[j];
      }
    }
  }
}

template <class T> const cx<T> *tw_of(const AxisPlan &a) {
  if constexpr (sizeof(T) == 8)
    return a.tw_d;
  else
    return a.tw_f;
}

inline dim3 grid_rows(unsigned bx, long long rows) {
  long long y = rows, z = 1;
  while (y > 65535) {
    z *= 2;
    y = (rows + z - 1) / z;
  }
  return dim3(bx, (unsigned)y, (unsigned)z);
}

template <class K>
void set_smem(K kernel, size_t bytes) {
  TDLZ_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bytes));
}

constexpr int kTL = 16;

// Register z-line plan for length n3: (lanes per line, points per lane), or (0, 0)
// when n3 is neither a register length nor four times one.
inline void z_plan(int n3, int &n1, int &n2) {
  n1 = n2 = 0;
  if (reg_fft_length(n3)) {
    n1 = 1;
    n2 = n3;
  } else if (n3 % 4 == 0 && (n3 / 4 == 24 || n3 / 4 == 36 || n3 / 4 == 48)) {
    n1 = 4;
    n2 = n3 / 4;
  }
}

// Launch ZKERNEL<T, N1, N2, TR> for the z plan (n1, n2); leaves ok = false otherwise.
#define TDLZ_Z_LAUNCH(zn1, zn2, ZKERNEL, TRV, grid, ...)                                   \
  do {                                                                                   \
    ok = true;                                                                           \
    if (zn1 == 1 && zn2 == 12) ZKERNEL<T, 1, 12, TRV><<<grid, kZThreads, 0, st>>>(__VA_ARGS__, regtw<T, 12>(), regtw<T, 12>()); \
    else if (zn1 == 1 && zn2 == 16) ZKERNEL<T, 1, 16, TRV><<<grid, kZThreads, 0, st>>>(__VA_ARGS__, regtw<T, 16>(), regtw<T, 16>()); \
    else if (zn1 == 1 && zn2 == 24) ZKERNEL<T, 1, 24, TRV><<<grid, kZThreads, 0, st>>>(__VA_ARGS__, regtw<T, 24>(), regtw<T, 24>()); \
    else if (zn1 == 1 && zn2 == 36) ZKERNEL<T, 1, 36, TRV><<<grid, kZThreads, 0, st>>>(__VA_ARGS__, regtw<T, 36>(), regtw<T, 36>()); \
    else if (zn1 == 1 && zn2 == 45) ZKERNEL<T, 1, 45, TRV><<<grid, kZThreads, 0, st>>>(__VA_ARGS__, regtw<T, 45>(), regtw<T, 45>()); \
    else if (zn1 == 1 && zn2 == 48) ZKERNEL<T, 1, 48, TRV><<<grid, kZThreads, 0, st>>>(__VA_ARGS__, regtw<T, 48>(), regtw<T, 48>()); \
    else if (zn1 == 4 && zn2 == 24) ZKERNEL<T, 4, 24, TRV><<<grid, kZThreads, 0, st>>>(__VA_ARGS__, regtw<T, 24>(), regtw<T, 96>()); \
    else if (zn1 == 4 && zn2 == 36) ZKERNEL<T, 4, 36, TRV><<<grid, kZThreads, 0, st>>>(__VA_ARGS__, regtw<T, 36>(), regtw<T, 144>()); \
    else if (zn1 == 4 && zn2 == 48) ZKERNEL<T, 4, 48, TRV><<<grid, kZThreads, 0, st>>>(__VA_ARGS__, regtw<T, 48>(), regtw<T, 192>()); \
    else ok = false;                                                                     \
  } while (0)

// Register-line transforms: FP32 up to length 48, FP64 up to 45 (spill-free budget).
template <class T> bool use_reg_lines(int n) {
  return reg_fft_length(n) && (sizeof(T) == 4 || n <= 45);
}

// Shared memory of a fused Y + X CTA (the sphere's planes of kJ3 z planes).
size_t yx_smem_bytes(const QSlot &s, size_t elem) {
  int ps = 0;
  switch (s.fft[0]) {
    case 12: ps = yx_pstride<12>(); break;
    case 16: ps = yx_pstride<16>(); break;
    case 24: ps = yx_pstride<24>(); break;
    case 36: ps = yx_pstride<36>(); break;
    case 45: ps = yx_pstride<45>(); break;
    case 48: ps = yx_pstride<48>(); break;
    default: return 0;
  }
  return (size_t)s.nplane_max * ps * elem;
}

// Launch KERNEL<T, N> with the fused Y + X CTA shape for the register-line lengths.
#define TDLZ_YX_LAUNCH(n, KERNEL, rows, ...)                                              \
  switch (n) {                                                                           \
    case 12: TDLZ_YX_ONE(12, KERNEL, rows, __VA_ARGS__); break;                          \
    case 16: TDLZ_YX_ONE(16, KERNEL, rows, __VA_ARGS__); break;                          \
    case 24: TDLZ_YX_ONE(24, KERNEL, rows, __VA_ARGS__); break;                          \
    case 36: TDLZ_YX_ONE(36, KERNEL, rows, __VA_ARGS__); break;                          \
    case 45: TDLZ_YX_ONE(45, KERNEL, rows, __VA_ARGS__); break;                          \
    case 48: if constexpr (sizeof(T) == 4) { TDLZ_YX_ONE(48, KERNEL, rows, __VA_ARGS__); } break; \
    default: break;                                                                      \
  }
#define TDLZ_YX_ONE(NN, KERNEL, rows, ...)                                                \
  {                                                                                      \
    const size_t sm = yx_smem_bytes(s, sizeof(cx<T>));                                   \
    set_smem(KERNEL<T, NN>, sm);                                                         \
    KERNEL<T, NN><<<grid_rows((unsigned)((n3 + kJ3 - 1) / kJ3), rows), yx_threads<NN>(), sm, \
                    st>>>(__VA_ARGS__, regtw<T, NN>());                                  \
  }

}  // namespace

template <class T> bool yx_fused_supported(const QSlot &s) {
  // FP32 only: the FP64 path is bound by the FP64 pipe, and its fused lines (176-255
  // registers, spilling at 45 points) ran the C2 step 10% slower than the separate passes
  if (sizeof(T) == 8) return false;
  const size_t sm = yx_smem_bytes(s, sizeof(cx<T>));
  return s.fft[0] == s.fft[1] && use_reg_lines<T>(s.fft[0]) && sm > 0 && sm <= 227 * 1024;
}
template bool yx_fused_supported<float>(const QSlot &);
template bool yx_fused_supported<double>(const QSlot &);

void build_stick_tables(QSlot &s, const std::vector<int> &idx_kq) {
  const int n1 = s.fft[0], n2 = s.fft[1], n3 = s.fft[2];
  const int nk = s.nk, npwx = s.npwx;
  std::vector<std::vector<int>> sticks(nk), planes(nk);
  std::vector<std::vector<int>> stick_of_cell(nk);  // (j1*n2+j2) -> stick id
  int nsm = 0, npm = 0;
  for (int k = 0; k < nk; ++k) {
    std::vector<int> cell(n1 * n2, -1);
    std::vector<char> plane_used(n1, 0);
    for (int g = 0; g < s.npw_kq[k]; ++g) {
      int id = idx_kq[(size_t)k * npwx + g];
      int c = id / n3;
      if (cell[c] < 0) cell[c] = 0;
      plane_used[c / n2] = 1;
    }
    int cnt = 0;
    for (int c = 0; c < n1 * n2; ++c)
      if (cell[c] >= 0) {
        cell[c] = cnt++;
        sticks[k].push_back(c);
      }
    for (int j1 = 0; j1 < n1; ++j1)
      if (plane_used[j1]) planes[k].push_back(j1);
    stick_of_cell[k] = cell;
    nsm = std::max(nsm, cnt);
    npm = std::max(npm, (int)planes[k].size());
  }
  // even, so that each (row, plane) run of the [row][j3][stick] buffer starts on a 16-byte
  // boundary in FP32 (the plane stages stage it with 16-byte asynchronous copies)
  nsm = (nsm + 1) & ~1;
  s.nstick_max = nsm;
  s.nplane_max = npm;
  std::vector<int> nst(nk), smap((size_t)nk * nsm * n3, -1), npl(nk), plj((size_t)nk * npm, -1),
      plof((size_t)nk * n1, -1), sid((size_t)nk * npm * n2, -1);
  for (int k = 0; k < nk; ++k) {
    nst[k] = (int)sticks[k].size();
    npl[k] = (int)planes[k].size();
    for (int g = 0; g < s.npw_kq[k]; ++g) {
      int id = idx_kq[(size_t)k * npwx + g];
      int c = id / n3, j3 = id % n3;
      int st = stick_of_cell[k][c];
      smap[((size_t)k * nsm + st) * n3 + j3] = g;
    }
    for (int p = 0; p < npl[k]; ++p) {
      int j1 = planes[k][p];
      plj[(size_t)k * npm + p] = j1;
      plof[(size_t)k * n1 + j1] = p;
      for (int j2 = 0; j2 < n2; ++j2)
        sid[((size_t)k * npm + p) * n2 + j2] = stick_of_cell[k][j1 * n2 + j2];
    }
  }
  // Sticks as runs of the stick-major plane-wave order: run[k][st] = (first plane wave,
  // length of the first j3 run, its first j3, first j3 of the second run), run[k][nst] =
  // (npw, 0, 0, 0).  Needs every stick's j3 values to form at most two runs (true for a
  // sphere: one interval of Miller m3, split in two where it wraps); otherwise the Z
  // passes keep the per-point map.
  std::vector<int> run((size_t)nk * (nsm + 1) * 4, 0);
  bool runs_ok = true;
  for (int k = 0; k < nk && runs_ok; ++k) {
    const int *id = idx_kq.data() + (size_t)k * npwx;
    int st = -1, prev_c = -1, prev_z = -1, nrun = 0;
    for (int g = 0; g < s.npw_kq[k]; ++g) {
      const int c = id[g] / n3, z = id[g] % n3;
      int *r = nullptr;
      if (c != prev_c) {  // a new stick (cells ascend in the stick-major order)
        ++st;
        if (stick_of_cell[k][c] != st) { runs_ok = false; break; }
        r = run.data() + ((size_t)k * (nsm + 1) + st) * 4;
        r[0] = g; r[1] = 1; r[2] = z; r[3] = 0;
        nrun = 1;
      } else {
        r = run.data() + ((size_t)k * (nsm + 1) + st) * 4;
        if (z <= prev_z) { runs_ok = false; break; }
        if (z == prev_z + 1) {
          if (nrun == 1) ++r[1];
        } else if (nrun == 1) {
          r[3] = z;
          nrun = 2;
        } else {
          runs_ok = false;
          break;
        }
      }
      prev_c = c;
      prev_z = z;
    }
    if (st + 1 != nst[k]) runs_ok = false;
    int *end = run.data() + ((size_t)k * (nsm + 1) + nst[k]) * 4;
    end[0] = s.npw_kq[k];
  }
  s.st_runs = runs_ok;
  auto up = [&](DevBuf &b, const std::vector<int> &v) {
    b.alloc(v.size() * sizeof(int));
    TDLZ_CUDA_TRY(cudaMemcpy(b.p, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
  };
  up(s.st_run, run);
  up(s.st_n, nst);
  up(s.st_map, smap);
  up(s.pl_n, npl);
  up(s.pl_j1, plj);
  up(s.pl_of, plof);
  up(s.st_id, sid);
  s.nst_h = nst;
  s.npl_h = npl;
}

// Element counts and FLOPs of one pass over nvec stacked vectors, for the
// profiler's algorithmic bytes (each stage's minimum traffic for its design).
struct StageWork {
  double V, S1, S2, G, Gu;                // BR, stick, plane, grid, U-grid elements
  double z_flops, y_flops, x_flops;       // 5 N log2 N per line
};
template <class T> StageWork stage_work(const QSlot &s, int nvec) {
  StageWork w;
  const double rows = (double)s.rows() * nvec;
  const int n1 = s.fft[0], n2 = s.fft[1], n3 = s.fft[2];
  w.V = (double)s.br_elems() * nvec;
  w.S1 = rows * s.nstick_max * n3;
  w.S2 = rows * s.nplane_max * n2 * n3;
  w.G = rows * s.nr;
  w.Gu = (double)s.rows() * s.nr;
  w.z_flops = rows * s.nstick_max * 5.0 * n3 * std::log2((double)n3);
  w.y_flops = rows * s.nplane_max * n3 * 5.0 * n2 * std::log2((double)n2);
  w.x_flops = rows * (double)n2 * n3 * 5.0 * n1 * std::log2((double)n1);
  return w;
}

// h[row][i] = 0 for npw_kq[k] <= i < npwx: the sphere scatter writes every sphere point
// exactly once (each point is one (stick, j3) of its k+q sphere), so only the padding
// needs clearing before it.
template <class T>
__global__ void zero_padding_kernel(cx<T> *__restrict__ h, const int *__restrict__ npw, int nk,
                                    int nb, int npwx, long long rows) {
  const long long row = row_of_block();
  if (row >= rows) return;
  const int k = (int)((row / (2 * nb)) % nk);
  for (int i = __ldg(npw + k) + blockIdx.x * blockDim.x + threadIdx.x; i < npwx;
       i += gridDim.x * blockDim.x)
    h[row * npwx + i] = czero<T>();
}

template <class T>
void zero_padding(Context &ctx, QSlot &s, cx<T> *h, long long rows) {
  int npw_min = s.npwx;
  for (int v : s.npw_kq) npw_min = std::min(npw_min, v);
  const int pad = s.npwx - npw_min;
  if (pad <= 0) return;
  zero_padding_kernel<T><<<grid_rows((unsigned)((pad + 255) / 256), rows), 256, 0, ctx.stream>>>(
      h, s.npwkq_d.as<int>(), s.nk, s.nb, s.npwx, rows);
  TDLZ_LAUNCH_CHECK();
}

// Threads per CTA of a register-line pass (64, 128 or 256), picked by the autotuner per
// pass and problem shape; launch(rt) enqueues the pass with rt threads per CTA.  Every
// thread owns the same line whatever the CTA size, so the choice changes no result.
template <class F>
void tuned_lines(Context &ctx, const char *pass, size_t elem, int n, long long lines,
                 long long rows, F &&launch) {
  char key[160];
  snprintf(key, sizeof(key), "%s/%s/n=%d/lines=%lld/rows=%lld", pass,
           elem == 8 ? "f32" : "f64", n, lines, rows);
  ctx.tuner.pick(ctx.stream, key, {64, 128, 256}, kRegThreads, launch);
}

template <class T>
void pipeline_inverse(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *xr, cx<T> *i1, cx<T> *i2,
                      int nvec) {
  cudaStream_t st = ctx.stream;
  const int n1 = s.fft[0], n2 = s.fft[1], n3 = s.fft[2];
  const long long rows = s.rows() * nvec, n23 = (long long)n2 * n3;
  const int nsm = s.nstick_max, npm = s.nplane_max;
  const size_t c = sizeof(cx<T>);
  const StageWork wk = stage_work<T>(s, nvec);
  bool ok = false;
  {
    ProfScope ps(ctx.prof, st, ST_SCATTER, wk.V * c + wk.S1 * c, wk.z_flops);
    int zn1, zn2;
    z_plan(n3, zn1, zn2);
    if (zn1) {
      const int lpb = kZThreads / zn1;
      dim3 g = grid_rows((unsigned)((nsm + lpb - 1) / lpb), rows);
      TDLZ_Z_LAUNCH(zn1, zn2, inv_z_reg_kernel, false, g, x, i1, s.st_n.as<int>(),
                    s.st_map.as<int>(), s.nk, s.nb, s.npwx, nsm, (T)(1.0 / std::sqrt(s.omega)),
                    rows, s.st_runs ? s.st_run.as<int4>() : (const int4 *)nullptr);
    }
    if (!ok) {
      size_t sm = 2ull * n3 * (kTL + 1) * c;
      set_smem(inv_z_kernel<T, kTL>, sm);
      inv_z_kernel<T, kTL><<<grid_rows((nsm + kTL - 1) / kTL, rows), 256, sm, st>>>(
          x, i1, s.st_n.as<int>(), s.st_map.as<int>(), s.nk, s.nb, s.npwx, nsm, n3,
          (T)(1.0 / std::sqrt(s.omega)), rows, stages(s.plan.ax[2]), tw_of<T>(s.plan.ax[2]));
    }
    TDLZ_LAUNCH_CHECK();
  }
  if (sizeof(T) == 4 ? s.yx32 : s.yx64) {
    // sticks in, real-space grids out; the planes stay on chip
    ProfScope ps(ctx.prof, st, ST_FFT_INV, wk.S1 * c + wk.G * c, wk.y_flops + wk.x_flops);
    TDLZ_YX_LAUNCH(n1, inv_yx_reg_kernel, rows, i1, xr, s.pl_n.as<int>(), s.st_id.as<int>(),
                   s.pl_of.as<int>(), s.nk, s.nb, nsm, npm, n3, s.nr, rows);
    TDLZ_LAUNCH_CHECK();
    return;
  }
  // sticks in, planes out and back in, real-space grids out
  ProfScope ps(ctx.prof, st, ST_FFT_INV, wk.S1 * c + 2 * wk.S2 * c + wk.G * c,
               wk.y_flops + wk.x_flops);
  ok = use_reg_lines<T>(n2);
  if (ok) {
    tuned_lines(ctx, "inv_y", c, n2, (long long)npm * n3, rows, [&](int rt) {
      dim3 g = grid_rows((unsigned)(((long long)npm * n3 + rt - 1) / rt), rows);
      TDLZ_REG_LAUNCH(n2, inv_y_reg_kernel, g, i1, i2, s.pl_n.as<int>(), s.st_id.as<int>(),
                      s.nk, s.nb, nsm, npm, n3, rows);
      TDLZ_LAUNCH_CHECK();
    });
  }
  if (!ok) {
    size_t sm = 2ull * n2 * (kTL + 1) * c;
    set_smem(inv_y_kernel<T, kTL>, sm);
    inv_y_kernel<T, kTL><<<grid_rows((n3 + kTL - 1) / kTL, rows * npm), 256, sm, st>>>(
        i1, i2, s.pl_n.as<int>(), s.st_id.as<int>(), s.nk, s.nb, nsm, npm, n2, n3, rows,
        stages(s.plan.ax[1]), tw_of<T>(s.plan.ax[1]));
    TDLZ_LAUNCH_CHECK();
  }
  ok = use_reg_lines<T>(n1);
  if (ok) {
    tuned_lines(ctx, "inv_x", c, n1, n23, rows, [&](int rt) {
      dim3 g = grid_rows((unsigned)((n23 + rt - 1) / rt), rows);
      TDLZ_REG_LAUNCH(n1, inv_x_reg_kernel, g, i2, xr, s.pl_of.as<int>(), s.nk, s.nb, npm, n23,
                      s.nr, rows);
      TDLZ_LAUNCH_CHECK();
    });
  }
  if (!ok) {
    size_t sm = 2ull * n1 * (kTL + 1) * c;
    set_smem(inv_x_kernel<T, kTL>, sm);
    inv_x_kernel<T, kTL><<<grid_rows((unsigned)((n23 + kTL - 1) / kTL), rows), 256, sm, st>>>(
        i2, xr, s.pl_of.as<int>(), s.nk, s.nb, npm, n1, n23, s.nr, rows, stages(s.plan.ax[0]),
        tw_of<T>(s.plan.ax[0]));
    TDLZ_LAUNCH_CHECK();
  }
}

template <class T>
void pipeline_forward(Context &ctx, QSlot &s, const cx<T> *x, const cx<T> *xr, const cx<T> *ur,
                      const T *vloc, const T *bf, const cx<T> *v, const T *kin, const T *evals,
                      cx<T> *i1, cx<T> *i2, cx<T> *h, int nvec) {
  cudaStream_t st = ctx.stream;
  const int n1 = s.fft[0], n2 = s.fft[1], n3 = s.fft[2];
  const long long rows = s.rows() * nvec, nbs = rows / 2, n23 = (long long)n2 * n3;
  const int nsm = s.nstick_max, npm = s.nplane_max;
  const size_t c = sizeof(cx<T>);
  const StageWork wk = stage_work<T>(s, nvec);
  // potentials of every vector and the local fields, read once per point
  const double pot_bytes = 4.0 * nvec * s.nr * (c + sizeof(T));
  bool ok = use_reg_lines<T>(n1);
  if (ok) {
    // products in place (xr is not needed afterwards): x(r) read and written, U(r)
    // once per stacked group
    {
      ProfScope ps(ctx.prof, st, ST_PRODUCT, 2 * wk.G * c + wk.Gu * c + pot_bytes,
                   (double)nbs * s.nr * 64.0);
      const long long nbs1 = nbs / nvec;
      product_group_kernel<T><<<grid_rows((unsigned)((s.nr + 255) / 256), nbs1), 256, 0, st>>>(
          const_cast<cx<T> *>(xr), ur, vloc, bf, v, s.nk, s.nb, s.nr, nvec);
      TDLZ_LAUNCH_CHECK();
    }
    if (sizeof(T) == 4 ? s.yx32 : s.yx64) {
      // real-space grids in, sticks out; the planes stay on chip
      ProfScope ps(ctx.prof, st, ST_FFT_FWD, wk.G * c + wk.S1 * c, wk.x_flops + wk.y_flops);
      TDLZ_YX_LAUNCH(n1, fwd_xy_reg_kernel, rows, xr, i1, s.pl_n.as<int>(), s.st_id.as<int>(),
                     s.pl_of.as<int>(), s.nk, s.nb, nsm, npm, n3, s.nr, rows);
      TDLZ_LAUNCH_CHECK();
      ok = true;
    } else {
    ProfScope ps(ctx.prof, st, ST_FFT_FWD, wk.G * c + 2 * wk.S2 * c + wk.S1 * c,
                 wk.x_flops + wk.y_flops);
    tuned_lines(ctx, "fwd_x", c, n1, n23, rows, [&](int rt) {
      dim3 g = grid_rows((unsigned)((n23 + rt - 1) / rt), rows);
      TDLZ_REG_LAUNCH(n1, fwd_x_reg_kernel, g, xr, i2, s.pl_of.as<int>(), s.nk, s.nb, npm, n23,
                      s.nr, rows);
      TDLZ_LAUNCH_CHECK();
    });
    ok = use_reg_lines<T>(n2);
    if (ok) {
      tuned_lines(ctx, "fwd_y", c, n2, (long long)npm * n3, rows, [&](int rt) {
        dim3 gy = grid_rows((unsigned)(((long long)npm * n3 + rt - 1) / rt), rows);
        TDLZ_REG_LAUNCH(n2, fwd_y_reg_kernel, gy, i2, i1, s.pl_n.as<int>(), s.st_id.as<int>(),
                        s.nk, s.nb, nsm, npm, n3, rows);
        TDLZ_LAUNCH_CHECK();
      });
    }
    if (!ok) {
      size_t sm = 2ull * n2 * (kTL + 1) * c;
      set_smem(fwd_y_kernel<T, kTL>, sm);
      fwd_y_kernel<T, kTL><<<grid_rows((n3 + kTL - 1) / kTL, rows * npm), 256, sm, st>>>(
          i2, i1, s.pl_n.as<int>(), s.st_id.as<int>(), s.nk, s.nb, nsm, npm, n2, n3, rows,
          stages(s.plan.ax[1]), tw_of<T>(s.plan.ax[1]));
      TDLZ_LAUNCH_CHECK();
    }
    }
  } else {
    // X pass with the products formed in shared memory (no separate product pass)
    ProfScope ps(ctx.prof, st, ST_FFT_FWD,
                 wk.G * c + wk.Gu * c + pot_bytes + 2 * wk.S2 * c + wk.S1 * c,
                 wk.x_flops + wk.y_flops + (double)nbs * s.nr * 64.0);
    size_t sm = 4ull * n1 * (kTL + 1) * c;
    set_smem(fwd_x_product_kernel<T, kTL>, sm);
    fwd_x_product_kernel<T, kTL><<<grid_rows((unsigned)((n23 + kTL - 1) / kTL), nbs), 256, sm,
                                   st>>>(xr, ur, vloc, bf, v, i2, s.pl_n.as<int>(),
                                         s.pl_j1.as<int>(), s.nk, s.nb, npm, n1, n23, s.nr, nbs,
                                         stages(s.plan.ax[0]), tw_of<T>(s.plan.ax[0]));
    TDLZ_LAUNCH_CHECK();
    ok = use_reg_lines<T>(n2);
    if (ok) {
      tuned_lines(ctx, "fwd_y", c, n2, (long long)npm * n3, rows, [&](int rt) {
        dim3 gy = grid_rows((unsigned)(((long long)npm * n3 + rt - 1) / rt), rows);
        TDLZ_REG_LAUNCH(n2, fwd_y_reg_kernel, gy, i2, i1, s.pl_n.as<int>(), s.st_id.as<int>(),
                        s.nk, s.nb, nsm, npm, n3, rows);
        TDLZ_LAUNCH_CHECK();
      });
    }
    if (!ok) {
      size_t smy = 2ull * n2 * (kTL + 1) * c;
      set_smem(fwd_y_kernel<T, kTL>, smy);
      fwd_y_kernel<T, kTL><<<grid_rows((n3 + kTL - 1) / kTL, rows * npm), 256, smy, st>>>(
          i2, i1, s.pl_n.as<int>(), s.st_id.as<int>(), s.nk, s.nb, nsm, npm, n2, n3, rows,
          stages(s.plan.ax[1]), tw_of<T>(s.plan.ax[1]));
      TDLZ_LAUNCH_CHECK();
    }
  }
  {
    // sticks in; x read, h written on the sphere and zero on the padding
    ProfScope ps(ctx.prof, st, ST_GATHER, wk.S1 * c + 3 * wk.V * c, wk.z_flops);
    zero_padding<T>(ctx, s, h, rows);
    int zn1, zn2;
    z_plan(n3, zn1, zn2);
    ok = false;
    if (zn1) {
      const int lpb = kZThreads / zn1;
      dim3 g = grid_rows((unsigned)((nsm + lpb - 1) / lpb), rows);
      TDLZ_Z_LAUNCH(zn1, zn2, fwd_z_reg_kernel, false, g, i1, x, h, s.st_n.as<int>(),
                    s.st_map.as<int>(), kin, evals, s.nk, s.nb, s.npwx, nsm,
                    (T)(std::sqrt(s.omega) / s.nr), rows, s.st_runs ? s.st_run.as<int4>() : (const int4 *)nullptr);
    }
    if (!ok) {
      size_t sm = 2ull * n3 * (kTL + 1) * c;
      set_smem(fwd_z_gather_kernel<T, kTL>, sm);
      fwd_z_gather_kernel<T, kTL><<<grid_rows((nsm + kTL - 1) / kTL, rows), 256, sm, st>>>(
          i1, x, h, s.st_n.as<int>(), s.st_map.as<int>(), kin, evals, s.nk, s.nb, s.npwx, nsm,
          n3, (T)(std::sqrt(s.omega) / s.nr), rows, stages(s.plan.ax[2]),
          tw_of<T>(s.plan.ax[2]));
    }
    TDLZ_LAUNCH_CHECK();
  }
}

// Z passes alone, stick buffer in [row][j3][stick] order (fused plane stages).
template <class T>
void sticks_inverse(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *i1t, int nvec) {
  cudaStream_t st = ctx.stream;
  const int n3 = s.fft[2];
  const long long rows = s.rows() * nvec;
  const int nsm = s.nstick_max;
  int zn1, zn2;
  z_plan(n3, zn1, zn2);
  bool ok = false;
  if (zn1) {
    const int lpb = kZThreads / zn1;
    dim3 g = grid_rows((unsigned)((nsm + lpb - 1) / lpb), rows);
    TDLZ_Z_LAUNCH(zn1, zn2, inv_z_reg_kernel, true, g, x, i1t, s.st_n.as<int>(),
                  s.st_map.as<int>(), s.nk, s.nb, s.npwx, nsm, (T)(1.0 / std::sqrt(s.omega)),
                  rows, (const int4 *)nullptr);
  }
  if (!ok) {
    size_t sm = 2ull * n3 * (kTL + 1) * sizeof(cx<T>);
    set_smem(inv_z_kernel<T, kTL, true>, sm);
    inv_z_kernel<T, kTL, true><<<grid_rows((nsm + kTL - 1) / kTL, rows), 256, sm, st>>>(
        x, i1t, s.st_n.as<int>(), s.st_map.as<int>(), s.nk, s.nb, s.npwx, nsm, n3,
        (T)(1.0 / std::sqrt(s.omega)), rows, stages(s.plan.ax[2]), tw_of<T>(s.plan.ax[2]));
  }
  TDLZ_LAUNCH_CHECK();
}

template <class T>
void sticks_forward(Context &ctx, QSlot &s, const cx<T> *x, const cx<T> *i1t, const T *kin,
                    const T *evals, cx<T> *h, int nvec) {
  cudaStream_t st = ctx.stream;
  const int n3 = s.fft[2];
  const long long rows = s.rows() * nvec;
  const int nsm = s.nstick_max;
  zero_padding<T>(ctx, s, h, rows);
  int zn1, zn2;
  z_plan(n3, zn1, zn2);
  bool ok = false;
  if (zn1) {
    const int lpb = kZThreads / zn1;
    dim3 g = grid_rows((unsigned)((nsm + lpb - 1) / lpb), rows);
    TDLZ_Z_LAUNCH(zn1, zn2, fwd_z_reg_kernel, true, g, i1t, x, h, s.st_n.as<int>(),
                  s.st_map.as<int>(), kin, evals, s.nk, s.nb, s.npwx, nsm,
                  (T)(std::sqrt(s.omega) / s.nr), rows, (const int4 *)nullptr);
  }
  if (!ok) {
    size_t sm = 2ull * n3 * (kTL + 1) * sizeof(cx<T>);
    set_smem(fwd_z_gather_kernel<T, kTL, true>, sm);
    fwd_z_gather_kernel<T, kTL, true><<<grid_rows((nsm + kTL - 1) / kTL, rows), 256, sm, st>>>(
        i1t, x, h, s.st_n.as<int>(), s.st_map.as<int>(), kin, evals, s.nk, s.nb, s.npwx, nsm,
        n3, (T)(std::sqrt(s.omega) / s.nr), rows, stages(s.plan.ax[2]), tw_of<T>(s.plan.ax[2]));
  }
  TDLZ_LAUNCH_CHECK();
}

template void sticks_inverse<float>(Context &, QSlot &, const float2 *, float2 *, int);
template void sticks_inverse<double>(Context &, QSlot &, const double2 *, double2 *, int);
template void sticks_forward<float>(Context &, QSlot &, const float2 *, const float2 *,
                                    const float *, const float *, float2 *, int);
template void sticks_forward<double>(Context &, QSlot &, const double2 *, const double2 *,
                                     const double *, const double *, double2 *, int);
template void pipeline_inverse<double>(Context &, QSlot &, const double2 *, double2 *, double2 *,
                                       double2 *, int);
template void pipeline_inverse<float>(Context &, QSlot &, const float2 *, float2 *, float2 *,
                                      float2 *, int);
template void pipeline_forward<double>(Context &, QSlot &, const double2 *, const double2 *,
                                       const double2 *, const double *, const double *,
                                       const double2 *, const double *, const double *, double2 *,
                                       double2 *, double2 *, int);
template void pipeline_forward<float>(Context &, QSlot &, const float2 *, const float2 *,
                                      const float2 *, const float *, const float *, const float2 *,
                                      const float *, const float *, float2 *, float2 *, float2 *,
                                      int);

}  // namespace tdlz
