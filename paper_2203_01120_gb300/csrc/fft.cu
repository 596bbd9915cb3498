// Batched mixed-radix 3D FFT (see fft.cuh).
#include "fft.cuh"

#include <cmath>
#include <vector>

namespace tdlz {

namespace {

struct Stages {
  int nrad;
  int radix[8];
};

template <class T>
__device__ __forceinline__ cx<T> mul_i(cx<T> a, int dir) {  // a * (dir * i)
  return dir > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

template <class T>
__device__ __forceinline__ cx<T> root(const cx<T> *tw, int t, int dir) {
  cx<T> w = tw[t];
  if (dir < 0) w.y = -w.y;
  return w;
}

// In-register DFT of length R (R in {2,3,4,5}); w3/w5 are exp(dir 2 pi i / R).
template <class T>
__device__ __forceinline__ void small_dft(cx<T> *v, int R, int dir, cx<T> w3, cx<T> w5a,
                                          cx<T> w5b) {
  if (R == 2) {
    cx<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  } else if (R == 4) {
    cx<T> a = cadd<T>(v[0], v[2]), b = csub<T>(v[0], v[2]);
    cx<T> c = cadd<T>(v[1], v[3]), e = mul_i<T>(csub<T>(v[1], v[3]), dir);
    v[0] = cadd<T>(a, c);
    v[2] = csub<T>(a, c);
    v[1] = cadd<T>(b, e);
    v[3] = csub<T>(b, e);
  } else if (R == 3) {
    // w3 = c + i d s with c = -1/2: y1 = v0 + c s + i d s' t, y2 = v0 + c s - i d s' t
    cx<T> s = cadd<T>(v[1], v[2]), t = csub<T>(v[1], v[2]);
    cx<T> m = mk<T>(v[0].x + w3.x * s.x, v[0].y + w3.x * s.y);
    cx<T> r = mk<T>(-w3.y * t.y, w3.y * t.x);  // i * Im(w3) * t  (Im(w3) carries dir)
    v[0] = cadd<T>(v[0], s);
    v[1] = cadd<T>(m, r);
    v[2] = csub<T>(m, r);
  } else {  // R == 5, w5a = exp(dir 2 pi i/5), w5b = exp(dir 4 pi i/5)
    cx<T> a1 = cadd<T>(v[1], v[4]), b1 = csub<T>(v[1], v[4]);
    cx<T> a2 = cadd<T>(v[2], v[3]), b2 = csub<T>(v[2], v[3]);
    T c1 = w5a.x, s1 = w5a.y, c2 = w5b.x, s2 = w5b.y;  // s carry dir
    cx<T> m1 = mk<T>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    cx<T> m2 = mk<T>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    // i*(s1 b1 + s2 b2) and i*(s2 b1 - s1 b2)
    cx<T> p1 = mk<T>(-(s1 * b1.y + s2 * b2.y), s1 * b1.x + s2 * b2.x);
    cx<T> p2 = mk<T>(-(s2 * b1.y - s1 * b2.y), s2 * b1.x - s1 * b2.x);
    v[0] = cadd<T>(v[0], cadd<T>(a1, a2));
    v[1] = cadd<T>(m1, p1);
    v[4] = csub<T>(m1, p1);
    v[2] = cadd<T>(m2, p2);
    v[3] = csub<T>(m2, p2);
  }
}

// One axis pass.  A tile holds TL lines of length n in shared memory laid out
// [j][TL+1] (line index fastest, padded) so butterflies on neighbouring lines
// hit distinct banks.  S == 1: lines are contiguous rows (tile = TL rows);
// S > 1: lines have stride S and the tile takes TL consecutive inner offsets.
template <class T, int TL>
__global__ void __launch_bounds__(256) fft_axis_kernel(cx<T> *__restrict__ data, int n, long long S,
                                                      long long outer, Stages st,
                                                      const cx<T> *__restrict__ tw, int dir) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int P = TL + 1;
  cx<T> *buf0 = reinterpret_cast<cx<T> *>(smem_raw);
  cx<T> *buf1 = buf0 + (size_t)n * P;
  long long tile = blockIdx.x;
  long long base, jstride, lstride;
  int nlines;
  if (S == 1) {
    long long o0 = tile * TL;
    long long rem = outer - o0;
    nlines = rem < TL ? (int)rem : TL;
    base = o0 * n;
    jstride = 1;
    lstride = n;
  } else {
    long long tpo = (S + TL - 1) / TL;
    long long o = tile / tpo;
    long long i0 = (tile - o * tpo) * TL;
    long long rem = S - i0;
    nlines = rem < TL ? (int)rem : TL;
    base = o * (long long)n * S + i0;
    jstride = S;
    lstride = 1;
  }
  const int total = n * TL;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int j, l;
    if (S == 1) {
      l = e / n;
      j = e - l * n;
    } else {
      j = e / TL;
      l = e - j * TL;
    }
    if (l < nlines) buf0[j * P + l] = data[base + j * jstride + l * lstride];
  }
  __syncthreads();
  cx<T> w3 = czero<T>(), w5a = czero<T>(), w5b = czero<T>();
  if (n % 3 == 0) w3 = root<T>(tw, n / 3, dir);
  if (n % 5 == 0) {
    w5a = root<T>(tw, n / 5, dir);
    w5b = root<T>(tw, (2 * n) / 5, dir);
  }
  cx<T> *in = buf0, *out = buf1;
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
          if (r < R) v[r] = cmul<T>(v[r], root<T>(tw, (r * k * tstride) % n, dir));
      }
      small_dft<T>(v, R, dir, w3, w5a, w5b);
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
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int j, l;
    if (S == 1) {
      l = e / n;
      j = e - l * n;
    } else {
      j = e / TL;
      l = e - j * TL;
    }
    if (l < nlines) data[base + j * jstride + l * lstride] = in[j * P + l];
  }
}

Stages stages_of(const AxisPlan &a) {
  Stages s;
  s.nrad = a.nrad;
  for (int i = 0; i < 8; ++i) s.radix[i] = a.radix[i];
  return s;
}

template <class T, int TL>
void launch_axis(const AxisPlan &a, cx<T> *data, long long S, long long outer, int dir,
                 cudaStream_t st) {
  size_t smem = 2ull * a.n * (TL + 1) * sizeof(cx<T>);
  long long tiles = (S == 1) ? (outer + TL - 1) / TL : outer * ((S + TL - 1) / TL);
  TDLZ_CUDA_TRY(cudaFuncSetAttribute(fft_axis_kernel<T, TL>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const cx<T> *tw;
  if constexpr (sizeof(T) == 8)
    tw = a.tw_d;
  else
    tw = a.tw_f;
  fft_axis_kernel<T, TL><<<(unsigned)tiles, 256, smem, st>>>(data, a.n, S, outer, stages_of(a), tw,
                                                            dir);
  TDLZ_LAUNCH_CHECK();
}

template <class T>
void axis_pass(const AxisPlan &a, cx<T> *data, long long S, long long outer, int dir,
               cudaStream_t st) {
  if (a.n <= 64)
    launch_axis<T, 32>(a, data, S, outer, dir, st);
  else
    launch_axis<T, 16>(a, data, S, outer, dir, st);
}

}  // namespace

bool fft_length_supported(int n) {
  if (n < 1 || n > 512) return false;
  int m = n;
  for (int r : {4, 2, 3, 5})
    while (m % r == 0) m /= r;
  return m == 1;
}

void FFTPlan::init(const int fft[3]) {
  nr = 1;
  for (int d = 0; d < 3; ++d) {
    n[d] = fft[d];
    nr *= fft[d];
    AxisPlan &a = ax[d];
    a.n = fft[d];
    int m = fft[d];
    a.nrad = 0;
    for (int r : {4, 2, 3, 5})
      while (m % r == 0) {
        a.radix[a.nrad++] = r;
        m /= r;
      }
    std::vector<double2> hd(a.n);
    std::vector<float2> hf(a.n);
    for (int t = 0; t < a.n; ++t) {
      long double ang = 2.0L * 3.141592653589793238462643383279502884L * (long double)t /
                        (long double)a.n;
      hd[t] = make_double2((double)cosl(ang), (double)sinl(ang));
      hf[t] = make_float2((float)hd[t].x, (float)hd[t].y);
    }
    TDLZ_CUDA_TRY(cudaMalloc(&a.tw_d, sizeof(double2) * a.n));
    TDLZ_CUDA_TRY(cudaMalloc(&a.tw_f, sizeof(float2) * a.n));
    TDLZ_CUDA_TRY(cudaMemcpy(a.tw_d, hd.data(), sizeof(double2) * a.n, cudaMemcpyHostToDevice));
    TDLZ_CUDA_TRY(cudaMemcpy(a.tw_f, hf.data(), sizeof(float2) * a.n, cudaMemcpyHostToDevice));
  }
}

void FFTPlan::release() {
  for (auto &a : ax) {
    if (a.tw_d) cudaFree(a.tw_d);
    if (a.tw_f) cudaFree(a.tw_f);
    a.tw_d = nullptr;
    a.tw_f = nullptr;
  }
}

template <class T>
void fft3d(const FFTPlan &plan, cx<T> *data, long long batch, int dir, cudaStream_t st) {
  const long long n1 = plan.n[0], n2 = plan.n[1], n3 = plan.n[2];
  // axis 3 (contiguous): lines = batch*n1*n2, stride 1
  axis_pass<T>(plan.ax[2], data, 1, batch * n1 * n2, dir, st);
  // axis 2: stride n3, outer = batch*n1
  axis_pass<T>(plan.ax[1], data, n3, batch * n1, dir, st);
  // axis 1: stride n2*n3, outer = batch
  axis_pass<T>(plan.ax[0], data, n2 * n3, batch, dir, st);
}

template void fft3d<double>(const FFTPlan &, double2 *, long long, int, cudaStream_t);
template void fft3d<float>(const FFTPlan &, float2 *, long long, int, cudaStream_t);

}  // namespace tdlz
