// The Liouvillian of the batch representation on the GPU.
//
// y = L x with x = (X, Y) on the k+q spheres (Eq. Liouvillian_BR_q and the
// block actions after it):
//   out_X =  P_{k+q}  [ (H+_{k+q} - e_{n,k}) x_n + V'_HXC U_{n,k} ]
//   out_Y = -P+_{k+q} [ (H-_{k+q} - e_{n,k}) y_n + V'+_HXC (TU)_{n,k} ]
// Stages (one launch each, every band-side of every k batched together):
//   1  scatter x onto the grid, inverse 3D FFT          -> x(r)          (all band-sides)
//   2  response densities n', m' (Eqs. charge_dens_resp_q, spin_dens_resp_q)
//   3  Hartree at q (Eq. v_H_q): FFT, 4 pi/|q+G|^2, inverse FFT
//   4  ALSDA kernel v'_a = d_a0 v'_H + f_ab rho'_b (Eqs. v_XC_q, b_XC_q)
//   5  [v_loc + s B.sigma] x(r) + W^s U(r) (W^X = v0 + v.sigma, W^Y = v0 - v.sigma)
//   6  forward 3D FFT, gather to the k+q sphere, + (|k+q+G|^2/2 - e_n) x
//   7  V_NL: <beta|x> (split-K reduction GEMM), D mixing, beta (D <beta|x>)
//   8  P_c: <U_m|h> (split-K reduction GEMM), h - U <U|h>, row sign (Y side -)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.cuh"
#include "pipeline.cuh"
#include "planes.cuh"
#include "tc_gemm.cuh"

namespace tdlz {

namespace {

constexpr int kThreads = 256;


// ------------------------------------------------------------ grid <-> sphere
template <class T>
__global__ void scatter_rows_kernel(const cx<T> *__restrict__ x, cx<T> *__restrict__ grid,
                                    const int *__restrict__ idx, int nk, int nb, int npwx,
                                    long long nr, T scale, long long nrows) {
  long long row = blockIdx.y + (long long)gridDim.y * blockIdx.z;
  if (row >= nrows) return;
  int k = (int)((row / (2 * nb)) % nk);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npwx; g += gridDim.x * blockDim.x) {
    int ig = idx[(long long)k * npwx + g];
    if (ig >= 0) grid[row * nr + ig] = cscale<T>(x[row * npwx + g], scale);
  }
}

inline dim3 row_grid(long long nrows, int npwx) {
  unsigned bx = (unsigned)((npwx + kThreads - 1) / kThreads);
  long long y = nrows, z = 1;
  while (y > 65535) {
    z *= 2;
    y = (nrows + z - 1) / z;
  }
  return dim3(bx, (unsigned)y, (unsigned)z);
}

// ------------------------------------------------------------- density (a3)
// rho'_a(r) = sum_k w_k sum_n [ U^X_n^+ s_a x_n + t_a U^Y_n^+ s_a y_n ],
// t = (1,-1,-1,-1); fixed summation order (deterministic).
// nvec response vectors share the occupied orbitals: each U(r) value is read once
// and contracted with every vector's x(r); rho is [nvec][4][Nr].
// Block row y sums the (side, k) pairs [y*ppg, (y+1)*ppg) into partial slice y
// ([gridDim.y][nvec][4][Nr]); density_reduce_kernel adds the slices in order.
template <class T, int NV>
__global__ void __launch_bounds__(256)
    density_kernel(const cx<T> *__restrict__ ur, const cx<T> *__restrict__ xr,
                   const T *__restrict__ wk, cx<T> *__restrict__ rho, int nk, int nb,
                   long long nr, int ppg, int vstride) {
  const long long rows1 = 4LL * nk * nb;
  const int pb = blockIdx.y * ppg, pe = min(2 * nk, pb + ppg);
  rho += (long long)blockIdx.y * vstride * 4 * nr;
  if constexpr (sizeof(T) == 4) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr;
         r += (long long)gridDim.x * blockDim.x) {
      // acc[v][a] = sum over the group's (side, k) pairs and bands of w t_a U^+ s_a x, with
      // t = (1, -1, -1, -1) on the Y side: U is scaled once per band by w t_1 (= +-w), and
      // the charge part (t_0 = 1) takes the same products with the side's sign, so no
      // per-pair partial sums are needed
      cx<T> acc[NV][4];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[v][a] = czero<T>();
      const int nit = (pe - pb) * nb;
      // loads of iteration it + 1 issued before the products of iteration it
      auto load = [&](int it, cx<T> &u0, cx<T> &u1, cx<T> (&x)[NV][2]) {
        const int pair = pb + it / nb, n = it - (it / nb) * nb;
        const long long row = ((long long)pair * nb + n) * 2;
        u0 = __ldg(ur + row * nr + r);
        u1 = __ldg(ur + (row + 1) * nr + r);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const long long rv = row + v * rows1;
          x[v][0] = xr[rv * nr + r];
          x[v][1] = xr[(rv + 1) * nr + r];
        }
      };
      cx<T> u0, u1, xv[NV][2];
      if (nit > 0) load(0, u0, u1, xv);
      for (int it = 0; it < nit; ++it) {
        const cx<T> cu0 = u0, cu1 = u1;
        cx<T> cx_[NV][2];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          cx_[v][0] = xv[v][0];
          cx_[v][1] = xv[v][1];
        }
        if (it + 1 < nit) load(it + 1, u0, u1, xv);
        const int pair = pb + it / nb;
        const int side = pair / nk, k = pair - side * nk;
        const T w = wk[k], wt = side == 0 ? w : -w;
        const cx<T> b0 = cscale<T>(cu0, wt), b1 = cscale<T>(cu1, wt);   // magnetic weight
#pragma unroll
        for (int v = 0; v < NV; ++v) {  // every vector of the pass: no early exit
          const cx<T> x0 = cx_[v][0], x1 = cx_[v][1];
          const cx<T> p00 = cmulc<T>(b0, x0), p01 = cmulc<T>(b0, x1);
          const cx<T> p10 = cmulc<T>(b1, x0), p11 = cmulc<T>(b1, x1);
          const cx<T> c = cadd<T>(p00, p11);  // charge: w (U^+ x), i.e. +-(b^+ x)
          acc[v][0] = side == 0 ? cadd<T>(acc[v][0], c) : csub<T>(acc[v][0], c);
          acc[v][1] = cadd<T>(acc[v][1], cadd<T>(p01, p10));
          const cx<T> d = csub<T>(p10, p01);  // m_y: i (p10 - p01)
          acc[v][2] = cadd<T>(acc[v][2], mk<T>(-d.y, d.x));
          acc[v][3] = cadd<T>(acc[v][3], csub<T>(p00, p11));
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int a = 0; a < 4; ++a) rho[((long long)v * 4 + a) * nr + r] = acc[v][a];
    }
  } else {
    // FP64 (bound by the FP64 rate): products shared by the charge and magnetic parts,
    // the k weights applied once per (side, k) pair
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr;
         r += (long long)gridDim.x * blockDim.x) {
      cx<T> acc[NV][4];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[v][a] = czero<T>();
      for (int pair = pb; pair < pe; ++pair) {
        const int side = pair / nk, k = pair - side * nk;
        const T w = wk[k], wt = side == 0 ? w : -w;
        cx<T> a[NV][4];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int c = 0; c < 4; ++c) a[v][c] = czero<T>();
        for (int n = 0; n < nb; ++n) {
          const long long row = ((long long)pair * nb + n) * 2;
          const cx<T> u0 = __ldg(ur + row * nr + r), u1 = __ldg(ur + (row + 1) * nr + r);
#pragma unroll
          for (int v = 0; v < NV; ++v) {  // every vector of the pass: no early exit, so
            const long long rv = row + v * rows1;  // all loads of a band issue together
            const cx<T> x0 = xr[rv * nr + r], x1 = xr[(rv + 1) * nr + r];
            const cx<T> p00 = cmulc<T>(u0, x0), p01 = cmulc<T>(u0, x1);
            const cx<T> p10 = cmulc<T>(u1, x0), p11 = cmulc<T>(u1, x1);
            a[v][0] = cadd<T>(a[v][0], cadd<T>(p00, p11));
            a[v][1] = cadd<T>(a[v][1], cadd<T>(p01, p10));
            const cx<T> d = csub<T>(p10, p01);  // m_y: i (p10 - p01)
            a[v][2] = cadd<T>(a[v][2], mk<T>(-d.y, d.x));
            a[v][3] = cadd<T>(a[v][3], csub<T>(p00, p11));
          }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          acc[v][0] = cadd<T>(acc[v][0], cscale<T>(a[v][0], w));
#pragma unroll
          for (int c = 1; c < 4; ++c) acc[v][c] = cadd<T>(acc[v][c], cscale<T>(a[v][c], wt));
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int a = 0; a < 4; ++a) rho[((long long)v * 4 + a) * nr + r] = acc[v][a];
    }
  }
}

// rho[v][a][r] = sum_g part[g][v][a][r] in fixed order
template <class T>
__global__ void density_reduce_kernel(const cx<T> *__restrict__ part, cx<T> *__restrict__ rho,
                                      int ngroup, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cx<T> s = part[i];
    for (int g = 1; g < ngroup; ++g) s = cadd<T>(s, part[(long long)g * n + i]);
    rho[i] = s;
  }
}

constexpr int kDensityGroups = 8;

template <class T>
void density_passes(cudaStream_t st, const cx<T> *ur, const cx<T> *xr, const T *wk, cx<T> *rho,
                    cx<T> *part, int nk, int nb, long long nr, int nvec, int per, dim3 grid,
                    int ppg, int ng, long long rows1);

template <class T>
void launch_density(Context &ctx, const cx<T> *ur, const cx<T> *xr, const T *wk, cx<T> *rho,
                    cx<T> *part, int nk, int nb, long long nr, int nvec) {
  cudaStream_t st = ctx.stream;
  // (side, k) pairs split over kDensityGroups block rows for parallelism; up to 3
  // vectors per pass (register budget), each sharing the U(r) reads
  const long long rows1 = 4LL * nk * nb;
  const int npair = 2 * nk;
  const int ngroup = std::min(kDensityGroups, npair);
  const int ppg = (npair + ngroup - 1) / ngroup;
  const int ng = (npair + ppg - 1) / ppg;
  const dim3 grid(blocks_for(nr), ng);
  // vectors per pass (2 or 3, autotuned; 3 is the default): each pass reads U(r) once,
  // more vectors per pass raise the register count.  Each vector's sums run in the
  // same order whatever the grouping, so the choice changes no result.
  char key[128];
  snprintf(key, sizeof(key), "density/%s/nr=%lld/rows=%lld/nvec=%d",
           sizeof(T) == 4 ? "f32" : "f64", nr, rows1, nvec);
  ctx.tuner.pick(st, key, nvec > 1 ? std::vector<int>{2, 3} : std::vector<int>{3}, 3,
                 [&](int per) { density_passes<T>(st, ur, xr, wk, rho, part, nk, nb, nr, nvec,
                                                  per, grid, ppg, ng, rows1); });
}

template <class T>
void density_passes(cudaStream_t st, const cx<T> *ur, const cx<T> *xr, const T *wk, cx<T> *rho,
                    cx<T> *part, int nk, int nb, long long nr, int nvec, int per, dim3 grid,
                    int ppg, int ng, long long rows1) {
  for (int v0 = 0; v0 < nvec; v0 += per) {
    const int nv = std::min(per, nvec - v0);
    const cx<T> *xv = xr + (long long)v0 * rows1 * nr;
    cx<T> *pv = part + (long long)v0 * 4 * nr;
    if (nv == 1)
      density_kernel<T, 1><<<grid, kThreads, 0, st>>>(ur, xv, wk, pv, nk, nb, nr, ppg, nvec);
    else if (nv == 2)
      density_kernel<T, 2><<<grid, kThreads, 0, st>>>(ur, xv, wk, pv, nk, nb, nr, ppg, nvec);
    else
      density_kernel<T, 3><<<grid, kThreads, 0, st>>>(ur, xv, wk, pv, nk, nb, nr, ppg, nvec);
    TDLZ_LAUNCH_CHECK();
  }
  long long n = (long long)nvec * 4 * nr;
  density_reduce_kernel<T><<<blocks_for(n), kThreads, 0, st>>>(part, rho, ng, n);
  TDLZ_LAUNCH_CHECK();
}

// --------------------------------------------------------- Hartree + ALSDA
// v_a = delta_a0 vH + sum_b f_ab rho_b ; f packed 00,01,02,03,11,12,13,22,23,33
template <class T>
__global__ void potential_kernel(const cx<T> *__restrict__ rho, const cx<T> *__restrict__ vh,
                                 const T *__restrict__ f, cx<T> *__restrict__ v, long long nr,
                                 int use_h, int use_xc) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr;
       r += (long long)gridDim.x * blockDim.x) {
    cx<T> out[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
    if (use_xc) {
      cx<T> p[4];
      for (int a = 0; a < 4; ++a) p[a] = rho[a * nr + r];
      T fm[4][4];
      int q = 0;
      for (int a = 0; a < 4; ++a)
        for (int b = a; b < 4; ++b) {
          T val = f[q++ * nr + r];
          fm[a][b] = val;
          fm[b][a] = val;
        }
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          out[a].x += fm[a][b] * p[b].x;
          out[a].y += fm[a][b] * p[b].y;
        }
    }
    if (use_h) out[0] = cadd<T>(out[0], vh[r]);
    for (int a = 0; a < 4; ++a) v[a * nr + r] = out[a];
  }
}

// ------------------------------------------------------------------ GEMMs
// Split-K reduction GEMM: part[z][b][m][n] = sum_{k in split z} conj(A[bA][m][k]) B[b][n][k].
// 16 x 16 threads, each holding an R x R register tile (rows ty + 16 i, columns
// tx + 16 j), so one CTA covers a (16 R) x (16 R) output tile: per shared-memory
// load a thread does R complex multiply-adds.
constexpr int KC = 16;
template <class T, int R>
__global__ void __launch_bounds__(256)
    gemm_tn_kernel(const cx<T> *__restrict__ A, long long lda, long long sA, int amod,
                   const cx<T> *__restrict__ B, long long ldb, long long sB,
                   cx<T> *__restrict__ part, int M, int N, long long K, int batch, int nsplit) {
  constexpr int TT = 16 * R;
  __shared__ cx<T> As[TT][KC + 1];
  __shared__ cx<T> Bs[TT][KC + 1];
  int z = blockIdx.z;
  int b = z % batch;
  int sp = z / batch;
  int m0 = blockIdx.y * TT, n0 = blockIdx.x * TT;
  long long kchunk = (K + nsplit - 1) / nsplit;
  long long kb = sp * kchunk, ke = kb + kchunk < K ? kb + kchunk : K;
  const cx<T> *Ab = A + (long long)(b % amod) * sA;
  const cx<T> *Bb = B + (long long)b * sB;
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  cx<T> acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = czero<T>();
  for (long long k0 = kb; k0 < ke; k0 += KC) {
    for (int e = threadIdx.x; e < TT * KC; e += blockDim.x) {
      int rr = e / KC, kk = e % KC;
      long long kg = k0 + kk;
      cx<T> av = czero<T>(), bv = czero<T>();
      if (kg < ke) {
        if (m0 + rr < M) av = Ab[(long long)(m0 + rr) * lda + kg];
        if (n0 + rr < N) bv = Bb[(long long)(n0 + rr) * ldb + kg];
      }
      As[rr][kk] = av;
      Bs[rr][kk] = bv;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      cx<T> av[R], bv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) av[i] = As[ty + 16 * i][kk];
#pragma unroll
      for (int j = 0; j < R; ++j) bv[j] = Bs[tx + 16 * j][kk];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) cfmac<T>(acc[i][j], av[i], bv[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N)
        part[(((long long)sp * batch + b) * M + m) * N + n] = acc[i][j];
    }
}

// C[b*sC + m*ldcm + n*ldcn] = sum_z part[z][b][m][n] (fixed order)
template <class T>
__global__ void split_reduce_kernel(const cx<T> *__restrict__ part, cx<T> *__restrict__ C,
                                    int M, int N, int batch, int nsplit, long long sC,
                                    long long ldcm, long long ldcn) {
  long long total = (long long)batch * M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    cx<T> s = czero<T>();
    for (int z = 0; z < nsplit; ++z) s = cadd<T>(s, part[(long long)z * total + i]);
    long long b = i / ((long long)M * N);
    long long rem = i - b * M * N;
    long long m = rem / N, n = rem - m * N;
    C[b * sC + m * ldcm + n * ldcn] = s;
  }
}

// Out[b][row][col] = sgn_b (In[b][row][col] + alpha sum_k A(b,row,k) B[b % bmod][k][col])
constexpr int NN_ROWS = 16, NN_COLS = 128, NN_KMAX = 256;
// grid: x = row chunk (fastest, so the CTAs that share a B column tile run together
// and re-read it from L2), y = column chunk, z = batch; A chunk in dynamic smem.
// Each thread owns NC columns (tid + j NN_COLS, coalesced for every j), so every
// shared-memory load of A feeds NC complex multiply-adds.
template <class T, int NC>
__global__ void __launch_bounds__(NN_COLS)
    gemm_nn_kernel(const cx<T> *__restrict__ A, long long sA, long long sar, long long sak,
                   const cx<T> *__restrict__ B, long long ldb, long long sB, int bmod,
                   const cx<T> *In, cx<T> *Out, long long ldo, long long sO, int rows,
                   long long ncol, int K, T alpha, int neg_from, int neg_mod) {
  extern __shared__ unsigned char nn_smem[];
  cx<T> *As = reinterpret_cast<cx<T> *>(nn_smem);  // [NN_ROWS][K]
  int b = blockIdx.z;
  int r0 = blockIdx.x * NN_ROWS;
  const cx<T> *Ab = A + (long long)b * sA;
  for (int e = threadIdx.x; e < NN_ROWS * K; e += blockDim.x) {
    int rr = e / K, kk = e % K;
    As[e] = (r0 + rr < rows) ? Ab[(long long)(r0 + rr) * sar + (long long)kk * sak] : czero<T>();
  }
  __syncthreads();
  const long long col0 = (long long)blockIdx.y * NN_COLS * NC + threadIdx.x;
  if (col0 >= ncol) return;
  const cx<T> *Bb = B + (long long)(b % bmod) * sB;
  cx<T> acc[NC][NN_ROWS];
#pragma unroll
  for (int j = 0; j < NC; ++j)
#pragma unroll
    for (int r = 0; r < NN_ROWS; ++r) acc[j][r] = czero<T>();
  // B columns prefetched 4 entries at a time (independent loads in flight)
  constexpr int U = 4;
  for (int kk = 0; kk < K; kk += U) {
    cx<T> bv[U][NC];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const long long c = col0 + j * NN_COLS;
        bv[u][j] = (kk + u < K && c < ncol) ? __ldg(Bb + (long long)(kk + u) * ldb + c)
                                            : czero<T>();
      }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (kk + u >= K) break;
#pragma unroll
      for (int r = 0; r < NN_ROWS; ++r) {
        const cx<T> av = As[r * K + kk + u];
#pragma unroll
        for (int j = 0; j < NC; ++j) cfma<T>(acc[j][r], av, bv[u][j]);
      }
    }
  }
  T sg = (b % neg_mod) >= neg_from ? T(-1) : T(1);
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const long long col = col0 + j * NN_COLS;
    if (col >= ncol) break;
#pragma unroll
    for (int r = 0; r < NN_ROWS; ++r) {
      if (r0 + r >= rows) break;
      long long o = (long long)b * sO + (long long)(r0 + r) * ldo + col;
      cx<T> iv = In[o];
      Out[o] = mk<T>(sg * (iv.x + alpha * acc[j][r].x), sg * (iv.y + alpha * acc[j][r].y));
    }
  }
}

// dmix[b][(n,s)][i] = sum_{j,t} D[2i+s][2j+t] proj[b][j][(n,t)], over the nonzero
// entries of row 2i+s only (ELL form: D couples the projectors of one atom)
template <class T>
__global__ void dmix_kernel(const cx<T> *__restrict__ proj, const cx<T> *__restrict__ dval,
                            const int *__restrict__ dcol, int dw, cx<T> *__restrict__ dmix,
                            int nproj, int nb, int batch) {
  long long total = (long long)batch * nb * 2 * nproj;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % nproj);
    long long rest = e / nproj;
    int s = (int)(rest % 2);
    rest /= 2;
    int n = (int)(rest % nb);
    long long b = rest / nb;
    const cx<T> *pb = proj + b * (long long)nproj * 2 * nb;
    const long long row = (long long)(2 * i + s) * dw;
    cx<T> acc = czero<T>();
    for (int q = 0; q < dw; ++q) {
      const int c = __ldg(dcol + row + q);
      if (c < 0) break;
      cfma<T>(acc, dval[row + q], pb[(long long)(c >> 1) * 2 * nb + 2 * n + (c & 1)]);
    }
    dmix[e] = acc;
  }
}

template <class T>
void gemm_tn(Context &ctx, DevBuf &partbuf, const cx<T> *A, long long lda, long long sA, int amod,
             const cx<T> *B, long long ldb, long long sB, cx<T> *C, long long sC, long long ldcm,
             long long ldcn, int M, int N, long long K, int batch) {
  // register tile R (CTA tile 16 R) from the larger output dimension, at most 5 (80)
  const int R = std::max(1, std::min(5, (std::max(M, N) + 15) / 16));
  const int TT = 16 * R;
  const int tiles = ((M + TT - 1) / TT) * ((N + TT - 1) / TT);
  // enough CTAs to fill the GPU: split K so that batch * tiles * nsplit >= ~4 waves
  long long want = (4LL * 152 + (long long)batch * tiles - 1) / ((long long)batch * tiles);
  long long ns = std::min(want, (K + 255) / 256);
  int nsplit = (int)std::max(1LL, std::min(ns, 32LL));
  size_t need = (size_t)nsplit * batch * M * N * sizeof(cx<T>);
  TDLZ_REQUIRE(need <= partbuf.bytes, TDLZ_ERR_STATE, "split-K scratch too small");
  dim3 grid((N + TT - 1) / TT, (M + TT - 1) / TT, (unsigned)(batch * nsplit));
  cx<T> *pp = partbuf.template as<cx<T>>();
  switch (R) {
    case 1: gemm_tn_kernel<T, 1><<<grid, 256, 0, ctx.stream>>>(A, lda, sA, amod, B, ldb, sB, pp, M, N, K, batch, nsplit); break;
    case 2: gemm_tn_kernel<T, 2><<<grid, 256, 0, ctx.stream>>>(A, lda, sA, amod, B, ldb, sB, pp, M, N, K, batch, nsplit); break;
    case 3: gemm_tn_kernel<T, 3><<<grid, 256, 0, ctx.stream>>>(A, lda, sA, amod, B, ldb, sB, pp, M, N, K, batch, nsplit); break;
    case 4: gemm_tn_kernel<T, 4><<<grid, 256, 0, ctx.stream>>>(A, lda, sA, amod, B, ldb, sB, pp, M, N, K, batch, nsplit); break;
    default: gemm_tn_kernel<T, 5><<<grid, 256, 0, ctx.stream>>>(A, lda, sA, amod, B, ldb, sB, pp, M, N, K, batch, nsplit); break;
  }
  TDLZ_LAUNCH_CHECK();
  long long tot = (long long)batch * M * N;
  split_reduce_kernel<T><<<blocks_for(tot), kThreads, 0, ctx.stream>>>(
      partbuf.template as<cx<T>>(), C, M, N, batch, nsplit, sC, ldcm, ldcn);
  TDLZ_LAUNCH_CHECK();
}

template <class T>
void gemm_nn(Context &ctx, const cx<T> *A, long long sA, long long sar, long long sak,
             const cx<T> *B, long long ldb, long long sB, int bmod, const cx<T> *In, cx<T> *Out,
             long long ldo, long long sO, int rows, long long ncol, int K, T alpha, int batch,
             int neg_from, int neg_mod = 1 << 30) {
  TDLZ_REQUIRE(K <= NN_KMAX, TDLZ_ERR_ARG, "contraction length above 256 (nocc or nproj)");
  // two columns per thread in FP32, one in FP64 (register budget)
  constexpr int NC = sizeof(T) == 4 ? 2 : 1;
  dim3 grid((rows + NN_ROWS - 1) / NN_ROWS, (unsigned)((ncol + NN_COLS * NC - 1) / (NN_COLS * NC)),
            batch);
  size_t sm = (size_t)NN_ROWS * K * sizeof(cx<T>);
  TDLZ_CUDA_TRY(cudaFuncSetAttribute(gemm_nn_kernel<T, NC>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  gemm_nn_kernel<T, NC><<<grid, NN_COLS, sm, ctx.stream>>>(A, sA, sar, sak, B, ldb, sB, bmod, In,
                                                         Out, ldo, sO, rows, ncol, K, alpha,
                                                         neg_from, neg_mod);
  TDLZ_LAUNCH_CHECK();
}

// ------------------------------------------------- precision conversion
template <class S, class D>
__global__ void convert_kernel(const S *__restrict__ a, D *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (D)a[i];
}

template <class T>
void convert_buf(Context &ctx, const DevBuf &src, DevBuf &dst) {
  long long n = src.bytes / sizeof(double);
  dst.alloc(n * sizeof(T));
  convert_kernel<double, T><<<blocks_for(n), kThreads, 0, ctx.stream>>>(
      src.as<double>(), dst.as<T>(), n);
  TDLZ_LAUNCH_CHECK();
}

// ----------------------------------------------------- XC kernel table
// Spin-polarised Slater exchange e = -(3/4)(6/pi)^{1/3}(n_u^{4/3} + n_d^{4/3}),
// n_u/d = (n +- |m|)/2 floored at 1e-4, f = 0 for n < 1e-10; second
// derivatives w.r.t. (n, m) through |m| (Eqs. v_XC_q, b_XC_q).
__global__ void fxc_kernel(const double *__restrict__ n0, const double *__restrict__ m0,
                           double *__restrict__ f, long long nr) {
  const double c6 = cbrt(6.0 / 3.14159265358979323846);
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr;
       r += (long long)gridDim.x * blockDim.x) {
    double fm[4][4] = {{0}};
    double n = n0[r];
    if (n >= 1e-10) {
      double mx = m0[r], my = m0[nr + r], mz = m0[2 * nr + r];
      double ma = sqrt(mx * mx + my * my + mz * mz);
      double nu = fmax(0.5 * (n + ma), 1e-4), nd = fmax(0.5 * (n - ma), 1e-4);
      double fu = -(c6 / 3.0) / cbrt(nu * nu), fd = -(c6 / 3.0) / cbrt(nd * nd);
      double h[3], tr;
      if (ma < 1e-12 * n) {
        h[0] = 0.0;
        h[1] = 0.0;
        h[2] = 1.0;
        double nh = fmax(0.5 * n, 1e-4);
        tr = 0.5 * (-(c6 / 3.0) / cbrt(nh * nh));
      } else {
        h[0] = mx / ma;
        h[1] = my / ma;
        h[2] = mz / ma;
        double vu = -cbrt(6.0 * nu / 3.14159265358979323846);
        double vd = -cbrt(6.0 * nd / 3.14159265358979323846);
        tr = (vu - vd) / (2.0 * ma);
      }
      double sp = 0.25 * (fu + fd), sm = 0.25 * (fu - fd);
      fm[0][0] = sp;
      for (int i = 0; i < 3; ++i) {
        fm[0][i + 1] = fm[i + 1][0] = sm * h[i];
        for (int j = 0; j < 3; ++j)
          fm[i + 1][j + 1] = sp * h[i] * h[j] + tr * ((i == j ? 1.0 : 0.0) - h[i] * h[j]);
      }
    }
    int q = 0;
    for (int a = 0; a < 4; ++a)
      for (int b = a; b < 4; ++b) f[(long long)(q++) * nr + r] = fm[a][b];
  }
}

// ---------------------------------------------------------- start vectors
// v[b][n][s][g] = sum_t sigma^mu[s][t] c_k[b][n][t][map[g]]  (G of the k+q sphere
// found in the k sphere; 0 otherwise), mu = 0, 1, 2: the Pauli matrices, 3: sigma^0
// (the charge).  ysign multiplies the Y side of the spin components; the charge
// density has the opposite Y-side sign (Eqs. charge_dens_resp_q, spin_dens_resp_q),
// so the charge's Y side is multiplied by -ysign.
template <class T>
__global__ void sigma_u_kernel(const cx<T> *__restrict__ ck, const int *__restrict__ map, int mu,
                               cx<T> *__restrict__ out, int nk, int nb, int npwx, T ysign) {
  long long total = 2LL * nk * nb * npwx;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int g = (int)(e % npwx);
    long long band = e / npwx;  // (side, k, n)
    int k = (int)((band / nb) % nk);
    int side = (int)(band / ((long long)nk * nb));
    int mg = map[(long long)k * npwx + g];
    cx<T> c0 = czero<T>(), c1 = czero<T>();
    if (mg >= 0) {
      c0 = ck[(band * 2) * npwx + mg];
      c1 = ck[(band * 2 + 1) * npwx + mg];
    }
    cx<T> o0, o1;
    if (mu == 0) {  // sigma_x
      o0 = c1;
      o1 = c0;
    } else if (mu == 1) {  // sigma_y: (-i c1, i c0)
      o0 = mk<T>(c1.y, -c1.x);
      o1 = mk<T>(-c0.y, c0.x);
    } else if (mu == 2) {  // sigma_z
      o0 = c0;
      o1 = mk<T>(-c1.x, -c1.y);
    } else {  // sigma^0
      o0 = c0;
      o1 = c1;
    }
    T sg = side == 1 ? (mu == 3 ? -ysign : ysign) : T(1);
    out[(band * 2) * npwx + g] = cscale<T>(o0, sg);
    out[(band * 2 + 1) * npwx + g] = cscale<T>(o1, sg);
  }
}


// Bytes of the staged pipeline's buffers for one stacked vector: the real-space grids,
// the plane buffer and the stick buffer of every row, complex elements of c bytes.
double staged_vector_bytes(const QSlot &s, size_t c) {
  const bool fused = c == sizeof(float2) ? s.yx32 : s.yx64;
  const double per_row = (double)s.nr +
                         (fused ? 0.0 : (double)s.nplane_max * s.fft[1] * s.fft[2]) +
                         (double)s.nstick_max * s.fft[2];
  return (double)s.rows() * per_row * (double)c;
}

// Stacked vectors the staged pipeline's buffers are sized for, decided when they are
// allocated: all nvec where they take at most 70% of the memory then free (and at most
// half the device), else the largest count that does (at least one).  The count
// changes no result (every vector's stages are independent of the others'), only how
// often the orbitals U(r) are read per pass; q-slots allocated later see what is left.
int staged_cap(const QSlot &s, size_t c, int nvec) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    (void)cudaGetLastError();
    free_b = 0;
  }
  const double budget = std::min(0.5 * (double)s.dev_total, 0.7 * (double)free_b);
  int n = (int)std::floor(budget / staged_vector_bytes(s, c));
  n = std::max(1, std::min(n, nvec));
  if (s.staged_sub_env > 0) n = std::min(n, s.staged_sub_env);
  return n;
}

// Vectors per sub-batch of a pass over nvec stacked vectors: the sub-batches balanced
// under the workspace's capacity ns (never above it).
int staged_sub(int ns, int nvec) {
  const int n = std::max(1, std::min(ns, nvec));
  const int nbatch = (nvec + n - 1) / n;
  return (nvec + nbatch - 1) / nbatch;
}

template <class T>
void alloc_workspace(QSlot &s, int nvec) {
  Workspace<T> &w = slot_ws<T>(s);
  if (w.ready && w.nvec_cap >= nvec) return;
  const size_t c = sizeof(cx<T>), nv = (size_t)nvec;
  w.ready = false;
  const bool planes = sizeof(T) == 4 ? s.planes32 : s.planes64;
  // fused plane stages: no real-space grids or plane buffer in HBM, only the stick
  // buffer, per-chunk partial densities and the potential planes
  if (planes) {
    w.xr.reset();
    w.i2.reset();
    size_t pmax = 0;
    for (int m = 1; m <= nvec; ++m)
      pmax = std::max(pmax, (size_t)planes_density_chunks(s, m, c) * m);
    w.rhopart.alloc(pmax * 4 * (size_t)s.nr * c);
    w.vpot.alloc(nv * s.fft[2] * 6 * (size_t)planes_nnp(s) * c);
    w.i1.alloc(nv * s.rows() * s.nstick_max * s.fft[2] * c);
    w.rho.alloc(nv * 4 * (size_t)s.nr * c);
    w.hgrid.alloc(nv * (size_t)s.nr * c);
  } else {
    // the real-space stages run over sub-batches of at most ns stacked vectors
    // release the old grids first so that the free memory the capacity is sized by
    // counts them
    w.xr.reset();
    w.i2.reset();
    w.i1.reset();
    const size_t ns = (size_t)staged_cap(s, c, nvec);
    w.ns_cap = (int)ns;
    const bool fused = sizeof(T) == 4 ? s.yx32 : s.yx64;
    w.xr.alloc(ns * s.rows() * s.nr * c);
    if (fused)
      w.i2.reset();  // the fused Y + X passes keep the planes on chip
    else
      w.i2.alloc(ns * s.rows() * s.nplane_max * s.fft[1] * s.fft[2] * c);
    w.i1.alloc(ns * s.rows() * s.nstick_max * s.fft[2] * c);
    w.rhopart.alloc((size_t)kDensityGroups * ns * 4 * (size_t)s.nr * c);
    w.vpot.alloc(ns * 4 * (size_t)s.nr * c);
    w.rho.alloc(ns * 4 * (size_t)s.nr * c);
    w.hgrid.alloc(ns * (size_t)s.nr * c);
  }
  w.h.alloc(nv * (size_t)s.br_elems() * c);
  w.xin.reset();  // the adjoint's input copy: allocated on its first use
  size_t batch = nv * 2 * s.nk;
  w.proj.alloc(batch * s.nproj * 2 * s.nb * c + c);
  w.dmix.alloc(batch * s.nproj * 2 * s.nb * c + c);
  w.ovl.alloc(batch * s.nb * s.nb * c);
  size_t p1 = (size_t)32 * batch * std::max(s.nproj, 1) * 2 * s.nb;
  size_t p2 = (size_t)32 * batch * s.nb * s.nb;
  w.part.alloc(std::max(p1, p2) * c);
  w.nvec_cap = nvec;
  w.ready = true;
}

// a[i] *= fac[i % n] (the Hartree factor of one grid applied to stacked grids)
template <class T>
__global__ void scale_periodic_kernel(cx<T> *__restrict__ a, const T *__restrict__ fac,
                                      long long n, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    a[i] = cscale<T>(a[i], fac[i % n]);
}

// b[v][i] = a[v][stride][i]  (component 0 of each vector's 4-component density)
template <class T>
__global__ void gather_component_kernel(const cx<T> *__restrict__ a, cx<T> *__restrict__ b,
                                        long long n, long long stride, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long v = i / n;
    b[i] = a[v * stride + (i - v * n)];
  }
}

}  // namespace

// ===================================================================== load
// f(i) for i in [0, n) on up to 16 host threads (interleaved indices); f must not throw.
template <class F>
void host_parallel_for(long long n, F &&f) {
  const long long nt =
      std::min<long long>(n, std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
  if (nt <= 1) {
    for (long long i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  for (long long t = 0; t < nt; ++t)
    th.emplace_back([&f, t, nt, n] {
      for (long long i = t; i < n; i += nt) f(i);
    });
  for (auto &x : th) x.join();
}

void load_slot(Context &ctx, QSlot &s, const tdlz_ground_state *gs) {
  NvtxRange range("tdlz/load_ground_state");
  // ---- validation (host; nothing launched on failure)
  TDLZ_REQUIRE(gs != nullptr, TDLZ_ERR_ARG, "ground state is NULL");
  TDLZ_REQUIRE(gs->nk >= 1 && gs->nocc >= 1 && gs->npwx >= 1 && gs->nproj >= 0, TDLZ_ERR_ARG,
               "nk, nocc, npwx must be >= 1 and nproj >= 0");
  TDLZ_REQUIRE(gs->nocc <= 256 && gs->nproj <= 256, TDLZ_ERR_ARG, "nocc and nproj must be <= 256");
  for (int d = 0; d < 3; ++d)
    TDLZ_REQUIRE(fft_length_supported(gs->fft[d]), TDLZ_ERR_ARG,
                 "FFT lengths must be products of 2, 3, 5 and <= 512");
  double qn = std::sqrt(gs->q[0] * gs->q[0] + gs->q[1] * gs->q[1] + gs->q[2] * gs->q[2]);
  TDLZ_REQUIRE(qn > 1e-8, TDLZ_ERR_ARG, "|q| must exceed 1e-8 (q = 0 is a separate limit)");
  TDLZ_REQUIRE(gs->ecutwfc > 0, TDLZ_ERR_ARG, "ecutwfc must be positive");
  const char *ptr_names[] = {"kpts", "wk", "npw_k", "npw_kq", "miller_k", "miller_kq", "evals",
                             "coeff_k", "coeff_kq", "vloc", "bfield", "n0", "m0", "dnl"};
  const void *ptrs[] = {gs->kpts, gs->wk, gs->npw_k, gs->npw_kq, gs->miller_k, gs->miller_kq,
                        gs->evals, gs->coeff_k, gs->coeff_kq, gs->vloc, gs->bfield, gs->n0,
                        gs->m0, gs->dnl};
  for (int i = 0; i < 14; ++i)
    TDLZ_REQUIRE(ptrs[i] != nullptr || (i == 13 && gs->nproj == 0), TDLZ_ERR_ARG,
                 std::string("NULL array: ") + ptr_names[i]);
  TDLZ_REQUIRE(gs->nproj == 0 || gs->beta_kq != nullptr, TDLZ_ERR_ARG, "NULL array: beta_kq");
  const int nk = gs->nk, nb = gs->nocc, npwx = gs->npwx, np_ = gs->nproj;
  const long long nr = (long long)gs->fft[0] * gs->fft[1] * gs->fft[2];
  for (int k = 0; k < nk; ++k) {
    TDLZ_REQUIRE(gs->npw_k[k] >= 1 && gs->npw_k[k] <= npwx && gs->npw_kq[k] >= 1 &&
                     gs->npw_kq[k] <= npwx,
                 TDLZ_ERR_ARG, "npw_k / npw_kq out of range [1, npwx]");
    TDLZ_REQUIRE(std::isfinite(gs->wk[k]) && gs->wk[k] > 0, TDLZ_ERR_ARG, "k weights must be > 0");
  }
  auto finite_all = [](const double *p, long long n) {
    // chunks of 1 M values checked on the host threads
    const long long chunk = 1 << 20, nc = (n + chunk - 1) / chunk;
    std::vector<char> ok((size_t)nc, 1);
    host_parallel_for(nc, [&](long long c) {
      const long long e = std::min(n, (c + 1) * chunk);
      for (long long i = c * chunk; i < e; ++i)
        if (!std::isfinite(p[i])) {
          ok[(size_t)c] = 0;
          return;
        }
    });
    for (char v : ok)
      if (!v) return false;
    return true;
  };
  long long brd = 2LL * nk * nb * 2 * npwx * 2;
  TDLZ_REQUIRE(finite_all(gs->coeff_k, brd) && finite_all(gs->coeff_kq, brd) &&
                   finite_all(gs->evals, 2LL * nk * nb) && finite_all(gs->vloc, nr) &&
                   finite_all(gs->bfield, 3 * nr) && finite_all(gs->n0, nr) &&
                   finite_all(gs->m0, 3 * nr) && finite_all(gs->kpts, 3LL * nk),
               TDLZ_ERR_ARG, "non-finite value in the ground state");
  if (np_ > 0) {
    TDLZ_REQUIRE(finite_all(gs->dnl, 4LL * np_ * np_ * 2) &&
                     finite_all(gs->beta_kq, (long long)nk * np_ * npwx * 2),
                 TDLZ_ERR_ARG, "non-finite projector data");
    int nd = 2 * np_;
    double dmax = 0, herr = 0;
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j) {
        const double *a = gs->dnl + 2 * ((long long)i * nd + j);
        const double *b = gs->dnl + 2 * ((long long)j * nd + i);
        dmax = std::max(dmax, std::hypot(a[0], a[1]));
        herr = std::max(herr, std::hypot(a[0] - b[0], a[1] + b[1]));
      }
    TDLZ_REQUIRE(herr <= 1e-12 * std::max(dmax, 1e-300), TDLZ_ERR_ARG,
                 "dnl is not Hermitian");
  }
  // grid indices + sphere checks
  std::vector<int> idx_k((size_t)nk * npwx, -1), idx_kq((size_t)nk * npwx, -1),
      map((size_t)nk * npwx, -1);
  auto gidx = [&](const int *m, int &out) {
    long long id = 0;
    for (int d = 0; d < 3; ++d) {
      int n = gs->fft[d];
      if (m[d] < -(n / 2) || m[d] > (n - 1) / 2) return false;
      id = id * n + ((m[d] % n) + n) % n;
    }
    out = (int)id;
    return true;
  };
  for (int k = 0; k < nk; ++k) {
    std::unordered_map<int, int> where;
    for (int g = 0; g < gs->npw_k[k]; ++g) {
      int id;
      TDLZ_REQUIRE(gidx(gs->miller_k + 3 * ((long long)k * npwx + g), id), TDLZ_ERR_ARG,
                   "k sphere does not fit the FFT box");
      TDLZ_REQUIRE(where.emplace(id, g).second, TDLZ_ERR_ARG, "duplicate Miller index (k)");
      idx_k[(size_t)k * npwx + g] = id;
    }
    std::unordered_map<int, int> seen;
    for (int g = 0; g < gs->npw_kq[k]; ++g) {
      int id;
      TDLZ_REQUIRE(gidx(gs->miller_kq + 3 * ((long long)k * npwx + g), id), TDLZ_ERR_ARG,
                   "k+q sphere does not fit the FFT box");
      TDLZ_REQUIRE(seen.emplace(id, g).second, TDLZ_ERR_ARG, "duplicate Miller index (k+q)");
      idx_kq[(size_t)k * npwx + g] = id;
      auto it = where.find(id);
      map[(size_t)k * npwx + g] = it == where.end() ? -1 : it->second;
    }
  }
  // ---- internal plane-wave order of the k+q spheres: ascending grid index (stick by
  // stick, j3 ascending inside a stick), so that the Z passes read and write contiguous
  // runs of each stick; perm[k][i] = caller index of internal index i
  std::vector<int> perm((size_t)nk * npwx, -1), iperm((size_t)nk * npwx, -1);
  for (int k = 0; k < nk; ++k) {
    const int npw = gs->npw_kq[k];
    int *pk = perm.data() + (size_t)k * npwx;
    const int *id = idx_kq.data() + (size_t)k * npwx;
    for (int i = 0; i < npw; ++i) pk[i] = i;
    std::sort(pk, pk + npw, [id](int a, int b) { return id[a] < id[b]; });  // ids distinct
    for (int i = 0; i < npw; ++i) iperm[(size_t)k * npwx + pk[i]] = i;
  }
  // [outer][nk][rows][npwx] complex arrays in the internal order (zero padding)
  auto to_internal = [&](const double *src, long long outer, long long rws) {
    std::vector<double> dst((size_t)(outer * nk * rws * npwx * 2), 0.0);
    host_parallel_for(outer * nk, [&](long long ok) {
      const int k = (int)(ok % nk);
      const int *pk = perm.data() + (size_t)k * npwx;
      for (long long r = 0; r < rws; ++r) {
        const size_t base = (size_t)((ok * rws + r) * npwx) * 2;
        for (int i = 0; i < gs->npw_kq[k]; ++i) {
          dst[base + 2 * i] = src[base + 2 * (size_t)pk[i]];
          dst[base + 2 * i + 1] = src[base + 2 * (size_t)pk[i] + 1];
        }
      }
    });
    return dst;
  };
  {
    std::vector<int> ip((size_t)nk * npwx, -1), mp((size_t)nk * npwx, -1);
    for (int k = 0; k < nk; ++k)
      for (int i = 0; i < gs->npw_kq[k]; ++i) {
        const size_t g = (size_t)k * npwx + perm[(size_t)k * npwx + i];
        ip[(size_t)k * npwx + i] = idx_kq[g];
        mp[(size_t)k * npwx + i] = map[g];
      }
    idx_kq.swap(ip);
    map.swap(mp);
  }
  const std::vector<double> ukq_int = to_internal(gs->coeff_kq, 2, 2LL * nb);
  const std::vector<double> beta_int =
      np_ > 0 ? to_internal(gs->beta_kq, 1, np_) : std::vector<double>();
  // ---- host-side geometry
  s.nk = nk;
  s.nb = nb;
  s.npwx = npwx;
  s.nproj = np_;
  s.kernel_mask = gs->kernel_mask;
  for (int d = 0; d < 3; ++d) s.fft[d] = gs->fft[d];
  s.nr = nr;
  for (int d = 0; d < 3; ++d) s.q[d] = gs->q[d];
  const double *A = gs->lattice;
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
  TDLZ_REQUIRE(std::fabs(det) > 1e-12, TDLZ_ERR_ARG, "singular lattice");
  s.omega = std::fabs(det);
  // reciprocal rows b_j = 2 pi (A^{-1})^T  rows
  double inv[9];
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = -(A[1] * A[8] - A[2] * A[7]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = -(A[3] * A[8] - A[5] * A[6]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = -(A[0] * A[5] - A[2] * A[3]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = -(A[0] * A[7] - A[1] * A[6]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  double bv[3][3];  // bv[j][c] = 2 pi inv[c][j]
  for (int j = 0; j < 3; ++j)
    for (int c = 0; c < 3; ++c) bv[j][c] = 2.0 * 3.14159265358979323846 * inv[c * 3 + j];
  s.npw_k.assign(gs->npw_k, gs->npw_k + nk);
  s.npw_kq.assign(gs->npw_kq, gs->npw_kq + nk);
  s.wk.assign(gs->wk, gs->wk + nk);
  std::vector<double> kin((size_t)nk * npwx, 0.0);
  for (int k = 0; k < nk; ++k)
    for (int i = 0; i < gs->npw_kq[k]; ++i) {
      const int *m = gs->miller_kq + 3 * ((long long)k * npwx + perm[(size_t)k * npwx + i]);
      double v[3];
      for (int c = 0; c < 3; ++c)
        v[c] = gs->kpts[3 * k + c] + gs->q[c] + m[0] * bv[0][c] + m[1] * bv[1][c] + m[2] * bv[2][c];
      kin[(size_t)k * npwx + i] = 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }
  // Hartree factor on the grid: 4 pi/|q+G|^2 / Nr where |q+G|^2/2 <= 4 ecut
  std::vector<double> vh(nr, 0.0);
  {
    long long id = 0;
    for (int i1 = 0; i1 < gs->fft[0]; ++i1)
      for (int i2 = 0; i2 < gs->fft[1]; ++i2)
        for (int i3 = 0; i3 < gs->fft[2]; ++i3, ++id) {
          int m[3] = {i1, i2, i3};
          for (int d = 0; d < 3; ++d)
            if (m[d] >= (gs->fft[d] + 1) / 2) m[d] -= gs->fft[d];
          double v[3];
          for (int c = 0; c < 3; ++c)
            v[c] = gs->q[c] + m[0] * bv[0][c] + m[1] * bv[1][c] + m[2] * bv[2][c];
          double g2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
          if (0.5 * g2 <= 4.0 * gs->ecutwfc) vh[id] = 4.0 * 3.14159265358979323846 / g2 / nr;
        }
  }
  // ---- device upload (FP64 master copies)
  cudaStream_t st = ctx.stream;
  auto up = [&](DevBuf &b, const void *src, size_t bytes) {
    b.alloc(bytes);
    TDLZ_CUDA_TRY(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st));
  };
  s.plan.init(gs->fft);
  build_stick_tables(s, idx_kq);
  // Real-space stages, per precision: the staged pipeline (real-space grids of the stacked
  // vectors in HBM, in sub-batches that take at most a tenth of the device) where one
  // vector's buffers take at most 30% of the device memory; otherwise the fused plane
  // stages, whose workspace is the stick buffer.  Where both fit, the staged pipeline is
  // the faster (its grid traffic costs less HBM time than the plane stages' extra line
  // transforms cost issue slots).  TDLZ_PLANES=1 forces the plane stages where the grid
  // allows them, TDLZ_PLANES=0 the staged pipeline.
  {
    size_t free_b = 0, total_b = 0;
    TDLZ_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    s.dev_total = total_b;
    const char *sub_env = std::getenv("TDLZ_STAGED_SUB");
    s.staged_sub_env = sub_env ? std::max(0, std::atoi(sub_env)) : 0;
    const char *yx_env = std::getenv("TDLZ_YX_FUSED");
    const bool yx_on = !(yx_env && yx_env[0] == '0');
    s.yx32 = yx_on && yx_fused_supported<float>(s);
    s.yx64 = yx_on && yx_fused_supported<double>(s);
    const char *pl_env = std::getenv("TDLZ_PLANES");
    auto want_planes = [&](size_t c) {
      bool want = staged_vector_bytes(s, c) > 0.3 * (double)total_b;
      if (pl_env && pl_env[0] == '0') want = false;
      if (pl_env && pl_env[0] == '1') want = true;
      return want;
    };
    s.planes32 = want_planes(sizeof(float2)) && planes_supported<float>(s);
    s.planes64 = want_planes(sizeof(double2)) && planes_supported<double>(s);
  }
  // TDLZ_TC=0 keeps the V_NL / P_c reductions and updates on the CUDA-core GEMMs (A/B timing)
  const char *tc_env = std::getenv("TDLZ_TC");
  s.tensor_gemm = !(tc_env && tc_env[0] == '0');
  // TDLZ_TC_IMG=0 keeps the updates on the register-staged GEMM (no operand images)
  const char *img_env = std::getenv("TDLZ_TC_IMG");
  s.tc_images = !(img_env && img_env[0] == '0');
  up(s.perm, perm.data(), perm.size() * sizeof(int));
  up(s.iperm, iperm.data(), iperm.size() * sizeof(int));
  up(s.idx_k, idx_k.data(), idx_k.size() * sizeof(int));
  up(s.idx_kq, idx_kq.data(), idx_kq.size() * sizeof(int));
  up(s.map_kq_k, map.data(), map.size() * sizeof(int));
  up(s.npwkq_d, gs->npw_kq, nk * sizeof(int));
  SlotData<double> &d = s.d64;
  size_t brb = (size_t)s.br_elems() * sizeof(double2);
  up(d.ukq, ukq_int.data(), brb);
  up(s.coeff_k, gs->coeff_k, brb);
  // the occupied states at k and k+q of each side must be orthonormal (U^+ U = 1): the
  // conduction projector P_c = 1 - sum |U><U| and the pseudo-Hermiticity of L rest on it
  {
    const int batch = 2 * nk;
    const long long bstride = (long long)nb * 2 * npwx;
    DevBuf gram, gpart;
    gram.alloc((size_t)batch * nb * nb * sizeof(double2));
    gpart.alloc((size_t)32 * batch * nb * nb * sizeof(double2));
    std::vector<double> g((size_t)batch * nb * nb * 2);
    double err = 0.0;
    for (const DevBuf *u : {&d.ukq, &s.coeff_k}) {
      gemm_tn<double>(ctx, gpart, u->as<double2>(), 2LL * npwx, bstride, batch,
                      u->as<double2>(), 2LL * npwx, bstride, gram.as<double2>(),
                      (long long)nb * nb, nb, 1, nb, nb, 2LL * npwx, batch);
      TDLZ_CUDA_TRY(cudaMemcpyAsync(g.data(), gram.p, g.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
      TDLZ_CUDA_TRY(cudaStreamSynchronize(st));
      for (int b = 0; b < batch; ++b)
        for (int m = 0; m < nb; ++m)
          for (int n = 0; n < nb; ++n) {
            const double *e = g.data() + 2 * (((size_t)b * nb + m) * nb + n);
            err = std::max(err, std::hypot(e[0] - (m == n ? 1.0 : 0.0), e[1]));
          }
    }
    TDLZ_REQUIRE(err <= 1e-6, TDLZ_ERR_ARG,
                 "occupied states are not orthonormal (max |U^+U - 1| = " + std::to_string(err) +
                     " > 1e-6)");
  }
  if (np_ > 0) {
    up(d.beta, beta_int.data(), (size_t)nk * np_ * npwx * sizeof(double2));
    up(d.dnl, gs->dnl, (size_t)4 * np_ * np_ * sizeof(double2));
    // D is block diagonal over the atoms: keep each row's nonzero entries (ELL form)
    const int nd = 2 * np_;
    int w = 1;
    for (int r = 0; r < nd; ++r) {
      int cnt = 0;
      for (int c = 0; c < nd; ++c) {
        const double *v = gs->dnl + 2 * ((long long)r * nd + c);
        cnt += (v[0] != 0.0 || v[1] != 0.0);
      }
      w = std::max(w, cnt);
    }
    std::vector<int> col((size_t)nd * w, -1);
    std::vector<double> val((size_t)2 * nd * w, 0.0);
    for (int r = 0; r < nd; ++r) {
      int cnt = 0;
      for (int c = 0; c < nd; ++c) {
        const double *v = gs->dnl + 2 * ((long long)r * nd + c);
        if (v[0] == 0.0 && v[1] == 0.0) continue;
        col[(size_t)r * w + cnt] = c;
        val[2 * ((size_t)r * w + cnt)] = v[0];
        val[2 * ((size_t)r * w + cnt) + 1] = v[1];
        ++cnt;
      }
    }
    s.dnl_w = w;
    up(s.dnl_col, col.data(), col.size() * sizeof(int));
    up(d.dnl_val, val.data(), val.size() * sizeof(double));
  }
  up(d.kin, kin.data(), kin.size() * sizeof(double));
  up(d.evals, gs->evals, (size_t)2 * nk * nb * sizeof(double));
  up(d.vloc, gs->vloc, nr * sizeof(double));
  up(d.bfield, gs->bfield, 3 * nr * sizeof(double));
  up(d.vhfac, vh.data(), nr * sizeof(double));
  up(d.wk, gs->wk, nk * sizeof(double));
  DevBuf n0d, m0d;
  up(n0d, gs->n0, nr * sizeof(double));
  up(m0d, gs->m0, 3 * nr * sizeof(double));
  d.fxc.alloc(10 * nr * sizeof(double));
  fxc_kernel<<<blocks_for(nr), kThreads, 0, st>>>(n0d.as<double>(), m0d.as<double>(),
                                                  d.fxc.as<double>(), nr);
  TDLZ_LAUNCH_CHECK();
  // real-space occupied orbitals U(r) = Omega^{-1/2} sum_G c exp(iG.r)
  d.ur.alloc((size_t)s.rows() * nr * sizeof(double2));
  TDLZ_CUDA_TRY(cudaMemsetAsync(d.ur.p, 0, d.ur.bytes, st));
  scatter_rows_kernel<double><<<row_grid(s.rows(), npwx), kThreads, 0, st>>>(
      s.coeff_k.as<double2>(), d.ur.as<double2>(), s.idx_k.as<int>(), nk, nb, npwx, nr,
      1.0 / std::sqrt(s.omega), s.rows());
  TDLZ_LAUNCH_CHECK();
  fft3d<double>(s.plan, d.ur.as<double2>(), s.rows(), +1, st);
  // plane stages read U(r) as z-major slabs; the FP32 data of either layout are built
  // later from the slabs, so the grid-order copy goes
  if (s.planes64) {
    planes_build_u<double>(ctx, s, d.ur.as<double2>(), d.us);
    TDLZ_CUDA_TRY(cudaStreamSynchronize(st));
    d.ur.reset();
  }
  // u^lambda = (sigma^lambda U, t sigma^lambda T U) on the k+q sphere (unprojected):
  // t = -1 for the spin components x, y, z, +1 for the charge (lambda = 3)
  d.uvec.alloc(4 * brb);
  for (int l = 0; l < 4; ++l) {
    sigma_u_kernel<double><<<blocks_for(2LL * nk * nb * npwx), kThreads, 0, st>>>(
        s.coeff_k.as<double2>(), s.map_kq_k.as<int>(), l, d.uvec.as<double2>() + l * s.br_elems(),
        nk, nb, npwx, -1.0);
    TDLZ_LAUNCH_CHECK();
  }
  d.ready = true;
  // TDLZ_MIXED_ONLY=1: build the FP32 data now and release the FP64 real-space orbitals
  // (the largest FP64 array), for runs of many q-slots in mixed precision
  const char *mo = std::getenv("TDLZ_MIXED_ONLY");
  if (mo && mo[0] == '1') {
    ensure_precision<float>(ctx, s);
    TDLZ_CUDA_TRY(cudaStreamSynchronize(st));
    d.us.reset();
    d.ur.reset();
    d.uvec.reset();  // the chains' left vectors are read in FP32 only
    s.mixed_only = true;
  }
  TDLZ_CUDA_TRY(cudaStreamSynchronize(st));
}

template <class T>
void ensure_precision(Context &ctx, QSlot &s) {
  if constexpr (sizeof(T) == 4) {
    SlotData<float> &f = s.d32;
    if (!f.ready) {
      SlotData<double> &d = s.d64;
      convert_buf<float>(ctx, d.ukq, f.ukq);
      if (s.planes32) {
        if (d.us.p)
          convert_buf<float>(ctx, d.us, f.us);  // same slab layout
        else
          planes_build_u<float>(ctx, s, d.ur.as<double2>(), f.us);
      } else if (d.ur.p) {
        convert_buf<float>(ctx, d.ur, f.ur);
      } else {
        planes_grid_from_slabs<float>(ctx, s, d.us.as<double2>(), f.ur);
      }
      if (s.nproj > 0) {
        convert_buf<float>(ctx, d.beta, f.beta);
        convert_buf<float>(ctx, d.dnl, f.dnl);
        convert_buf<float>(ctx, d.dnl_val, f.dnl_val);
      }
      convert_buf<float>(ctx, d.kin, f.kin);
      convert_buf<float>(ctx, d.evals, f.evals);
      convert_buf<float>(ctx, d.vloc, f.vloc);
      convert_buf<float>(ctx, d.bfield, f.bfield);
      convert_buf<float>(ctx, d.fxc, f.fxc);
      convert_buf<float>(ctx, d.vhfac, f.vhfac);
      convert_buf<float>(ctx, d.wk, f.wk);
      convert_buf<float>(ctx, d.uvec, f.uvec);
      if (s.tensor_gemm && s.tc_images) {
        const long long bstride = (long long)s.nb * 2 * s.npwx;
        tc_image_build(ctx, f.ukq_img, f.ukq.as<float2>(), 2LL * s.npwx, bstride, 2 * s.nk,
                       s.nb, 2LL * s.npwx);
        if (s.nproj > 0)
          tc_image_build(ctx, f.beta_img, f.beta.as<float2>(), s.npwx,
                         (long long)s.nproj * s.npwx, s.nk, s.nproj, s.npwx);
      }
      f.ready = true;
    }
  }
  alloc_workspace<T>(s, std::max(1, slot_ws<T>(s).nvec_cap));
}

// ==================================================================== apply
template <class T>
void apply_liouvillian(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *y, int nvec,
                       unsigned adj_mask) {
  TDLZ_REQUIRE(nvec >= 1 && nvec <= 32, TDLZ_ERR_ARG, "nvec must be in [1, 32]");
  TDLZ_REQUIRE(sizeof(T) == 4 || !s.mixed_only, TDLZ_ERR_STATE,
               "q-slot loaded for mixed precision only (TDLZ_MIXED_ONLY=1): no FP64 application");
  ensure_precision<T>(ctx, s);
  alloc_workspace<T>(s, nvec);
  SlotData<T> &d = slot_data<T>(s);
  Workspace<T> &w = slot_ws<T>(s);
  cudaStream_t st = ctx.stream;
  Profiler &pf = ctx.prof;
  const int nk = s.nk, nb = s.nb, npwx = s.npwx, np_ = s.nproj;
  const long long nr = s.nr, rows = s.rows() * nvec, nbs = rows / 2, br = s.br_elems();
  const int batch1 = 2 * nk, batch = batch1 * nvec;
  // algorithmic traffic / work per stage: the bytes each stage must move at minimum for
  // its design and its nominal flops, accumulated by the profiler
  const double c = sizeof(cx<T>), re = sizeof(T);
  const double V = (double)br * nvec, G = (double)rows * nr, Gu = (double)s.rows() * nr;
  if (adj_mask) {  // L^H x = J L J x for the flagged vectors
    if (w.xin.bytes < (size_t)V * sizeof(cx<T>)) w.xin.alloc((size_t)V * sizeof(cx<T>));
    ProfScope ps(pf, st, ST_LANCZOS, 2 * V * c, 0);
    cx<T> *xin = w.xin.template as<cx<T>>();
    for (int v = 0; v < nvec; ++v) {
      if (adj_mask >> v & 1u)
        jflip_copy<T>(ctx, s, x + v * br, xin + v * br);
      else
        TDLZ_CUDA_TRY(cudaMemcpyAsync(xin + v * br, x + v * br, br * sizeof(cx<T>),
                                      cudaMemcpyDeviceToDevice, st));
    }
    x = xin;
  }
  cx<T> *i1 = w.i1.template as<cx<T>>();
  cx<T> *rho = w.rho.template as<cx<T>>();
  cx<T> *vp = w.vpot.template as<cx<T>>();
  cx<T> *hg = w.hgrid.template as<cx<T>>();
  cx<T> *h = w.h.template as<cx<T>>();
  const bool use_h = s.kernel_mask & TDLZ_KERNEL_HARTREE, use_xc = s.kernel_mask & TDLZ_KERNEL_XC;
  // Hartree at q (Eq. v_H_q): rho'_0 -> G, 4 pi / |q+G|^2 on the density sphere, -> r
  auto hartree = [&](int nv) {
    ProfScope ps(pf, st, ST_HARTREE, 8.0 * nv * nr * c,
                 2 * 5.0 * nv * nr * std::log2((double)nr));
    long long tot = (long long)nv * nr;
    gather_component_kernel<T><<<blocks_for(tot), kThreads, 0, st>>>(rho, hg, nr, 4 * nr, tot);
    TDLZ_LAUNCH_CHECK();
    fft3d<T>(s.plan, hg, nv, -1, st);
    scale_periodic_kernel<T><<<blocks_for(tot), kThreads, 0, st>>>(
        hg, d.vhfac.template as<T>(), nr, tot);
    TDLZ_LAUNCH_CHECK();
    fft3d<T>(s.plan, hg, nv, +1, st);
  };
  const bool planes = sizeof(T) == 4 ? s.planes32 : s.planes64;
  if (planes) {
    // 1-6 on the fused plane stages (planes.cu): the stick buffer is the only real-space
    // intermediate in HBM.  Exact work of one pass: sticks and planes of every row's k.
    const int n2 = s.fft[1], n3 = s.fft[2];
    double st_rows = 0, yx_lines = 0;
    for (int k = 0; k < nk; ++k) {
      st_rows += 4.0 * nb * s.nst_h[k];
      yx_lines += 4.0 * nb * (s.npl_h[k] + n2);
    }
    const double S1 = nvec * st_rows * n3;  // stick buffer elements touched
    const double z_fl = nvec * st_rows * 5.0 * n3 * std::log2((double)n3);
    const double yx_fl = nvec * yx_lines * n3 * 5.0 * n2 * std::log2((double)n2);
    const double pot_bytes = 6.0 * nvec * nr * c;
    {
      // sphere in, sticks out
      ProfScope ps(pf, st, ST_SCATTER, V * c + S1 * c, z_fl);
      sticks_inverse<T>(ctx, s, x, i1, nvec);
    }
    if (use_h || use_xc) {
      // sticks and U planes in, partial densities out and back, rho out
      const double nch = planes_density_chunks(s, nvec, sizeof(cx<T>));
      ProfScope ps(pf, st, ST_DENSITY, S1 * c + Gu * c + (2 * nch + 1) * 4 * nvec * nr * c,
                   yx_fl + (double)nbs * nr * 40.0);
      planes_density<T>(ctx, s, i1, d.us.template as<cx<T>>(), d.wk.template as<T>(),
                        w.rhopart.template as<cx<T>>(), rho, nvec);
    }
    if (use_h) hartree(nvec);
    {
      ProfScope ps(pf, st, ST_POTENTIAL,
                   nvec * (5 * nr * c + 14 * nr * re) + pot_bytes, 16.0 * 4 * nr * nvec);
      planes_potential<T>(ctx, s, rho, hg, d.fxc.template as<T>(), d.vloc.template as<T>(),
                          d.bfield.template as<T>(), vp, nvec, use_h, use_xc);
    }
    {
      // sticks in and out (in place), U planes, potential planes once per CTA
      ProfScope ps(pf, st, ST_PRODUCT, 2 * S1 * c + Gu * c + pot_bytes,
                   2 * yx_fl + (double)nbs * nr * 64.0);
      planes_product_forward<T>(ctx, s, i1, d.us.template as<cx<T>>(), vp, nvec,
                                [&] { sticks_inverse<T>(ctx, s, x, i1, nvec); });
    }
    {
      // sticks in; x read, h written on the sphere and zero on the padding
      ProfScope ps(pf, st, ST_GATHER, S1 * c + 3 * V * c, z_fl);
      sticks_forward<T>(ctx, s, x, i1, d.kin.template as<T>(), d.evals.template as<T>(), h,
                        nvec);
    }
  } else {
    cx<T> *xr = w.xr.template as<cx<T>>();
    cx<T> *i2 = w.i2.template as<cx<T>>();
    const int nsub = staged_sub(w.ns_cap, nvec);
    for (int v0 = 0; v0 < nvec; v0 += nsub) {
      // vectors v0 .. v0 + m - 1: their grids, plane and stick buffers fill the workspace
      const int m = std::min(nsub, nvec - v0);
      const cx<T> *xs = x + (long long)v0 * br;
      cx<T> *hs = h + (long long)v0 * br;
      const double Gm = (double)s.rows() * m * nr;
      // 1. sphere -> real space (pruned Z, Y passes; full X pass)
      pipeline_inverse<T>(ctx, s, xs, xr, i1, i2, m);  // profiled per stage inside
      // 2-4. densities and HXC potentials (one set per vector)
      if (use_h || use_xc) {
        {
          ProfScope ps(pf, st, ST_DENSITY, Gm * c + Gu * c * ((m + 2) / 3) + 4 * m * nr * c,
                       (double)Gm / 2 * 40.0);
          launch_density<T>(ctx, d.ur.template as<cx<T>>(), xr, d.wk.template as<T>(), rho,
                            w.rhopart.template as<cx<T>>(), nk, nb, nr, m);
        }
        if (use_h) hartree(m);
        ProfScope ps(pf, st, ST_POTENTIAL, m * (9 * nr * c + 10 * nr * re),
                     16.0 * 4 * nr * m);
        for (int v = 0; v < m; ++v) {
          potential_kernel<T><<<blocks_for(nr), kThreads, 0, st>>>(
              rho + (long long)v * 4 * nr, hg + (long long)v * nr, d.fxc.template as<T>(),
              vp + (long long)v * 4 * nr, nr, use_h ? 1 : 0, use_xc ? 1 : 0);
          TDLZ_LAUNCH_CHECK();
        }
      } else {
        TDLZ_CUDA_TRY(cudaMemsetAsync(vp, 0, w.vpot.bytes, st));
      }
      // 5-6. local products; pruned X, Y, Z forward passes with the sphere gather and
      //      + (kin - e) x fused into the last one
      pipeline_forward<T>(ctx, s, xs, xr, d.ur.template as<cx<T>>(), d.vloc.template as<T>(),
                          d.bfield.template as<T>(), vp, d.kin.template as<T>(),
                          d.evals.template as<T>(), i1, i2, hs, m);  // profiled inside
    }
  }
  // 7. nonlocal pseudopotential (projector tables shared by all vectors: batch b -> k = b % nk)
  const long long bstride = (long long)nb * 2 * npwx;
  if (np_ > 0) {
    double bb = (double)nk * np_ * npwx * c;
    ProfScope ps(pf, st, ST_VNL, 3 * V * c + 2 * bb,
                 2 * 8.0 * batch * (double)np_ * 2 * nb * npwx);
    cx<T> *proj = w.proj.template as<cx<T>>();
    cx<T> *dm = w.dmix.template as<cx<T>>();
    bool tc = false;
    if constexpr (sizeof(T) == 4)
      if (s.tensor_gemm)
        tc = tc_gemm_tn(ctx, w.part, d.beta.template as<float2>(), npwx, (long long)np_ * npwx,
                        nk, x, npwx, bstride, proj, (long long)np_ * 2 * nb, 2 * nb, 1, np_,
                        2 * nb, npwx, batch);
    if (!tc)
      gemm_tn<T>(ctx, w.part, d.beta.template as<cx<T>>(), npwx, (long long)np_ * npwx, nk, x,
                 npwx, bstride, proj, (long long)np_ * 2 * nb, 2 * nb, 1, np_, 2 * nb, npwx,
                 batch);
    long long tot = (long long)batch * nb * 2 * np_;
    dmix_kernel<T><<<blocks_for(tot), kThreads, 0, st>>>(
        proj, d.dnl_val.template as<cx<T>>(), s.dnl_col.as<int>(), s.dnl_w, dm, np_, nb, batch);
    TDLZ_LAUNCH_CHECK();
    bool tcu = false;
    if constexpr (sizeof(T) == 4)
      if (s.tensor_gemm) {
        if (d.beta_img.buf.p)
          tcu = tc_gemm_nn_img(ctx, d.beta_img, w.part, dm, (long long)2 * nb * np_, np_, 1, h,
                               h, npwx, bstride, 2 * nb, 1.f, batch, batch, 1 << 30);
        if (!tcu)
          tcu = tc_gemm_nn(ctx, dm, (long long)2 * nb * np_, np_, 1,
                           d.beta.template as<float2>(), npwx, (long long)np_ * npwx, nk, h, h,
                           npwx, bstride, 2 * nb, npwx, np_, 1.f, batch, batch, 1 << 30);
      }
    if (!tcu)
      gemm_nn<T>(ctx, dm, (long long)2 * nb * np_, np_, 1, d.beta.template as<cx<T>>(), npwx,
                 (long long)np_ * npwx, nk, h, h, npwx, bstride, 2 * nb, npwx, np_, T(1), batch,
                 batch);
  }
  // 8. P_c and the row sign (occupied k+q states shared: batch b -> (side, k) = b % 2nk;
  //    Y-side batches (b % 2nk >= nk) negated)
  {
    ProfScope ps(pf, st, ST_PC, 4 * V * c + (double)br * c,
                 2 * 8.0 * batch * (double)nb * nb * 2 * npwx);
    cx<T> *ov = w.ovl.template as<cx<T>>();
    const cx<T> *ukq = d.ukq.template as<cx<T>>();
    bool tc = false;
    if constexpr (sizeof(T) == 4)
      if (s.tensor_gemm)
        tc = tc_gemm_tn(ctx, w.part, ukq, 2LL * npwx, bstride, batch1, h, 2LL * npwx, bstride,
                        ov, (long long)nb * nb, nb, 1, nb, nb, 2LL * npwx, batch);
    if (!tc)
      gemm_tn<T>(ctx, w.part, ukq, 2LL * npwx, bstride, batch1, h, 2LL * npwx, bstride, ov,
                 (long long)nb * nb, nb, 1, nb, nb, 2LL * npwx, batch);
    bool tcu = false;
    if constexpr (sizeof(T) == 4)
      if (s.tensor_gemm) {
        if (d.ukq_img.buf.p)
          tcu = tc_gemm_nn_img(ctx, d.ukq_img, w.part, ov, (long long)nb * nb, 1, nb, h, y,
                               2LL * npwx, bstride, nb, -1.f, batch, nk, batch1);
        if (!tcu)
          tcu = tc_gemm_nn(ctx, ov, (long long)nb * nb, 1, nb, ukq, 2LL * npwx, bstride, batch1,
                           h, y, 2LL * npwx, bstride, nb, 2LL * npwx, nb, -1.f, batch, nk,
                           batch1);
      }
    if (!tcu)
      gemm_nn<T>(ctx, ov, (long long)nb * nb, 1, nb, ukq, 2LL * npwx, bstride, batch1, h, y,
                 2LL * npwx, bstride, nb, 2LL * npwx, nb, T(-1), batch, nk, batch1);
  }
  if (adj_mask) {
    ProfScope ps(pf, st, ST_LANCZOS, 2 * V * c, 0);
    for (int v = 0; v < nvec; ++v)
      if (adj_mask >> v & 1u) jflip_copy<T>(ctx, s, y + v * br, y + v * br);
  }
}

// v^mu = (P sigma^mu U, P+ sigma^mu T U) on the k+q spheres (Sec. 2.5).
template <class T>
void start_vector(Context &ctx, QSlot &s, int mu, cx<T> *v) {
  cudaStream_t st = ctx.stream;
  const int nk = s.nk, nb = s.nb, npwx = s.npwx;
  const int batch = 2 * nk;
  const long long bstride = (long long)nb * 2 * npwx;
  DevBuf tmpb, ovb, partb;
  tmpb.alloc((size_t)s.br_elems() * sizeof(double2));
  ovb.alloc((size_t)batch * nb * nb * sizeof(double2));
  partb.alloc((size_t)32 * batch * nb * nb * sizeof(double2));
  double2 *tmp = tmpb.as<double2>();
  sigma_u_kernel<double><<<blocks_for(2LL * nk * nb * npwx), kThreads, 0, st>>>(
      s.coeff_k.as<double2>(), s.map_kq_k.as<int>(), mu, tmp, nk, nb, npwx, 1.0);
  TDLZ_LAUNCH_CHECK();
  double2 *ov = ovb.as<double2>();
  const double2 *ukq = s.d64.ukq.as<double2>();
  gemm_tn<double>(ctx, partb, ukq, 2LL * npwx, bstride, batch, tmp, 2LL * npwx, bstride, ov,
                  (long long)nb * nb, nb, 1, nb, nb, 2LL * npwx, batch);
  if constexpr (sizeof(T) == 8) {
    gemm_nn<double>(ctx, ov, (long long)nb * nb, 1, nb, ukq, 2LL * npwx, bstride, batch, tmp, v,
                    2LL * npwx, bstride, nb, 2LL * npwx, nb, -1.0, batch, batch);
  } else {
    gemm_nn<double>(ctx, ov, (long long)nb * nb, 1, nb, ukq, 2LL * npwx, bstride, batch, tmp, tmp,
                    2LL * npwx, bstride, nb, 2LL * npwx, nb, -1.0, batch, batch);
    long long n = s.br_elems() * 2;
    convert_kernel<double, float><<<blocks_for(n), kThreads, 0, st>>>(
        reinterpret_cast<const double *>(tmp), reinterpret_cast<float *>(v), n);
    TDLZ_LAUNCH_CHECK();
  }
  TDLZ_CUDA_TRY(cudaStreamSynchronize(st));
}

// caller order <-> internal order of one BR vector: out[row][i] = in[row][idx[k][i]]
// (idx = perm: caller -> internal; idx = iperm: internal -> caller), zero where idx < 0
template <class T>
__global__ void permute_rows_kernel(const cx<T> *__restrict__ in, cx<T> *__restrict__ out,
                                    const int *__restrict__ idx, int nk, int nb, int npwx,
                                    long long nrows) {
  const long long row = blockIdx.y + (long long)gridDim.y * blockIdx.z;
  if (row >= nrows) return;
  const int k = (int)((row / (2 * nb)) % nk);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npwx; i += gridDim.x * blockDim.x) {
    const int g = idx[(long long)k * npwx + i];
    out[row * npwx + i] = g >= 0 ? in[row * npwx + g] : czero<T>();
  }
}

template <class T>
void apply_liouvillian_caller_order(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *y,
                                    bool adjoint) {
  const size_t bytes = (size_t)s.br_elems() * sizeof(cx<T>);
  if (s.io_x.bytes < bytes) s.io_x.alloc(bytes);
  if (s.io_y.bytes < bytes) s.io_y.alloc(bytes);
  cx<T> *xi = s.io_x.as<cx<T>>(), *yi = s.io_y.as<cx<T>>();
  const dim3 g = row_grid(s.rows(), s.npwx);
  permute_rows_kernel<T><<<g, kThreads, 0, ctx.stream>>>(x, xi, s.perm.as<int>(), s.nk, s.nb,
                                                         s.npwx, s.rows());
  TDLZ_LAUNCH_CHECK();
  apply_liouvillian<T>(ctx, s, xi, yi, 1, adjoint ? 1u : 0u);
  permute_rows_kernel<T><<<g, kThreads, 0, ctx.stream>>>(yi, y, s.iperm.as<int>(), s.nk, s.nb,
                                                         s.npwx, s.rows());
  TDLZ_LAUNCH_CHECK();
}

template void ensure_precision<double>(Context &, QSlot &);
template void ensure_precision<float>(Context &, QSlot &);
template void apply_liouvillian<double>(Context &, QSlot &, const double2 *, double2 *, int,
                                        unsigned);
template void apply_liouvillian<float>(Context &, QSlot &, const float2 *, float2 *, int,
                                       unsigned);
template void start_vector<double>(Context &, QSlot &, int, double2 *);
template void start_vector<float>(Context &, QSlot &, int, float2 *);
template void apply_liouvillian_caller_order<double>(Context &, QSlot &, const double2 *,
                                                     double2 *, bool);
template void apply_liouvillian_caller_order<float>(Context &, QSlot &, const float2 *,
                                                    float2 *, bool);

}  // namespace tdlz
