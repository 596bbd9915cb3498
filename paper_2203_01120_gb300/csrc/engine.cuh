// Internal state of the tdlz library: per-q-slot ground-state data resident in
// HBM, the Liouvillian workspaces, and the kernels' host-side entry points.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "../../include/tdlz.h"
#include "common.cuh"
#include "fft.cuh"
#include "profile.cuh"
#include "tuner.cuh"

namespace tdlz {

// Device buffer owned by the library (cudaMalloc / cudaFree).
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) {
    o.p = nullptr;
    o.bytes = 0;
  }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) {
      reset();
      p = o.p;
      bytes = o.bytes;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { reset(); }
  void alloc(size_t n) {
    reset();
    if (n == 0) return;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      throw Error{TDLZ_ERR_OOM, "cudaMalloc(" + std::to_string(n) + " bytes) failed: " +
                                    cudaGetErrorString(e)};
    }
    bytes = n;
  }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class U> U *as() const { return reinterpret_cast<U *>(p); }
};

// TF32 operand images of a constant matrix B[g][k][n] (tc_gemm.cu): for every 128-column
// tile and K tile of 8 complex k, the hi and lo parts in the canonical shared-memory
// layout the update GEMM's MMA reads, so that the GEMM moves them with bulk copies and
// converts nothing.  Twice the FP32 matrix in size, rounded up to whole tiles.
struct TcImage {
  DevBuf buf;
  int G = 0, K = 0, nct = 0, nkt = 0;
  long long ncol = 0;
};

// Ground-state data of one precision (T = double or float) on the device.
template <class T> struct SlotData {
  DevBuf ukq;    // [2][nk][nb][2][npwx] occupied k+q spinors (P_c)
  DevBuf ur;     // [2][nk][nb][2][Nr]   occupied k orbitals in real space
  DevBuf beta;   // [nk][nproj][npwx]
  DevBuf dnl;    // [2nproj][2nproj]
  DevBuf dnl_val;  // [2nproj][dnl_w] nonzero entries of each row of D (ELL form)
  DevBuf kin;    // [nk][npwx]  |k+q+G|^2/2   (real)
  DevBuf evals;  // [2][nk][nb]               (real)
  DevBuf vloc;   // [Nr]   (real)
  DevBuf bfield; // [3][Nr] (real)
  DevBuf fxc;    // [10][Nr] (real)
  DevBuf vhfac;  // [Nr]   4 pi / |q+G|^2 / Nr on the Hartree sphere (real)
  DevBuf wk;     // [nk]   (real)
  DevBuf uvec;   // [3][BR] u^lambda = J sigma^lambda U (unprojected)
  DevBuf us;     // plane stages: [2][nk][nb][2][n3][n1*n2 (even)] U(r) in z-major slabs
  // FP32 tensor-core path: operand images of U_kq (G = 2 nk, K = nb, 2 npwx columns) and
  // of the projectors (G = nk, K = nproj, npwx columns) for the P_c and V_NL updates
  TcImage ukq_img, beta_img;
  bool ready = false;
};

template <class T> struct Workspace {
  DevBuf xr;    // staged pipeline: [nvec][2][nk][nb][2][Nr] real-space response orbitals
  DevBuf rho;   // [nvec][4][Nr]
  DevBuf rhopart;  // [groups][nvec][4][Nr] partial densities
  DevBuf vpot;  // [nvec][4][Nr]; plane stages: potential planes [nvec][n3][6][n1*n2 (even)]
  DevBuf hgrid; // [Nr] Hartree scratch
  DevBuf h;     // [BR] sphere intermediate
  DevBuf xin;   // [BR] sign-flipped input for the adjoint
  DevBuf proj;  // [2nk][nproj][2nb]  <beta|x>
  DevBuf dmix;  // [2nk][2nb][nproj]
  DevBuf ovl;   // [2nk][nb][nb]      <U_kq|h>
  DevBuf part;  // split-K partial sums
  DevBuf i1;    // stick scratch: [rows][nstick_max][n3]; plane stages [rows][n3][nstick_max]
  DevBuf i2;    // staged pipeline: [rows][nplane_max][n2][n3] plane scratch
  int nvec_cap = 0;  // stacked vectors the buffers above are sized for
  int ns_cap = 1;    // staged pipeline: vectors per sub-batch its grids are sized for
  bool ready = false;
};

struct QSlot {
  int fft[3];
  long long nr;
  int nk, nb, npwx, nproj, kernel_mask;
  double omega;
  double q[3];
  std::vector<int> npw_k, npw_kq;
  std::vector<double> wk;
  // Every k+q-sphere array on the device (BR vectors, kin, beta, occupied k+q states,
  // idx_kq, map_kq_k, st_map) uses the internal plane-wave order: ascending grid index,
  // i.e. stick by stick with j3 ascending inside a stick.  perm[k][i] is the caller's
  // index of internal plane wave i; iperm[k][g] the internal index of caller index g.
  DevBuf perm, iperm;    // [nk][npwx] int32 (-1 beyond npw_kq)
  DevBuf io_x, io_y;     // caller-order <-> internal-order scratch of the apply entry point
  DevBuf idx_k, idx_kq;  // [nk][npwx] int32 grid index (-1 beyond npw)
  DevBuf map_kq_k;       // [nk][npwx] int32: index of the same G in the k sphere or -1
  DevBuf npwkq_d;        // [nk] int32
  DevBuf coeff_k;        // [2][nk][nb][2][npwx] occupied k spinors (FP64; start vectors)
  // stick / plane tables of the k+q spheres (pipeline.cu)
  int nstick_max = 0, nplane_max = 0;
  std::vector<int> nst_h, npl_h;  // sticks and planes per k (host copies)
  DevBuf st_n;    // [nk] sticks per k
  DevBuf st_map;  // [nk][nstick_max][n3] sphere index of (stick, j3) or -1
  DevBuf st_run;  // [nk][nstick_max + 1] int4 (first plane wave, run A length, run A j3, run B j3)
  bool st_runs = false;  // every stick is at most two j3 runs (st_run valid)
  DevBuf pl_n;    // [nk] planes per k
  DevBuf pl_j1;   // [nk][nplane_max] grid index j1 of each plane
  DevBuf pl_of;   // [nk][n1] plane index of j1 or -1
  DevBuf st_id;   // [nk][nplane_max][n2] stick index of (plane, j2) or -1
  int dnl_w = 0;   // nonzeros per row of D in the ELL form (padded)
  DevBuf dnl_col;  // [2nproj][dnl_w] column of each entry of dnl_val, -1 past the row's end
  // the Liouvillian of each precision runs the fused plane stages (planes.cu); otherwise
  // the staged pipeline with real-space grids in HBM (pipeline.cu)
  bool planes32 = false, planes64 = false;
  // the staged pipeline's Y and X line passes of each precision run fused (no plane
  // buffer in HBM; TDLZ_YX_FUSED=0 keeps the separate passes)
  bool yx32 = false, yx64 = false;
  // loaded for mixed precision only (TDLZ_MIXED_ONLY=1): the FP32 data is built at load
  // and the FP64 real-space orbitals are released; FP64 applications are refused
  bool mixed_only = false;
  size_t dev_total = 0;    // device memory (bytes): sizes the staged pipeline's sub-batches
  int staged_sub_env = 0;  // TDLZ_STAGED_SUB=n: at most n stacked vectors per staged pass
  bool tc_images = true;    // the updates read precomputed operand images (TcImage)
  bool tensor_gemm = true;  // FP32 V_NL / P_c reductions and updates on tcgen05 (tc_gemm.cu)
  FFTPlan plan;
  SlotData<double> d64;
  SlotData<float> d32;
  Workspace<double> w64;
  Workspace<float> w32;
  long long br_elems() const { return 2LL * nk * nb * 2 * npwx; }
  long long rows() const { return 2LL * nk * nb * 2; }
  ~QSlot() { plan.release(); }
};

struct Context {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;
  std::vector<std::unique_ptr<QSlot>> slots;
  Profiler prof;
  Tuner tuner;
};

template <class T> inline SlotData<T> &slot_data(QSlot &s) {
  if constexpr (sizeof(T) == 8)
    return s.d64;
  else
    return s.d32;
}
template <class T> inline Workspace<T> &slot_ws(QSlot &s) {
  if constexpr (sizeof(T) == 8)
    return s.w64;
  else
    return s.w32;
}

// --- Liouvillian (liouvillian.cu) ---
template <class T> void ensure_precision(Context &ctx, QSlot &s);
// y_v = L x_v (or L^H x_v = J L J x_v where bit v of adj_mask is set) for nvec
// vectors stacked contiguously in x and y (one BR vector each), in one pass.
template <class T>
void apply_liouvillian(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *y, int nvec,
                       unsigned adj_mask);
template <class T> void start_vector(Context &ctx, QSlot &s, int mu, cx<T> *v);
// y = L x (or L^H x) for one vector in the caller's plane-wave order (x, y device).
template <class T>
void apply_liouvillian_caller_order(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *y,
                                    bool adjoint);
void load_slot(Context &ctx, QSlot &s, const tdlz_ground_state *gs);

// --- allocation-free spectrum (spectrum_noalloc.cu) ---
void spectrum_noalloc(Context &ctx, const tdlz_coeffs *c, const tdlz_spectrum_params *sp,
                      double *chi, int nomega);

// --- vector helpers (lanczos.cu) ---
template <class T>
void jflip_copy(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *y);

inline unsigned blocks_for(long long n, int t = 256) {
  long long b = (n + t - 1) / t;
  if (b > 2147483647LL) b = 2147483647LL;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace tdlz
