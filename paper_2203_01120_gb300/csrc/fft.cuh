// Batched 3D complex FFT on an n1 x n2 x n3 C-order grid (own kernels).
//
// The plane-wave maps of the method (sphere -> grid -> real space and back,
// and the Hartree solve of Eq. v_H_q) need many independent small 3D FFTs of
// mixed-radix lengths (12, 16, 36, 45, 96, 144: factors 2, 3, 4, 5).  Each axis
// pass loads a tile of lines into shared memory, runs a self-sorting Stockham
// transform there stage by stage (radix 4, 2, 3, 5), and writes the tile back;
// lines along the strided axes are grouped so that every global access is
// coalesced along the contiguous grid index.  Transforms are unnormalised:
//   dir = +1 : f_j = sum_m c_m exp(+2 pi i m j / n)   (sphere -> real space)
//   dir = -1 : c_m = sum_j f_j exp(-2 pi i m j / n)   (real space -> sphere)
#pragma once

#include "common.cuh"

namespace tdlz {

struct AxisPlan {
  int n = 0;
  int nrad = 0;
  int radix[8] = {0};
  double2 *tw_d = nullptr;  // exp(+2 pi i t / n), t in [0, n)
  float2 *tw_f = nullptr;
};

struct FFTPlan {
  int n[3] = {0, 0, 0};
  long long nr = 0;
  AxisPlan ax[3];
  void init(const int fft[3]);
  void release();
};

template <class T>
void fft3d(const FFTPlan &plan, cx<T> *data, long long batch, int dir, cudaStream_t st);

bool fft_length_supported(int n);

}  // namespace tdlz
