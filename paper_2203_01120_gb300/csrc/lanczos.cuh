// Lanczos chain state (device scalars + vectors) for the recursions of Sec. 2.5.
#pragma once

#include "engine.cuh"

namespace tdlz {

struct ChainScalars {
  double2 alpha;       // alpha_j of the current step
  double2 gamma_prev;  // gamma_j (coefficient of q_{j-1})
  double beta_prev;    // beta_j
  double s;            // J-metric sign s_j (PH)
  double n0;           // start-vector norm in the flavour's metric
  double2 scale_q, scale_p;  // rescale factors for the new vectors
  int step, steps_done, status, stopped;
};

struct ChainCoeffs {
  int cap;
  double2 *alpha;  // [cap]
  double2 *gamma;  // [cap]
  double2 *z;      // [3][cap]
  double *beta;    // [cap]
};

struct Chain {
  int qslot = 0, mu = 0;
  DevBuf vec, coef, sc;
  void *v[6] = {nullptr};
  ChainCoeffs cf{};
  int host_step = 0;
};

struct ChainSet {
  Context *ctx = nullptr;
  int flavor = 0, precision = 0, cap = 0;
  std::vector<Chain> chains;
  DevBuf red;
  void init();
  void advance(int nsteps);
  void read(tdlz_lanczos_result *res);

 private:
  template <class T> void init_impl();
  template <class T> void advance_impl(int nsteps);
};

}  // namespace tdlz
