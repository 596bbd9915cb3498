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
  double2 *z;      // [4][cap] (z^x, z^y, z^z, and the charge's where ncomp = 4)
  double *beta;    // [cap]
};

struct Chain {
  int qslot = 0, mu = 0;  // mu = 0, 1, 2: sigma^x,y,z perturbation; 3: the charge
  int group = -1, index = 0;  // its group and position in the group's vector blocks
  DevBuf coef, sc;
  ChainCoeffs cf{};
};

// Chains on one q-slot: their vectors are stacked so one Liouvillian pass serves all.
struct Group {
  int qslot = 0;
  std::vector<int> members;
  int nv = 0;  // vectors per slot block (2 x members for NH)
  DevBuf vec;
  void *slot[4] = {nullptr, nullptr, nullptr, nullptr};
  int host_step = 0;
};

struct ChainSet {
  Context *ctx = nullptr;
  int flavor = 0, precision = 0, cap = 0;
  int ncomp = 3;  // left vectors u^l recorded per step: 3 (spin) or 4 (spin and charge)
  std::vector<Chain> chains;
  std::vector<Group> groups;
  DevBuf red;
  // Two steps captured as one CUDA graph (the vector-slot rotation has period 2) and
  // replayed; valid while the slot arrangement equals the captured one.
  cudaGraphExec_t gexec = nullptr;
  std::vector<void *> graph_key;  // slot pointers of every group at capture
  long long graph_kernels = 0;    // kernels in the captured graph
  bool use_graphs = true;
  ~ChainSet();
  void init();
  void advance(int nsteps);
  void read(tdlz_lanczos_result *res);
  // restart image: header, each group's vector slots in logical order, each
  // chain's device scalars and coefficients
  size_t state_bytes() const;
  void save(void *host, size_t bytes);
  void restore(const void *host, size_t bytes);

 private:
  template <class T> void init_impl();
  template <class T> void advance_impl(int nsteps);
  void advance_eager(int nsteps);
  std::vector<void *> slot_key() const;
  void capture_two_steps();
};

}  // namespace tdlz
