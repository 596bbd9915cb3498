// Spectrum kernel arguments (device pointers).
#pragma once

#include "engine.cuh"

namespace tdlz {

struct SpecArgs {
  int nchain, nomega, cap;
  const int *steps;      // [nchain]
  const double2 *alpha;  // [nchain][cap]
  const double *beta;    // [nchain][cap]
  const double2 *gamma;  // [nchain][cap]
  const double2 *z;      // [nchain][nl][cap]
  int nl;                // left vectors per chain: 3 (spin) or 4 (spin and charge)
  const double *n0, *wk; // [nchain]
  double start, step, eta;
  int itermax0, itermax, extrap;  // itermax0 <= 0: all computed; extrap 0 no, 1 constant, 2 osc
  double2 *scratch;      // [4][cap][nchain*nomega]
  double2 *chi;          // [nchain][nl][nomega]
};

void launch_spectrum(cudaStream_t st, const SpecArgs &a);

// P_perp(q) = 1 - q q^T / q^2
struct PerpProj {
  double m[3][3];
};
// S[w] = -Im Tr[P chi(w)] from the 3 x 3 susceptibility chi[mu][lambda][w] (device arrays).
void launch_structure_factor(cudaStream_t st, const double2 *chi, int nomega, const PerpProj &p,
                             double *S);

}  // namespace tdlz
