// Fused plane-by-plane real-space stages of the Liouvillian (planes.cu).
#pragma once

#include <functional>

#include "engine.cuh"

namespace tdlz {

// True when slot s can run the fused plane stages in precision T: square x-y grid
// (n1 == n2) of a register-line length, a register plan for the z lines, and the
// per-CTA shared memory of both passes within the limit.
template <class T> bool planes_supported(const QSlot &s);

// Elements per z plane of the plane-ordered arrays (n1*n2 rounded up to even).
long long planes_nnp(const QSlot &s);

// U slabs us[row][j3][i] (row = 2*band-side + spin, i = j1*n2 + j2, padded to
// planes_nnp) from the real-space orbitals ur[row][i*n3 + j3].
template <class T> void planes_build_u(Context &ctx, QSlot &s, const double2 *ur, DevBuf &us);

// The inverse reordering, rounded to T: ur[row][i*n3 + j3] = us[row][j3][i] (the
// staged pipeline's orbitals from the FP64 slabs, once the grid-order copy is gone).
template <class T> void planes_grid_from_slabs(Context &ctx, QSlot &s, const double2 *us,
                                               DevBuf &ur);

// Number of band-side chunks of the density pass for nvec stacked vectors (a
// function of the problem shape and the device only: it fixes the summation order).
int planes_density_chunks(const QSlot &s, int nvec, size_t elem);

// Pass A: rho[v][a][r] (standard grid order) of nvec stacked vectors from the stick
// buffer i1t ([nvec*rows][n3][nstick_max], after the inverse Z pass).  Each z plane
// of every band-side is transformed (Y then X lines) on chip and contracted with U
// there; only partial densities part[chunk][v][4][n3][n1*n2] reach HBM.
template <class T>
void planes_density(Context &ctx, QSlot &s, const cx<T> *i1t, const cx<T> *us, const T *wk,
                    cx<T> *part, cx<T> *rho, int nvec);

// Potential planes pot[v][j3][6][nnp]: v'_0..v'_3 = delta_a0 vH + f_ab rho_b, then
// (v_loc, B_z) and (B_x, B_y) packed as complex pairs.
template <class T>
void planes_potential(Context &ctx, QSlot &s, const cx<T> *rho, const cx<T> *vh, const T *fxc,
                      const T *vloc, const T *bf, cx<T> *pot, int nvec, bool use_h, bool use_xc);

// Pass B: for every band-side and z plane, the inverse Y and X lines again, the local
// products [v_loc + s B.sigma] x + W^s U, and the forward X and Y lines, written back
// into the stick buffer i1t in place (the forward Z pass follows).  refill() enqueues
// what recreates i1t's input (the inverse Z pass); the autotuner calls it between its
// timed candidate runs of this in-place stage.
template <class T>
void planes_product_forward(Context &ctx, QSlot &s, cx<T> *i1t, const cx<T> *us,
                            const cx<T> *pot, int nvec, const std::function<void()> &refill);

}  // namespace tdlz
