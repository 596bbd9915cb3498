// Pruned, fused sphere <-> real-space transforms (pipeline.cu).
#pragma once

#include <vector>

#include "engine.cuh"

namespace tdlz {

// Stick / plane tables of every k+q sphere (host-built at load, uploaded).
void build_stick_tables(QSlot &s, const std::vector<int> &idx_kq);

// True when the Y and X line passes of precision T can run fused, one CTA per (row,
// chunk of z planes) with the sphere's planes in shared memory (square x-y grid of a
// register-line length, the planes within the shared-memory limit): no plane buffer.
template <class T> bool yx_fused_supported(const QSlot &s);

// x (nvec stacked BR vectors) -> xr (real space, [nvec*rows][Nr]); i1, i2 are the
// stick and plane scratch ([rows][nstick_max][n3], [rows][nplane_max][n2][n3]).
template <class T>
void pipeline_inverse(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *xr, cx<T> *i1, cx<T> *i2,
                      int nvec);

// h = P_sphere FFT{[v_loc + s B.sigma] xr + W^s U} + (kin - e) x  (BR layout).
template <class T>
void pipeline_forward(Context &ctx, QSlot &s, const cx<T> *x, const cx<T> *xr, const cx<T> *ur,
                      const T *vloc, const T *bf, const cx<T> *v, const T *kin, const T *evals,
                      cx<T> *i1, cx<T> *i2, cx<T> *h, int nvec);

// Z passes alone, with the stick buffer i1t in [nvec*rows][n3][nstick_max] order
// (fused plane stages, planes.cu): sphere -> sticks, and sticks -> sphere + (kin - e) x.
template <class T>
void sticks_inverse(Context &ctx, QSlot &s, const cx<T> *x, cx<T> *i1t, int nvec);
template <class T>
void sticks_forward(Context &ctx, QSlot &s, const cx<T> *x, const cx<T> *i1t, const T *kin,
                    const T *evals, cx<T> *h, int nvec);

}  // namespace tdlz
