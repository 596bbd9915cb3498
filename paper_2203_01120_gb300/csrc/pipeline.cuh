// Pruned, fused sphere <-> real-space transforms (pipeline.cu).
#pragma once

#include <vector>

#include "engine.cuh"

namespace tdlz {

// Stick / plane tables of every k+q sphere (host-built at load, uploaded).
void build_stick_tables(QSlot &s, const std::vector<int> &idx_kq);

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

}  // namespace tdlz
