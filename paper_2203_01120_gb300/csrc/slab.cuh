// Plane-slab real-space stages of the mixed-precision Liouvillian (slab.cu).
#pragma once

#include "engine.cuh"

namespace tdlz {

// True when the FP32 Liouvillian of slot s can run the plane-slab stages: square
// x-y grid (n1 == n2) of a register-line length and per-CTA shared memory that fits.
bool slab_supported(const QSlot &s);

// us[band-side][spin][j3][j1*n2 + j2] (FP32) from the FP64 orbitals ur[band-side][spin][Nr].
void slab_build_u(Context &ctx, QSlot &s, const double2 *ur, DevBuf &us);

// Y and X inverse passes: stick buffer i1t ([nvec*rows][n3][nstick_max], after the
// inverse Z pass) -> real-space slabs xr ([nvec*rows][n3][n1*n2]).
void slab_inverse_yx(Context &ctx, QSlot &s, const float2 *i1t, float2 *xr, int nvec);

// Number of partial-density slices the density stage writes (part is
// [groups][nvec][4][Nr] complex).
int slab_density_groups(const QSlot &s);

// Response densities rho[nvec][4][Nr] (standard grid order) from the slabs xr.
void slab_density(Context &ctx, QSlot &s, const float2 *xr, const float2 *us, const float *wk,
                  float2 *part, float2 *rho, int nvec);

// t = [v_loc + s B.sigma] x + W^s U on the slabs, forward X and Y passes -> stick
// buffer i1t.  vpot is [nvec][4][Nr]; coef is scratch of nvec * 2 * 6 * Nr complex.
void slab_product_forward(Context &ctx, QSlot &s, const float2 *xr, const float2 *us,
                          const float2 *vpot, const float *vloc, const float *bf, float2 *coef,
                          float2 *i1t, int nvec);

}  // namespace tdlz
