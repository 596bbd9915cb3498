// The tridiagonal solve behind chi(omega) (Eqs. resolvent_Liouvillian_Lanczos_q and
// post_processing), shared by tdlz_spectrum and tdlz_spectrum_noalloc.
#pragma once

#include <cuda_runtime.h>

namespace tdlz {

// a / b with scaling (Smith's method)
__device__ __forceinline__ double2 spec_cdiv(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  double r = b.x / b.y, den = b.x * r + b.y;
  return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}

// (zw - T) x = e_1 for the m x m tridiagonal T (diagonal alpha, sub-diagonal beta,
// super-diagonal gamma), with `tail` subtracted from the last diagonal entry (the
// continued fraction of an extrapolated part; zero without one), by Gaussian
// elimination with partial pivoting (a row interchange creates a second
// super-diagonal).  The eliminated rows d, du, du2, b of thread tid go to
// scratch[(q cap + j) nthr + tid], q = 0..3, so that every step's accesses of the
// nthr threads are coalesced.  The back substitution accumulates
// acc[l] = sum_i conj(z^l_i) x_i for l < nl (zz = z of the chain, [nl][cap], nl <= 4).
__device__ __forceinline__ void tridiag_chi(int m, int cap, const double2 *al, const double *be,
                                            const double2 *ga, const double2 *zz, double2 zw,
                                            double2 tail, double2 *scratch, long long nthr,
                                            long long tid, int nl, double2 (&acc)[4]) {
  double2 *sd = scratch, *sdu = scratch + (long long)cap * nthr,
          *sdu2 = scratch + 2LL * cap * nthr, *sb = scratch + 3LL * cap * nthr;
  // A = zw - T: d_j = zw - alpha_j, dl_j = -beta_j (A[j+1][j]), du_j = -gamma_j (A[j][j+1])
  double2 d = make_double2(zw.x - al[0].x, zw.y - al[0].y);
  if (m == 1) d = make_double2(d.x - tail.x, d.y - tail.y);
  double2 du = m > 1 ? make_double2(-ga[0].x, -ga[0].y) : make_double2(0, 0);
  double2 b = make_double2(1.0, 0.0);
  for (int i = 0; i < m - 1; ++i) {
    double2 dl = make_double2(-be[i], 0.0);
    double2 dn = make_double2(zw.x - al[i + 1].x, zw.y - al[i + 1].y);  // d_{i+1}
    if (i + 1 == m - 1) dn = make_double2(dn.x - tail.x, dn.y - tail.y);
    double2 dun = (i + 1 < m - 1) ? make_double2(-ga[i + 1].x, -ga[i + 1].y) : make_double2(0, 0);
    double2 bn = make_double2(0, 0), du2 = make_double2(0, 0);
    if (hypot(d.x, d.y) >= hypot(dl.x, dl.y)) {  // row i stays the pivot row
      double2 f = spec_cdiv(dl, d);
      dn = make_double2(dn.x - (f.x * du.x - f.y * du.y), dn.y - (f.x * du.y + f.y * du.x));
      bn = make_double2(-(f.x * b.x - f.y * b.y), -(f.x * b.y + f.y * b.x));
    } else {  // rows i and i+1 swap (row i+1 becomes the pivot row)
      double2 f = spec_cdiv(d, dl);
      double2 old_dn = dn;
      dn = make_double2(du.x - (f.x * old_dn.x - f.y * old_dn.y),
                        du.y - (f.x * old_dn.y + f.y * old_dn.x));
      du2 = dun;
      dun = make_double2(-(f.x * du2.x - f.y * du2.y), -(f.x * du2.y + f.y * du2.x));
      du = old_dn;
      d = dl;
      bn = b;  // the right-hand side of row i+1 was zero before the swap
      b = make_double2(0, 0);
    }
    long long o = (long long)i * nthr + tid;
    sd[o] = d;
    sdu[o] = du;
    sdu2[o] = du2;
    sb[o] = b;
    d = dn;
    du = dun;
    b = bn;
  }
  {
    long long o = (long long)(m - 1) * nthr + tid;
    sd[o] = d;
    sdu[o] = make_double2(0, 0);
    sdu2[o] = make_double2(0, 0);
    sb[o] = b;
  }
  double2 x1 = make_double2(0, 0), x2 = make_double2(0, 0);  // x_{i+1}, x_{i+2}
  for (int l = 0; l < 4; ++l) acc[l] = make_double2(0, 0);
  for (int i = m - 1; i >= 0; --i) {
    long long o = (long long)i * nthr + tid;
    double2 bi = sb[o], dui = sdu[o], du2i = sdu2[o];
    double2 num = make_double2(bi.x - (dui.x * x1.x - dui.y * x1.y) - (du2i.x * x2.x - du2i.y * x2.y),
                               bi.y - (dui.x * x1.y + dui.y * x1.x) - (du2i.x * x2.y + du2i.y * x2.x));
    double2 xi = spec_cdiv(num, sd[o]);
    for (int l = 0; l < nl; ++l) {
      double2 zv = zz[(long long)l * cap + i];
      acc[l].x += zv.x * xi.x + zv.y * xi.y;
      acc[l].y += zv.x * xi.y - zv.y * xi.x;
    }
    x2 = x1;
    x1 = xi;
  }
}

}  // namespace tdlz
