// chi(omega) from the Lanczos tridiagonal matrix (Eqs.
// resolvent_Liouvillian_Lanczos_q and post_processing), FP64 on the GPU.
//
// One thread per (chain, omega) solves (omega + i eta - T) x = e_1 by Gaussian
// elimination with partial pivoting on the tridiagonal (the row interchange
// creates a second super-diagonal), then forms chi_l = w n0 sum_i conj(z^l_i) x_i
// during the back substitution.  The eliminated rows are kept in a scratch
// array laid out [step][thread] so that every step's access is coalesced.
#include <cmath>
#include <vector>

#include "spectrum.cuh"

namespace tdlz {

namespace {

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // a / b with scaling (Smith's method)
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  double r = b.x / b.y, den = b.x * r + b.y;
  return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }

}  // namespace

__global__ void spectrum_kernel(SpecArgs a) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nthr = (long long)a.nchain * a.nomega;
  if (tid >= nthr) return;
  int c = (int)(tid / a.nomega);
  int iw = (int)(tid - (long long)c * a.nomega);
  int m = a.steps[c];
  if (a.itermax0 > 0 && a.itermax0 < m) m = a.itermax0;
  double2 *out = a.chi + ((long long)c * 3) * a.nomega + iw;
  if (m <= 0) {
    for (int l = 0; l < 3; ++l) out[(long long)l * a.nomega] = make_double2(0, 0);
    return;
  }
  const double2 *al = a.alpha + (long long)c * a.cap;
  const double *be = a.beta + (long long)c * a.cap;
  const double2 *ga = a.gamma + (long long)c * a.cap;
  const double2 *zz = a.z + (long long)c * 3 * a.cap;
  double om = a.start + a.step * iw;
  double2 zw = make_double2(om, a.eta);
  // Extrapolated tail (Sec. 3.3): coefficients m..itermax-1 are the means of the
  // computed ones over [m/2, m) (per parity for the bi-constant form), z = 0
  // there; the tail enters through the backward continued fraction g and one
  // modified diagonal entry d_{m-1} -= beta_{m-1} gamma_{m-1} g.
  double2 tail = make_double2(0, 0);
  if (a.extrap != 0 && a.itermax > m && m >= 2) {
    double2 ca[2] = {{0, 0}, {0, 0}}, cg[2] = {{0, 0}, {0, 0}};
    double cb[2] = {0, 0};
    int cnt[2] = {0, 0};
    for (int j = m / 2; j < m; ++j) {
      int p = a.extrap == 2 ? (j & 1) : 0;
      ca[p].x += al[j].x;
      ca[p].y += al[j].y;
      cb[p] += be[j];
      cg[p].x += ga[j].x;
      cg[p].y += ga[j].y;
      cnt[p]++;
    }
    if (a.extrap != 2) {
      ca[1] = ca[0];
      cb[1] = cb[0];
      cg[1] = cg[0];
      cnt[1] = cnt[0];
    }
    for (int p = 0; p < 2; ++p) {
      double inv = cnt[p] > 0 ? 1.0 / cnt[p] : 0.0;
      ca[p] = make_double2(ca[p].x * inv, ca[p].y * inv);
      cb[p] *= inv;
      cg[p] = make_double2(cg[p].x * inv, cg[p].y * inv);
    }
    double2 g = make_double2(0, 0);
    for (int j = a.itermax - 1; j >= m; --j) {
      int p = j & 1;
      double2 den = make_double2(zw.x - ca[p].x, zw.y - ca[p].y);
      if (j < a.itermax - 1) {  // - beta_j gamma_j g_{j+1}
        double2 bg = make_double2(cb[p] * cg[p].x, cb[p] * cg[p].y);
        den.x -= bg.x * g.x - bg.y * g.y;
        den.y -= bg.x * g.y + bg.y * g.x;
      }
      g = cdiv(make_double2(1.0, 0.0), den);
    }
    double2 bg = make_double2(be[m - 1] * ga[m - 1].x, be[m - 1] * ga[m - 1].y);
    tail = make_double2(bg.x * g.x - bg.y * g.y, bg.x * g.y + bg.y * g.x);
  }
  // scratch rows (final d, du, du2, b) at [j][tid]
  double2 *sd = a.scratch, *sdu = a.scratch + (long long)a.cap * nthr,
          *sdu2 = a.scratch + 2LL * a.cap * nthr, *sb = a.scratch + 3LL * a.cap * nthr;
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
    double2 bn = make_double2(0, 0);
    double2 du2 = make_double2(0, 0);
    if (cabs2(d) >= cabs2(dl)) {
      double2 f = cdiv(dl, d);
      dn = make_double2(dn.x - (f.x * du.x - f.y * du.y), dn.y - (f.x * du.y + f.y * du.x));
      bn = make_double2(bn.x - (f.x * b.x - f.y * b.y), bn.y - (f.x * b.y + f.y * b.x));
    } else {
      double2 f = cdiv(d, dl);
      double2 tmp = dn;
      double2 nd = dl;
      dn = make_double2(du.x - (f.x * tmp.x - f.y * tmp.y), du.y - (f.x * tmp.y + f.y * tmp.x));
      du2 = dun;
      dun = make_double2(-(f.x * du2.x - f.y * du2.y), -(f.x * du2.y + f.y * du2.x));
      du = tmp;
      d = nd;
      double2 tb = b;
      b = bn;  // = 0
      bn = make_double2(tb.x - (f.x * b.x - f.y * b.y), tb.y - (f.x * b.y + f.y * b.x));
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
  // back substitution with chi accumulation
  double2 x1 = make_double2(0, 0), x2 = make_double2(0, 0);  // x_{i+1}, x_{i+2}
  double2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int i = m - 1; i >= 0; --i) {
    long long o = (long long)i * nthr + tid;
    double2 bi = sb[o], dui = sdu[o], du2i = sdu2[o];
    double2 num = make_double2(bi.x - (dui.x * x1.x - dui.y * x1.y) - (du2i.x * x2.x - du2i.y * x2.y),
                               bi.y - (dui.x * x1.y + dui.y * x1.x) - (du2i.x * x2.y + du2i.y * x2.x));
    double2 xi = cdiv(num, sd[o]);
    for (int l = 0; l < 3; ++l) {
      double2 zv = zz[(long long)l * a.cap + i];
      acc[l].x += zv.x * xi.x + zv.y * xi.y;
      acc[l].y += zv.x * xi.y - zv.y * xi.x;
    }
    x2 = x1;
    x1 = xi;
  }
  double s = a.wk[c] * a.n0[c];
  for (int l = 0; l < 3; ++l)
    out[(long long)l * a.nomega] = make_double2(s * acc[l].x, s * acc[l].y);
}

// S(w) = -Im sum_ab P_ab chi_ba(w), chi[a][b][w] = chi_ba (chain a, row b)  (Eq. S_def)
__global__ void structure_factor_kernel(const double2 *__restrict__ chi, int nomega, PerpProj p,
                                        double *__restrict__ S) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nomega; w += gridDim.x * blockDim.x) {
    double im = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) im += p.m[a][b] * chi[((long long)a * 3 + b) * nomega + w].y;
    S[w] = -im;
  }
}

void launch_structure_factor(cudaStream_t st, const double2 *chi, int nomega, const PerpProj &p,
                             double *S) {
  structure_factor_kernel<<<blocks_for(nomega, 128), 128, 0, st>>>(chi, nomega, p, S);
  TDLZ_LAUNCH_CHECK();
}

void launch_spectrum(cudaStream_t st, const SpecArgs &a) {
  long long nthr = (long long)a.nchain * a.nomega;
  spectrum_kernel<<<blocks_for(nthr, 128), 128, 0, st>>>(a);
  TDLZ_LAUNCH_CHECK();
}

}  // namespace tdlz
