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
#include "spectrum_solve.cuh"

namespace tdlz {

__global__ void spectrum_kernel(SpecArgs a) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nthr = (long long)a.nchain * a.nomega;
  if (tid >= nthr) return;
  int c = (int)(tid / a.nomega);
  int iw = (int)(tid - (long long)c * a.nomega);
  int m = a.steps[c];
  if (a.itermax0 > 0 && a.itermax0 < m) m = a.itermax0;
  double2 *out = a.chi + ((long long)c * a.nl) * a.nomega + iw;
  if (m <= 0) {
    for (int l = 0; l < a.nl; ++l) out[(long long)l * a.nomega] = make_double2(0, 0);
    return;
  }
  const double2 *al = a.alpha + (long long)c * a.cap;
  const double *be = a.beta + (long long)c * a.cap;
  const double2 *ga = a.gamma + (long long)c * a.cap;
  const double2 *zz = a.z + (long long)c * a.nl * a.cap;
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
      g = spec_cdiv(make_double2(1.0, 0.0), den);
    }
    double2 bg = make_double2(be[m - 1] * ga[m - 1].x, be[m - 1] * ga[m - 1].y);
    tail = make_double2(bg.x * g.x - bg.y * g.y, bg.x * g.y + bg.y * g.x);
  }
  double2 acc[4];
  tridiag_chi(m, a.cap, al, be, ga, zz, zw, tail, a.scratch, nthr, tid, a.nl, acc);
  double s = a.wk[c] * a.n0[c];
  for (int l = 0; l < a.nl; ++l)
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
