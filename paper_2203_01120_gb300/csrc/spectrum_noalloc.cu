// tdlz_spectrum_noalloc: the pivoted tridiagonal spectrum solve for callers that
// cannot allocate device memory.  Inputs and outputs are the caller's device
// buffers; the elimination rows live in one file-scope static device array of
// fixed size, shared by every call on a device and kept by every GPU that loads
// the library until the process exits.
#include <cmath>
#include <mutex>

#include "engine.cuh"
#include "spectrum_solve.cuh"

namespace tdlz {

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)TDLZ_NOALLOC_SCRATCH_MB << 20;
constexpr int kMaxDevices = 64;

// The scratch.  Device code could name it directly; host code must not pass
// the symbol itself to a kernel (on the host it is only a stand-in), so the
// device address is looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) double2 g_spec_scratch[kNoallocScratchBytes / sizeof(double2)];

std::mutex g_mu;
double2 *g_scratch_ptr[kMaxDevices] = {nullptr};

// One thread per (chain, omega) of the chunk [w0, w0 + nw); rows stored at
// scratch[(q * cap + i) * nthr + tid] for q = d, du, du2, b.
__global__ void spectrum_noalloc_kernel(int nchain, int nomega, int cap, const int *steps,
                                        const double2 *alpha, const double *beta,
                                        const double2 *gamma, const double2 *z, const double *n0,
                                        const double *wk, double start, double step, double eta,
                                        int w0, int nw, int nl, double2 *scratch, double2 *chi) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nthr = (long long)nchain * nw;
  if (tid >= nthr) return;
  int c = (int)(tid / nw);
  int iw = w0 + (int)(tid - (long long)c * nw);
  int m = steps[c];  // read on the device: clamped to [0, cap]
  if (m > cap) m = cap;
  double2 *out = chi + ((long long)c * nl) * nomega + iw;
  if (m <= 0) {
    for (int l = 0; l < nl; ++l) out[(long long)l * nomega] = make_double2(0, 0);
    return;
  }
  const double2 *al = alpha + (long long)c * cap;
  const double *be = beta + (long long)c * cap;
  const double2 *ga = gamma + (long long)c * cap;
  const double2 *zz = z + (long long)c * nl * cap;
  double2 acc[4];
  tridiag_chi(m, cap, al, be, ga, zz, make_double2(start + step * iw, eta), make_double2(0, 0),
              scratch, nthr, tid, nl, acc);
  double s = wk[c] * n0[c];
  for (int l = 0; l < nl; ++l) out[(long long)l * nomega] = make_double2(s * acc[l].x, s * acc[l].y);
}

// Device address of the scratch on the current device; looked up once per device.
double2 *scratch_on_current_device(int dev) {
  TDLZ_REQUIRE(dev >= 0 && dev < kMaxDevices, TDLZ_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_spec_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw Error{TDLZ_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") +
                                     cudaGetErrorString(e)};
    g_scratch_ptr[dev] = static_cast<double2 *>(p);
  }
  return g_scratch_ptr[dev];
}

}  // namespace

void spectrum_noalloc(Context &ctx, const tdlz_coeffs *c, const tdlz_spectrum_params *sp,
                      double *chi, int nomega) {
  TDLZ_REQUIRE(c && sp && chi, TDLZ_ERR_ARG, "NULL coefficients, parameters or chi");
  TDLZ_REQUIRE(c->nchain >= 1 && c->nsteps >= 1, TDLZ_ERR_ARG, "empty coefficient set");
  TDLZ_REQUIRE(c->ncomp == 0 || c->ncomp == 3 || c->ncomp == 4, TDLZ_ERR_ARG,
               "ncomp must be 0 or 3 (spin) or 4 (spin and charge)");
  TDLZ_REQUIRE(c->steps && c->alpha && c->beta && c->gamma && c->z && c->n0 && c->wk,
               TDLZ_ERR_ARG, "NULL coefficient array");
  TDLZ_REQUIRE(sp->step > 0 && sp->end >= sp->start && std::isfinite(sp->eta) && sp->eta > 0,
               TDLZ_ERR_ARG, "need step > 0, end >= start and eta > 0");
  TDLZ_REQUIRE(sp->units == 0 || sp->units == 1, TDLZ_ERR_ARG, "units must be 0 (Ha) or 1 (meV)");
  TDLZ_REQUIRE(sp->itermax0 == 0 && sp->extrapolation == 0, TDLZ_ERR_ARG,
               "tdlz_spectrum_noalloc uses every computed step and no extrapolation");
  long long nw = (long long)std::floor((sp->end - sp->start) / sp->step + 0.5) + 1;
  TDLZ_REQUIRE(nw == nomega, TDLZ_ERR_ARG,
               "nomega does not match the frequency grid (query it with tdlz_spectrum, chi = NULL)");
  TDLZ_REQUIRE(nw <= (1LL << 24), TDLZ_ERR_ARG, "at most 2^24 frequencies");
  // every frequency needs 4 complex rows of length nsteps per chain
  const long long per_omega = 4LL * c->nsteps * c->nchain;  // double2 elements
  const long long cap_elems = (long long)(kNoallocScratchBytes / sizeof(double2));
  TDLZ_REQUIRE(per_omega <= cap_elems, TDLZ_ERR_ARG,
               "nchain * nsteps exceeds the static scratch of tdlz_spectrum_noalloc (" +
                   std::to_string(TDLZ_NOALLOC_SCRATCH_MB) + " MiB holds nchain * nsteps <= " +
                   std::to_string(cap_elems / 4) + ")");
  double2 *scratch = scratch_on_current_device(ctx.device);
  const double conv = sp->units == 1 ? 1.0 / 27211.386245988 : 1.0;
  const int chunk = (int)std::min<long long>(nw, cap_elems / per_omega);
  for (int w0 = 0; w0 < nomega; w0 += chunk) {
    int n = std::min(chunk, nomega - w0);
    long long nthr = (long long)c->nchain * n;
    spectrum_noalloc_kernel<<<blocks_for(nthr, 128), 128, 0, ctx.stream>>>(
        c->nchain, nomega, c->nsteps, c->steps, reinterpret_cast<const double2 *>(c->alpha),
        c->beta, reinterpret_cast<const double2 *>(c->gamma),
        reinterpret_cast<const double2 *>(c->z), c->n0, c->wk, sp->start * conv, sp->step * conv,
        sp->eta * conv, w0, n, c->ncomp == 4 ? 4 : 3, scratch, reinterpret_cast<double2 *>(chi));
    TDLZ_LAUNCH_CHECK();
  }
}

}  // namespace tdlz
