/*
 * tdlz -- Liouville-Lanczos spin susceptibility on one GB300 GPU (sm_103a).
 *
 * C ABI of the hot path of the paper's method (linear-response TDDFT in the
 * Liouville-Lanczos form for spin waves):
 *   tdlz_load_ground_state  -- the occupied spinor states, energies, ground
 *                              densities and pseudopotential data of Sec. 3.1
 *                              (the paper reads them from the SCF run);
 *   tdlz_apply_liouvillian  -- the Liouvillian in the batch representation,
 *                              Eq. Liouvillian_BR_q and the block actions that
 *                              follow it (Sec. 2.4);
 *   tdlz_lanczos_run / tdlz_chain_*
 *                           -- the non-Hermitian and pseudo-Hermitian Lanczos
 *                              recursions of Sec. 2.5 (coefficients alpha,
 *                              beta, gamma, z);
 *   tdlz_spectrum           -- chi(q, omega) from the tridiagonal matrix,
 *                              Eqs. resolvent_Liouvillian_Lanczos_q and
 *                              post_processing, with omega -> omega + i eta.
 *
 * Conventions (Hartree atomic units throughout; complex numbers are pairs of
 * doubles (re, im), or of floats where stated, the layout of C99 complex):
 *   - lattice rows are the direct vectors a_i (bohr); reciprocal b = 2 pi A^{-T};
 *   - FFT grid n1 x n2 x n3 in C order; Miller m lives at ((m mod n1) n2 + ...);
 *   - psi_s(r_j) = Omega^{-1/2} sum_g c[s][g] exp(i G.r_j) for sphere coefficients;
 *   - a response ("BR") vector is [2 sides X,Y][nk][nocc][2 spinor][npwx],
 *     zero beyond npw_kq[k]; side Y is the time-reversed (B -> -B) partner.
 *
 * Every call returns a status; tdlz_last_error() gives the message.  Invalid
 * input is rejected before any launch.  There is no CPU fallback: without a
 * usable GPU every call fails with TDLZ_ERR_CUDA.  Device work is enqueued on
 * the context's stream; asynchronous faults surface at the next synchronising
 * call (tdlz_synchronize, tdlz_chain_read, tdlz_lanczos_run, tdlz_spectrum).
 * A context is used by one host thread at a time.
 */
#ifndef TDLZ_H
#define TDLZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdlz_ctx tdlz_ctx;
typedef struct tdlz_chain tdlz_chain;

typedef enum {
  TDLZ_OK = 0,
  TDLZ_ERR_ARG = 1,       /* invalid argument (nothing was launched)            */
  TDLZ_ERR_STATE = 2,     /* call not valid in the current state                */
  TDLZ_ERR_CUDA = 3,      /* CUDA runtime error (incl. no device)               */
  TDLZ_ERR_OOM = 4,       /* device allocation failed                           */
  TDLZ_ERR_BREAKDOWN = 5, /* Lanczos breakdown: chain truncated (not an error   */
                          /* of the library; other chains continue)             */
  TDLZ_ERR_NUMERIC = 6,   /* non-finite coefficient / indefinite metric         */
  TDLZ_ERR_TIMEOUT = 7    /* a bounded device wait gave up                      */
} tdlz_status;

typedef enum { TDLZ_FP64 = 0, TDLZ_MIXED = 1 } tdlz_precision;

typedef enum {
  TDLZ_NONHERMITIAN = 0,           /* biorthogonal, two L products per step     */
  TDLZ_PSEUDOHERMITIAN = 1,        /* J metric (indefinite), one L per step     */
  TDLZ_PSEUDOHERMITIAN_POSDEF = 2  /* metric D+K = J L (positive), one L / step */
} tdlz_flavor;

enum { TDLZ_KERNEL_HARTREE = 1, TDLZ_KERNEL_XC = 2 };

/* Ground-state bundle (Sec. 3.1).  All pointers are HOST arrays, read during the
 * call and copied; the caller keeps ownership.  Sizes: Nr = fft[0]*fft[1]*fft[2].
 *   lattice[9]   rows a1,a2,a3 (bohr)            fft[3]     FFT grid
 *   ecutwfc      wavefunction cutoff (Ha); the Hartree sphere is |q+G|^2/2 <= 4 ecutwfc
 *   nk, nocc     k points, occupied spinor bands    npwx  padded sphere length
 *   nproj        number of Kleinman-Bylander projectors (all atoms)
 *   kpts[nk][3]  Cartesian (bohr^-1)      q[3] Cartesian (bohr^-1), |q| > 1e-8
 *   wk[nk]       k weights (the paper's 1/N_k)
 *   npw_k[nk], npw_kq[nk]            sphere sizes at k and k+q (<= npwx)
 *   miller_k[nk][npwx][3], miller_kq  Miller indices (int32), beyond npw ignored
 *   evals[2][nk][nocc]               e_{n,k} on sides X (H+) and Y (H-)
 *   coeff_k[2][nk][nocc][2][npwx]    occupied spinors at k     (complex double)
 *   coeff_kq[2][nk][nocc][2][npwx]   occupied spinors at k+q   (complex double)
 *   vloc[Nr], bfield[3][Nr]          local potential and exchange field (Ha)
 *   n0[Nr], m0[3][Nr]                ground charge and magnetisation densities
 *   beta_kq[nk][nproj][npwx]         projector values at k+q+G  (complex double)
 *   dnl[2nproj][2nproj]              projector coupling, index 2*i+spin, Hermitian
 *   kernel_mask                      TDLZ_KERNEL_HARTREE | TDLZ_KERNEL_XC (0 = chi0)
 */
typedef struct {
  double lattice[9];
  int fft[3];
  double ecutwfc;
  int nk, nocc, npwx, nproj;
  const double *kpts;
  double q[3];
  const double *wk;
  const int *npw_k, *npw_kq;
  const int *miller_k, *miller_kq;
  const double *evals;
  const double *coeff_k, *coeff_kq;
  const double *vloc, *bfield, *n0, *m0;
  const double *beta_kq;
  const double *dnl;
  int kernel_mask;
} tdlz_ground_state;

/* Lanczos parameters (Sec. 2.5; the paper's itermax, ipol, pseudo_hermitian).
 * Chain c runs on q-slot qslot[c] with start vector v^mu, mu = mu[c] in {0,1,2}
 * (the spin components x, y, z: v = (P sigma U, P+ sigma T U)) or 3 (the charge,
 * sigma^0: v = (P U, -P+ T U)), and records z^lambda for lambda = x, y, z and, with
 * ncomp = 4, the charge as a fourth (u^0 = (U, T U): the charge density enters the
 * Y side with +, the magnetisation with -, Eqs. charge_dens_resp_q /
 * spin_dens_resp_q) -- the 4 x 4 generalised susceptibility of Sec. 2.3.  ncomp 0
 * means 3. */
typedef struct {
  int nchain;
  const int *qslot; /* [nchain] */
  const int *mu;    /* [nchain] */
  int nsteps;       /* capacity (itermax) */
  int flavor;       /* tdlz_flavor */
  int precision;    /* tdlz_precision */
  int ncomp;        /* left vectors: 3 (spin; also 0) or 4 (spin and charge) */
} tdlz_lanczos_params;

/* Coefficients, caller-owned HOST arrays.  Step j = 0..M-1 stands for the
 * paper's j+1: alpha[j] = alpha_{j+1}, beta[j] = beta_{j+2}, gamma[j] = gamma_{j+2},
 * z[l][j] = z^l_{j+1} = q_{j+1}^H u^l.  chi = w n0 z^H (omega - T)^{-1} e_1. */
typedef struct {
  double *alpha;   /* [nchain][nsteps] complex */
  double *beta;    /* [nchain][nsteps] real    */
  double *gamma;   /* [nchain][nsteps] complex */
  double *z;       /* [nchain][ncomp][nsteps] complex */
  double *n0;      /* [nchain] start-vector norm in the flavour's metric */
  double *wk;      /* [nchain] k weight w */
  int *steps_done; /* [nchain] steps whose alpha and z are valid: a chain that breaks
                      down (TDLZ_ERR_BREAKDOWN: beta of the next step below the
                      tolerance) keeps the step it broke down on; one whose alpha or z
                      came out non-finite (TDLZ_ERR_NUMERIC) ends before that step */
  int *status;     /* [nchain] tdlz_status of each chain; a stopped chain leaves the
                      other chains of the set running */
} tdlz_lanczos_result;

typedef struct {
  int nchain, nsteps;   /* array strides as in tdlz_lanczos_result */
  const int *steps;     /* [nchain] number of coefficients to use (itermax0) */
  const double *alpha, *beta, *gamma, *z, *n0, *wk;
  int ncomp;            /* rows of z per chain: 3 (also 0) or 4; chi has as many */
} tdlz_coeffs;

/* Frequencies start..end step `step` (inclusive), broadening eta; units 0 = Ha,
 * 1 = meV (1 Ha = 27211.386245988 meV).
 * itermax0, itermax, extrapolation: the paper's post-processing options (Sec. 3.3).
 * itermax0 = number of computed coefficients used (0 = all computed steps);
 * extrapolation 0 = none, 1 = constant, 2 = bi-constant ("osc"): coefficients
 * itermax0 .. itermax-1 are the means of the computed ones over the window
 * [itermax0/2, itermax0) (per index parity for the bi-constant form) and z = 0
 * there; the tail is folded into the last computed row by its continued
 * fraction, so itermax may exceed the stored steps at no memory cost.
 * tdlz_spectrum_noalloc supports itermax0 = 0 and extrapolation = 0 only. */
typedef struct {
  double start, end, step, eta;
  int units;
  int itermax0, itermax, extrapolation;
} tdlz_spectrum_params;

/* Create a context on CUDA device `device`.  cuda_stream (a cudaStream_t) may be
 * NULL: the context then makes its own non-blocking stream. */
tdlz_status tdlz_create(tdlz_ctx **out, int device, void *cuda_stream);
void tdlz_destroy(tdlz_ctx *ctx);
const char *tdlz_last_error(const tdlz_ctx *ctx);
tdlz_status tdlz_synchronize(tdlz_ctx *ctx);

/* Upload a ground state (Sec. 3.1) and precompute what the Liouvillian needs
 * (real-space occupied orbitals, kinetic energies, XC kernel table, Hartree
 * factors).  Returns the q-slot id in *qslot.  Rejected: |q| <= 1e-8 (the paper
 * treats q = 0 separately), npw > npwx, spheres that do not fit the FFT box,
 * nocc < 1, non-Hermitian dnl, any non-finite value. */
tdlz_status tdlz_load_ground_state(tdlz_ctx *ctx, const tdlz_ground_state *gs, int *qslot);

/* Number of complex elements of one BR vector of q-slot `qslot` and its npwx. */
tdlz_status tdlz_vec_layout(const tdlz_ctx *ctx, int qslot, int64_t *nelem, int *npwx);

/* y = L x (adjoint = 0) or y = L^H x = J L J x (adjoint = 1), Eq. Liouvillian_BR_q.
 * x, y: caller-owned DEVICE buffers in the BR layout, complex double for
 * TDLZ_FP64 and complex float for TDLZ_MIXED; x and y must not overlap.
 * Enqueued on the context stream (asynchronous). */
tdlz_status tdlz_apply_liouvillian(tdlz_ctx *ctx, int qslot, const void *x, void *y,
                                   int adjoint, int precision);

/* Chains that advance on the device without host round trips; the
 * coefficients stay on the device until tdlz_chain_read. */
tdlz_status tdlz_chain_create(tdlz_ctx *ctx, const tdlz_lanczos_params *p, tdlz_chain **out);
/* Enqueue nsteps steps.  From four steps on, pairs of steps are replayed from a
 * CUDA graph recorded on the context stream at the first such call (the graph is
 * re-recorded when the chain's vector rotation differs from the recorded one);
 * results are identical to eager steps.  The caller must not capture the context
 * stream around this call.  With profiling on, every step runs eagerly. */
tdlz_status tdlz_chain_advance(tdlz_chain *ch, int nsteps);
tdlz_status tdlz_chain_read(tdlz_chain *ch, tdlz_lanczos_result *res); /* synchronises */
void tdlz_chain_destroy(tdlz_chain *ch);

/* Restart (the paper's restart / restart_step, Table of turbo_magnon.x inputs):
 * the chains' full state -- Lanczos vectors, device scalars and the
 * coefficients so far -- as one host image.  tdlz_chain_save synchronises and
 * copies into a caller-owned HOST buffer of tdlz_chain_state_size bytes.
 * tdlz_chain_restore loads an image into a chain set created with the same
 * q-slots, mu, flavour and precision and a capacity (nsteps) >= the saved one;
 * advancing it then continues the recursion exactly where it stopped (FP64 and
 * mixed resumes are bitwise identical to an uninterrupted run). */
tdlz_status tdlz_chain_state_size(tdlz_chain *ch, int64_t *bytes);
tdlz_status tdlz_chain_save(tdlz_chain *ch, void *host_image, int64_t bytes);
tdlz_status tdlz_chain_restore(tdlz_chain *ch, const void *host_image, int64_t bytes);

/* create + advance(nsteps) + read + destroy. */
tdlz_status tdlz_lanczos_run(tdlz_ctx *ctx, const tdlz_lanczos_params *p, tdlz_lanczos_result *res);

/* chi[nchain][ncomp][nomega] (complex double, caller-owned HOST array; ncomp = 3
 * or 4 as in tdlz_coeffs, so row l of chain c is chi_{l, mu_c}) for the
 * frequency grid of sp; FP64 on the GPU, one tridiagonal LU with partial
 * pivoting per (chain, omega).  *nomega receives the grid length; pass
 * chi = NULL to query it. */
tdlz_status tdlz_spectrum(tdlz_ctx *ctx, const tdlz_coeffs *c, const tdlz_spectrum_params *sp,
                          double *chi, int *nomega);

/* ---- allocation-free spectrum (the paper has no counterpart: it concerns the
 * callers of this library, not the method).
 * Same result as tdlz_spectrum, for callers that must not allocate device
 * memory: an application whose device memory is owned entirely by another
 * allocator (a framework's caching pool, or a fixed budget handed out up
 * front), or a latency-bound loop that cannot take the device-wide
 * synchronisation that cudaMalloc / cudaFree imply.  Coefficients and chi are
 * caller-owned DEVICE arrays (layouts as in tdlz_coeffs / tdlz_spectrum,
 * complex double); nomega must equal the grid length (query it with
 * tdlz_spectrum(ctx, c, sp, NULL, &nomega), which allocates nothing).
 * Scratch: one file-scope static device array of TDLZ_NOALLOC_SCRATCH_MB MiB,
 * held by every GPU that loads the library until the process exits; frequencies
 * are processed in chunks that fit it.  Rejected with TDLZ_ERR_ARG (nothing
 * launched): 4 * nchain * nsteps complex rows above the scratch, i.e.
 * nchain * nsteps > TDLZ_NOALLOC_SCRATCH_MB * 2^20 / 64, and grids longer than
 * 2^24 frequencies.  The per-chain step counts dev_coeffs->steps stay on the device,
 * so they are not checked: values outside [0, nsteps] are clamped to that range
 * (tdlz_spectrum, which receives them on the host, rejects them).  The first call on a
 * device looks up the scratch's device address (cudaGetSymbolAddress) and
 * caches it; make that first call before any stream capture.  Every call on a
 * device shares the one array and leaves its contents behind (each call writes
 * every row it reads, so nothing needs clearing); calls whose kernels overlap on
 * the GPU (other streams, other host threads) race on it.  Enqueued on the
 * context stream; no allocation of any kind, no synchronisation. */
#define TDLZ_NOALLOC_SCRATCH_MB 32
tdlz_status tdlz_spectrum_noalloc(tdlz_ctx *ctx, const tdlz_coeffs *dev_coeffs,
                                  const tdlz_spectrum_params *sp, double *dev_chi, int nomega);

/* Neutron-scattering structure factor S(q, omega) = -Im Tr[P_perp(q) chi(q, q; omega)]
 * with P_perp_ab = delta_ab - q_a q_b / q^2 (Eqs. cross_section and S_def, Sec. 2.1).
 * chi: caller-owned HOST array [3][3][nomega] complex double (interleaved re, im),
 * chi[mu][lambda][w] = chi_{lambda mu}(omega_w): the tdlz_spectrum rows of the three
 * chains mu = x, y, z of one q-slot, stacked in that order.
 * q[3]: the transferred momentum (Cartesian; only its direction enters).
 * S: caller-owned HOST array [nomega].  Computed on the context's device;
 * synchronises.  TDLZ_ERR_ARG for NULL pointers, nomega < 1 or q = 0. */
tdlz_status tdlz_structure_factor(tdlz_ctx *ctx, const double *chi, int nomega,
                                  const double *q, double *S);

/* ---- measurement (no counterpart in the paper, whose own numbers are wall
 * times only): per-stage device time from CUDA events recorded on the context
 * stream around each stage, with the stage's algorithmic bytes and flops. */
enum {
  TDLZ_STAGE_SCATTER = 0, TDLZ_STAGE_FFT_INV, TDLZ_STAGE_DENSITY, TDLZ_STAGE_HARTREE,
  TDLZ_STAGE_POTENTIAL, TDLZ_STAGE_PRODUCT, TDLZ_STAGE_FFT_FWD, TDLZ_STAGE_GATHER,
  TDLZ_STAGE_VNL, TDLZ_STAGE_PC, TDLZ_STAGE_LANCZOS, TDLZ_NSTAGE
};
/* enable != 0 starts recording (and clears the accumulators); 0 stops. Synchronises. */
tdlz_status tdlz_profile(tdlz_ctx *ctx, int enable);
/* Accumulated per-stage milliseconds, kernel launches, algorithmic bytes and
 * flops since tdlz_profile(ctx, 1); arrays of TDLZ_NSTAGE (any may be NULL).
 * Synchronises. */
tdlz_status tdlz_profile_read(tdlz_ctx *ctx, double *ms, int64_t *launches, double *bytes,
                              double *flops);
const char *tdlz_stage_name(int stage);
/* Kernels launched by this library in this process so far. */
int64_t tdlz_launch_count(void);

/* Autotuner decisions of this context so far, one "stage/shape=choice (ms)" line per
 * tuned stage and shape (threads per CTA of the register-line FFT passes, vectors per
 * density pass).  Every candidate computes identical results; the first eager call
 * with a new shape times each candidate on the context stream and keeps the fastest
 * (decisions are shared by the contexts of a process on the same device).
 * TDLZ_AUTOTUNE=0 in the environment at tdlz_create keeps the defaults.  Writes at most
 * len bytes including the terminating NUL into the caller's host buffer buf and the
 * full length (without NUL) into *needed (may be NULL).  Host-only, no launch. */
tdlz_status tdlz_autotune_report(tdlz_ctx *ctx, char *buf, int64_t len, int64_t *needed);

#ifdef __cplusplus
}
#endif
#endif /* TDLZ_H */
