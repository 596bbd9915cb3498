// extern "C" entry points of include/tdlz.h.  Every call validates its
// arguments on the host, runs inside a try block and maps failures to a
// tdlz_status with a message for tdlz_last_error(); no C++ exception crosses
// the boundary.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lanczos.cuh"
#include "spectrum.cuh"
#include "tc_gemm.cuh"

using namespace tdlz;

namespace tdlz {
std::atomic<long long> g_launches{0};
}

struct tdlz_ctx {
  Context c;
};
struct tdlz_chain {
  tdlz_ctx *owner;
  ChainSet set;
};

namespace {

tdlz_status fail(tdlz_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->c.last_error = msg;
  return (tdlz_status)code;
}

template <class F>
tdlz_status guarded(tdlz_ctx *ctx, F &&f) {
  if (!ctx) return TDLZ_ERR_ARG;
  try {
    TDLZ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    f();
    ctx->c.last_error.clear();
    return TDLZ_OK;
  } catch (const Error &e) {
    return fail(ctx, e.status, e.msg);
  } catch (const std::bad_alloc &) {
    return fail(ctx, TDLZ_ERR_OOM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(ctx, TDLZ_ERR_STATE, e.what());
  }
}

QSlot &slot_of(tdlz_ctx *ctx, int qslot) {
  TDLZ_REQUIRE(qslot >= 0 && qslot < (int)ctx->c.slots.size() && ctx->c.slots[qslot],
               TDLZ_ERR_ARG, "invalid q-slot");
  return *ctx->c.slots[qslot];
}

}  // namespace

extern "C" {

tdlz_status tdlz_create(tdlz_ctx **out, int device, void *cuda_stream) {
  if (!out) return TDLZ_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    (void)cudaGetLastError();
    return TDLZ_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return TDLZ_ERR_ARG;
  tdlz_ctx *ctx = new (std::nothrow) tdlz_ctx();
  if (!ctx) return TDLZ_ERR_OOM;
  ctx->c.device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return TDLZ_ERR_CUDA;
  }
  // TDLZ_AUTOTUNE=0 keeps every tunable stage at its default launch shape
  const char *at = std::getenv("TDLZ_AUTOTUNE");
  ctx->c.tuner.on = !(at && at[0] == '0');
  ctx->c.tuner.device = device;
  // test hook: TDLZ_TEST_INJECT_TC_TIMEOUT=n makes the next n completed mbarrier waits of
  // the tensor-core GEMMs report expiry (the abort and reporting path, no real timeout)
  if (const char *inj = std::getenv("TDLZ_TEST_INJECT_TC_TIMEOUT")) {
    try {
      tdlz::tc_gemm_inject_timeout(std::atoi(inj));
    } catch (const tdlz::Error &) {
      delete ctx;
      return TDLZ_ERR_CUDA;
    }
  }
  if (cuda_stream) {
    ctx->c.stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->c.stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return TDLZ_ERR_CUDA;
    }
    ctx->c.own_stream = true;
  }
  *out = ctx;
  return TDLZ_OK;
}

void tdlz_destroy(tdlz_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->c.device);
  cudaStreamSynchronize(ctx->c.stream);
  ctx->c.slots.clear();
  if (ctx->c.own_stream) cudaStreamDestroy(ctx->c.stream);
  delete ctx;
}

const char *tdlz_last_error(const tdlz_ctx *ctx) {
  return ctx ? ctx->c.last_error.c_str() : "NULL context";
}

tdlz_status tdlz_profile(tdlz_ctx *ctx, int enable) {
  return guarded(ctx, [&] {
    TDLZ_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
    ctx->c.prof.reset();
    ctx->c.prof.on = enable != 0;
  });
}

tdlz_status tdlz_profile_read(tdlz_ctx *ctx, double *ms, int64_t *launches, double *bytes,
                              double *flops) {
  return guarded(ctx, [&] {
    TDLZ_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
    Profiler &p = ctx->c.prof;
    p.flush();
    for (int i = 0; i < ST_COUNT; ++i) {
      if (ms) ms[i] = p.ms[i];
      if (launches) launches[i] = p.launches[i];
      if (bytes) bytes[i] = p.bytes[i];
      if (flops) flops[i] = p.flops[i];
    }
  });
}

tdlz_status tdlz_spectrum_noalloc(tdlz_ctx *ctx, const tdlz_coeffs *dev_coeffs,
                                  const tdlz_spectrum_params *sp, double *dev_chi, int nomega) {
  return guarded(ctx, [&] { spectrum_noalloc(ctx->c, dev_coeffs, sp, dev_chi, nomega); });
}

tdlz_status tdlz_structure_factor(tdlz_ctx *ctx, const double *chi, int nomega,
                                  const double *q, double *S) {
  return guarded(ctx, [&] {
    TDLZ_REQUIRE(chi && q && S, TDLZ_ERR_ARG, "NULL chi, q or S");
    TDLZ_REQUIRE(nomega >= 1, TDLZ_ERR_ARG, "nomega must be >= 1");
    const double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    TDLZ_REQUIRE(std::isfinite(q2) && q2 > 0, TDLZ_ERR_ARG, "q must be a finite non-zero vector");
    PerpProj p;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) p.m[a][b] = (a == b ? 1.0 : 0.0) - q[a] * q[b] / q2;
    cudaStream_t st = ctx->c.stream;
    DevBuf dchi, dS;
    dchi.alloc((size_t)9 * nomega * sizeof(double2));
    dS.alloc((size_t)nomega * sizeof(double));
    TDLZ_CUDA_TRY(cudaMemcpyAsync(dchi.p, chi, dchi.bytes, cudaMemcpyHostToDevice, st));
    launch_structure_factor(st, dchi.as<double2>(), nomega, p, dS.as<double>());
    TDLZ_CUDA_TRY(cudaMemcpyAsync(S, dS.p, dS.bytes, cudaMemcpyDeviceToHost, st));
    TDLZ_CUDA_TRY(cudaStreamSynchronize(st));
  });
}

const char *tdlz_stage_name(int stage) { return stage_name(stage); }

int64_t tdlz_launch_count(void) { return g_launches.load(); }

tdlz_status tdlz_autotune_report(tdlz_ctx *ctx, char *buf, int64_t len, int64_t *needed) {
  return guarded(ctx, [&] {
    TDLZ_REQUIRE(len >= 0 && (buf || len == 0), TDLZ_ERR_ARG, "NULL buffer with len > 0");
    const std::string r = ctx->c.tuner.report();
    if (needed) *needed = (int64_t)r.size();
    if (len > 0) {
      const size_t n = std::min((size_t)(len - 1), r.size());
      std::memcpy(buf, r.data(), n);
      buf[n] = '\0';
    }
  });
}

tdlz_status tdlz_synchronize(tdlz_ctx *ctx) {
  return guarded(ctx, [&] {
    TDLZ_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
    tc_gemm_check();
  });
}

tdlz_status tdlz_load_ground_state(tdlz_ctx *ctx, const tdlz_ground_state *gs, int *qslot) {
  return guarded(ctx, [&] {
    TDLZ_REQUIRE(qslot != nullptr, TDLZ_ERR_ARG, "qslot output pointer is NULL");
    auto s = std::make_unique<QSlot>();
    load_slot(ctx->c, *s, gs);
    ctx->c.slots.push_back(std::move(s));
    *qslot = (int)ctx->c.slots.size() - 1;
  });
}

tdlz_status tdlz_vec_layout(const tdlz_ctx *cctx, int qslot, int64_t *nelem, int *npwx) {
  tdlz_ctx *ctx = const_cast<tdlz_ctx *>(cctx);
  return guarded(ctx, [&] {
    QSlot &s = slot_of(ctx, qslot);
    if (nelem) *nelem = s.br_elems();
    if (npwx) *npwx = s.npwx;
  });
}

tdlz_status tdlz_apply_liouvillian(tdlz_ctx *ctx, int qslot, const void *x, void *y, int adjoint,
                                   int precision) {
  return guarded(ctx, [&] {
    QSlot &s = slot_of(ctx, qslot);
    TDLZ_REQUIRE(x && y, TDLZ_ERR_ARG, "x and y must be device pointers");
    TDLZ_REQUIRE(precision == TDLZ_FP64 || precision == TDLZ_MIXED, TDLZ_ERR_ARG,
                 "precision must be TDLZ_FP64 or TDLZ_MIXED");
    size_t bytes = (size_t)s.br_elems() * (precision == TDLZ_FP64 ? 16 : 8);
    const char *xa = (const char *)x;
    const char *ya = (const char *)y;
    TDLZ_REQUIRE(xa + bytes <= ya || ya + bytes <= xa, TDLZ_ERR_ARG, "x and y overlap");
    cudaPointerAttributes at{};
    TDLZ_REQUIRE(cudaPointerGetAttributes(&at, x) == cudaSuccess &&
                     (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged),
                 TDLZ_ERR_ARG, "x is not device memory");
    TDLZ_REQUIRE(cudaPointerGetAttributes(&at, y) == cudaSuccess &&
                     (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged),
                 TDLZ_ERR_ARG, "y is not device memory");
    if (precision == TDLZ_FP64)
      apply_liouvillian_caller_order<double>(ctx->c, s, (const double2 *)x, (double2 *)y,
                                             adjoint != 0);
    else
      apply_liouvillian_caller_order<float>(ctx->c, s, (const float2 *)x, (float2 *)y,
                                            adjoint != 0);
  });
}

tdlz_status tdlz_chain_create(tdlz_ctx *ctx, const tdlz_lanczos_params *p, tdlz_chain **out) {
  tdlz_chain *ch = nullptr;
  tdlz_status st = guarded(ctx, [&] {
    TDLZ_REQUIRE(p && out, TDLZ_ERR_ARG, "NULL params or output");
    TDLZ_REQUIRE(p->nchain >= 1 && p->nsteps >= 1, TDLZ_ERR_ARG, "nchain and nsteps must be >= 1");
    TDLZ_REQUIRE(p->ncomp == 0 || p->ncomp == 3 || p->ncomp == 4, TDLZ_ERR_ARG,
                 "ncomp must be 0 or 3 (spin) or 4 (spin and charge)");
    TDLZ_REQUIRE(p->flavor >= 0 && p->flavor <= 2, TDLZ_ERR_ARG, "unknown flavour");
    TDLZ_REQUIRE(p->precision == TDLZ_FP64 || p->precision == TDLZ_MIXED, TDLZ_ERR_ARG,
                 "unknown precision");
    TDLZ_REQUIRE(p->qslot && p->mu, TDLZ_ERR_ARG, "NULL qslot / mu arrays");
    for (int c = 0; c < p->nchain; ++c) {
      slot_of(ctx, p->qslot[c]);
      TDLZ_REQUIRE(p->mu[c] >= 0 && p->mu[c] <= 3, TDLZ_ERR_ARG,
                   "mu must be 0, 1, 2 (spin x, y, z) or 3 (charge)");
      int same = 0;
      for (int d = 0; d < p->nchain; ++d) same += p->qslot[d] == p->qslot[c];
      TDLZ_REQUIRE(same <= (p->flavor == TDLZ_NONHERMITIAN ? 16 : 32), TDLZ_ERR_ARG,
                   "at most 16 NH (32 PH) chains per q-slot in one chain set");
    }
    ch = new tdlz_chain();
    ch->owner = ctx;
    ch->set.ctx = &ctx->c;
    ch->set.flavor = p->flavor;
    ch->set.precision = p->precision;
    ch->set.cap = p->nsteps;
    ch->set.ncomp = p->ncomp == 4 ? 4 : 3;
    // TDLZ_GRAPHS=0 keeps every step eager (A/B timing of the graph replay)
    const char *ge = std::getenv("TDLZ_GRAPHS");
    ch->set.use_graphs = !(ge && ge[0] == '0');
    ch->set.chains.resize(p->nchain);
    for (int c = 0; c < p->nchain; ++c) {
      ch->set.chains[c].qslot = p->qslot[c];
      ch->set.chains[c].mu = p->mu[c];
    }
    ch->set.init();
  });
  if (st != TDLZ_OK) {
    delete ch;
    ch = nullptr;
  }
  if (out) *out = ch;
  return st;
}

tdlz_status tdlz_chain_advance(tdlz_chain *ch, int nsteps) {
  if (!ch) return TDLZ_ERR_ARG;
  return guarded(ch->owner, [&] {
    TDLZ_REQUIRE(nsteps >= 0, TDLZ_ERR_ARG, "nsteps must be >= 0");
    ch->set.advance(nsteps);
  });
}

tdlz_status tdlz_chain_read(tdlz_chain *ch, tdlz_lanczos_result *res) {
  if (!ch) return TDLZ_ERR_ARG;
  return guarded(ch->owner, [&] {
    TDLZ_REQUIRE(res != nullptr, TDLZ_ERR_ARG, "NULL result");
    ch->set.read(res);
  });
}

tdlz_status tdlz_chain_state_size(tdlz_chain *ch, int64_t *bytes) {
  if (!ch) return TDLZ_ERR_ARG;
  return guarded(ch->owner, [&] {
    TDLZ_REQUIRE(bytes != nullptr, TDLZ_ERR_ARG, "NULL output");
    *bytes = (int64_t)ch->set.state_bytes();
  });
}

tdlz_status tdlz_chain_save(tdlz_chain *ch, void *host_image, int64_t bytes) {
  if (!ch) return TDLZ_ERR_ARG;
  return guarded(ch->owner, [&] {
    TDLZ_REQUIRE(host_image != nullptr && bytes > 0, TDLZ_ERR_ARG, "NULL or empty image");
    ch->set.save(host_image, (size_t)bytes);
  });
}

tdlz_status tdlz_chain_restore(tdlz_chain *ch, const void *host_image, int64_t bytes) {
  if (!ch) return TDLZ_ERR_ARG;
  return guarded(ch->owner, [&] {
    TDLZ_REQUIRE(host_image != nullptr && bytes > 0, TDLZ_ERR_ARG, "NULL or empty image");
    ch->set.restore(host_image, (size_t)bytes);
  });
}

void tdlz_chain_destroy(tdlz_chain *ch) {
  if (!ch) return;
  cudaSetDevice(ch->owner->c.device);
  cudaStreamSynchronize(ch->owner->c.stream);
  delete ch;
}

tdlz_status tdlz_lanczos_run(tdlz_ctx *ctx, const tdlz_lanczos_params *p, tdlz_lanczos_result *res) {
  tdlz_chain *ch = nullptr;
  tdlz_status st = tdlz_chain_create(ctx, p, &ch);
  if (st != TDLZ_OK) return st;
  st = tdlz_chain_advance(ch, p->nsteps);
  if (st == TDLZ_OK) st = tdlz_chain_read(ch, res);
  tdlz_chain_destroy(ch);
  return st;
}

tdlz_status tdlz_spectrum(tdlz_ctx *ctx, const tdlz_coeffs *c, const tdlz_spectrum_params *sp,
                          double *chi, int *nomega) {
  return guarded(ctx, [&] {
    TDLZ_REQUIRE(c && sp && nomega, TDLZ_ERR_ARG, "NULL coefficients, parameters or nomega");
    TDLZ_REQUIRE(c->nchain >= 1 && c->nsteps >= 1, TDLZ_ERR_ARG, "empty coefficient set");
    TDLZ_REQUIRE(c->steps && c->alpha && c->beta && c->gamma && c->z && c->n0 && c->wk,
                 TDLZ_ERR_ARG, "NULL coefficient array");
    TDLZ_REQUIRE(c->ncomp == 0 || c->ncomp == 3 || c->ncomp == 4, TDLZ_ERR_ARG,
                 "ncomp must be 0 or 3 (spin) or 4 (spin and charge)");
    TDLZ_REQUIRE(sp->step > 0 && sp->end >= sp->start && std::isfinite(sp->eta) && sp->eta > 0,
                 TDLZ_ERR_ARG, "need step > 0, end >= start and eta > 0");
    TDLZ_REQUIRE(sp->units == 0 || sp->units == 1, TDLZ_ERR_ARG, "units must be 0 (Ha) or 1 (meV)");
    TDLZ_REQUIRE(sp->extrapolation >= 0 && sp->extrapolation <= 2 && sp->itermax0 >= 0,
                 TDLZ_ERR_ARG, "extrapolation must be 0, 1 or 2 and itermax0 >= 0");
    TDLZ_REQUIRE(sp->extrapolation == 0 || (sp->itermax0 >= 2 && sp->itermax >= sp->itermax0),
                 TDLZ_ERR_ARG, "extrapolation needs itermax0 >= 2 and itermax >= itermax0");
    long long nw = (long long)std::floor((sp->end - sp->start) / sp->step + 0.5) + 1;
    TDLZ_REQUIRE(nw >= 1 && nw <= (1 << 24), TDLZ_ERR_ARG, "frequency grid too long");
    *nomega = (int)nw;
    if (!chi) return;
    for (int i = 0; i < c->nchain; ++i)
      TDLZ_REQUIRE(c->steps[i] >= 0 && c->steps[i] <= c->nsteps, TDLZ_ERR_ARG,
                   "steps out of range");
    const double conv = sp->units == 1 ? 1.0 / 27211.386245988 : 1.0;
    const int nc = c->nchain, cap = c->nsteps, nl = c->ncomp == 4 ? 4 : 3;
    DevBuf d_steps, d_al, d_be, d_ga, d_z, d_n0, d_wk, d_chi, d_scr;
    cudaStream_t st = ctx->c.stream;
    auto up = [&](DevBuf &b, const void *src, size_t bytes) {
      b.alloc(bytes);
      TDLZ_CUDA_TRY(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st));
    };
    up(d_steps, c->steps, sizeof(int) * nc);
    up(d_al, c->alpha, sizeof(double2) * nc * cap);
    up(d_be, c->beta, sizeof(double) * nc * cap);
    up(d_ga, c->gamma, sizeof(double2) * nc * cap);
    up(d_z, c->z, sizeof(double2) * nc * nl * cap);
    up(d_n0, c->n0, sizeof(double) * nc);
    up(d_wk, c->wk, sizeof(double) * nc);
    d_chi.alloc(sizeof(double2) * nc * nl * nw);
    d_scr.alloc(sizeof(double2) * 4 * (size_t)cap * nc * nw);
    SpecArgs a{};
    a.nchain = nc;
    a.nomega = (int)nw;
    a.cap = cap;
    a.nl = nl;
    a.steps = d_steps.as<int>();
    a.alpha = d_al.as<double2>();
    a.beta = d_be.as<double>();
    a.gamma = d_ga.as<double2>();
    a.z = d_z.as<double2>();
    a.n0 = d_n0.as<double>();
    a.wk = d_wk.as<double>();
    a.start = sp->start * conv;
    a.step = sp->step * conv;
    a.eta = sp->eta * conv;
    a.scratch = d_scr.as<double2>();
    a.itermax0 = sp->itermax0;
    a.itermax = sp->itermax;
    a.extrap = sp->extrapolation;
    for (int i = 0; i < nc; ++i)
      TDLZ_REQUIRE(sp->itermax0 <= c->steps[i] || sp->itermax0 == 0 || sp->extrapolation == 0,
                   TDLZ_ERR_ARG, "itermax0 exceeds the computed steps of a chain");
    a.chi = d_chi.as<double2>();
    launch_spectrum(st, a);
    TDLZ_CUDA_TRY(cudaMemcpyAsync(chi, d_chi.p, sizeof(double2) * nc * nl * nw,
                                  cudaMemcpyDeviceToHost, st));
    TDLZ_CUDA_TRY(cudaStreamSynchronize(st));
  });
}

}  // extern "C"
