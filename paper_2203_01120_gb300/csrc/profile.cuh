// Per-stage device timing (CUDA events on the context stream) and a
// process-wide count of the library's kernel launches.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <vector>

namespace tdlz {

enum Stage {
  ST_SCATTER = 0,  // sphere -> grid
  ST_FFT_INV,      // 3D FFT, sphere side -> real space
  ST_DENSITY,      // 4-component response density
  ST_HARTREE,      // Hartree solve (2 single-grid FFTs + scaling)
  ST_POTENTIAL,    // ALSDA kernel contraction
  ST_PRODUCT,      // [v_loc + s B.sigma] x + W U
  ST_FFT_FWD,      // 3D FFT, real space -> sphere side
  ST_GATHER,       // grid -> sphere + kinetic - eps
  ST_VNL,          // Kleinman-Bylander projector contractions
  ST_PC,           // conduction projector contractions
  ST_LANCZOS,      // dot products, scalar updates, rescaling
  ST_COUNT
};

inline const char *stage_name(int s) {
  static const char *n[ST_COUNT] = {"scatter", "fft_inv", "density", "hartree", "potential",
                                    "product", "fft_fwd", "gather", "vnl", "pc", "lanczos"};
  return (s >= 0 && s < ST_COUNT) ? n[s] : "?";
}

// NVTX range names of the stages (host-side ranges around each stage's launches, seen
// by an attached profiler; without one the calls return at once)
inline const char *stage_range(int s) {
  static const char *n[ST_COUNT] = {"tdlz/scatter", "tdlz/fft_inv", "tdlz/density",
                                    "tdlz/hartree", "tdlz/potential", "tdlz/product",
                                    "tdlz/fft_fwd", "tdlz/gather", "tdlz/vnl", "tdlz/pc",
                                    "tdlz/lanczos"};
  return (s >= 0 && s < ST_COUNT) ? n[s] : "tdlz/?";
}

// RAII NVTX range on the calling host thread.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

extern std::atomic<long long> g_launches;

struct Profiler {
  struct Rec {
    int stage;
    cudaEvent_t a, b;
    double bytes, flops;
    int launches;
  };
  bool on = false;
  std::vector<Rec> pending;
  double ms[ST_COUNT] = {0}, bytes[ST_COUNT] = {0}, flops[ST_COUNT] = {0};
  long long launches[ST_COUNT] = {0};
  void reset() {
    flush_discard();
    for (int i = 0; i < ST_COUNT; ++i) {
      ms[i] = bytes[i] = flops[i] = 0;
      launches[i] = 0;
    }
  }
  void flush_discard() {
    for (auto &r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    pending.clear();
  }
  // Requires the stream to be synchronised.
  void flush() {
    for (auto &r : pending) {
      float t = 0;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.stage] += t;
      bytes[r.stage] += r.bytes;
      flops[r.stage] += r.flops;
      launches[r.stage] += r.launches;
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    pending.clear();
  }
};

// RAII scope: an NVTX range named after the stage around the enclosed launches, and
// when profiling an event pair on the stream.
struct ProfScope {
  Profiler *p;
  cudaStream_t st;
  Profiler::Rec r;
  long long l0;
  ProfScope(Profiler &prof, cudaStream_t s, int stage, double bytes, double flops)
      : p(prof.on ? &prof : nullptr), st(s) {
    nvtxRangePushA(stage_range(stage));
    l0 = g_launches.load();
    if (!p) return;
    r.stage = stage;
    r.bytes = bytes;
    r.flops = flops;
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, st);
  }
  ~ProfScope() {
    nvtxRangePop();
    if (!p) return;
    cudaEventRecord(r.b, st);
    r.launches = (int)(g_launches.load() - l0);
    p->pending.push_back(r);
  }
};

}  // namespace tdlz
