// Autotuner for launch shapes that leave the arithmetic unchanged.
//
// A tunable stage offers a few candidate shapes (threads per CTA of the register
// line passes, stacked vectors per thread of the density reduction).  Every candidate
// computes the same outputs bit for bit from the same inputs, so the choice only
// affects time: on the first eager call with a new key (stage + problem shape) each
// candidate runs once, timed with CUDA events on the context stream, and the fastest
// is kept for every later call with that key (and inside captured graphs).  Decisions
// are shared by the contexts of a process on the same device.  While the stream is
// capturing, or with TDLZ_AUTOTUNE=0 at context creation, the default candidate runs.
#pragma once

#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "common.cuh"

namespace tdlz {

struct TunedShape {
  int choice;
  float ms;
};

// decisions of every context of the process, keyed by device and stage/shape
inline std::map<std::string, TunedShape> &tuner_shared() {
  static std::map<std::string, TunedShape> m;
  return m;
}
inline std::mutex &tuner_mutex() {
  static std::mutex m;
  return m;
}

struct Tuner {
  bool on = true;
  int device = 0;
  std::map<std::string, int> choice;
  std::map<std::string, float> best_ms;

  // run(candidate) enqueues the stage on `stream`; returns the candidate used.
  template <class F>
  int pick(cudaStream_t stream, const std::string &key, const std::vector<int> &cands, int dflt,
           F &&run) {
    return pick(stream, key, cands, dflt, run, [] {});
  }
  // For a stage that overwrites its own input: prep() enqueues what recreates that input
  // and runs (untimed) before every timed candidate run, so each candidate sees the
  // same input and the last run leaves the stage's true output.
  template <class F, class P>
  int pick(cudaStream_t stream, const std::string &key, const std::vector<int> &cands, int dflt,
           F &&run, P &&prep) {
    auto it = choice.find(key);
    if (it != choice.end()) {
      run(it->second);
      return it->second;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    TDLZ_CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
    if (!on || cap != cudaStreamCaptureStatusNone || cands.size() < 2) {
      run(dflt);
      return dflt;
    }
    const std::string gkey = std::to_string(device) + ":" + key;
    {
      std::lock_guard<std::mutex> lk(tuner_mutex());
      auto g = tuner_shared().find(gkey);
      if (g != tuner_shared().end()) {
        choice[key] = g->second.choice;
        best_ms[key] = g->second.ms;
        run(g->second.choice);
        return g->second.choice;
      }
    }
    cudaEvent_t e0, e1;
    TDLZ_CUDA_TRY(cudaEventCreate(&e0));
    TDLZ_CUDA_TRY(cudaEventCreate(&e1));
    int best = dflt;
    float tbest = -1.f;
    for (size_t ci = 0; ci < cands.size(); ++ci) {  // each run leaves the same outputs
      const int c = cands[ci];
      if (ci > 0) prep();
      TDLZ_CUDA_TRY(cudaEventRecord(e0, stream));
      run(c);
      TDLZ_CUDA_TRY(cudaEventRecord(e1, stream));
      TDLZ_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      TDLZ_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (tbest < 0.f || ms < tbest) {
        tbest = ms;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    choice[key] = best;
    best_ms[key] = tbest;
    {
      std::lock_guard<std::mutex> lk(tuner_mutex());
      tuner_shared().emplace(gkey, TunedShape{best, tbest});
    }
    return best;
  }

  // "key=choice (ms)" lines of every decision so far
  std::string report() const {
    std::string s;
    for (const auto &kv : choice) {
      char buf[64];
      auto t = best_ms.find(kv.first);
      snprintf(buf, sizeof(buf), "=%d (%.4f ms)\n", kv.second,
               t == best_ms.end() ? 0.0 : (double)t->second);
      s += kv.first + buf;
    }
    return s;
  }
};

}  // namespace tdlz
