// Per-class kernel timing with CUDA events (see prof_begin / prof_end in kernels.h).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.h"

namespace mcs {

struct Profiler {
  struct Rec {
    cudaEvent_t a, b;
    int cls;
    double bytes, flops;
  };
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  std::vector<Rec> recs;
  cudaEvent_t open_ev = nullptr;
  int open_cls = -1;
  double ms[PROF_NCLASS] = {0}, bytes[PROF_NCLASS] = {0}, flops[PROF_NCLASS] = {0};
  int64_t launches[PROF_NCLASS] = {0};

  cudaEvent_t get() {
    if (next == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[next++];
  }
  void begin(int cls, cudaStream_t st) {
    open_ev = get();
    open_cls = cls;
    cudaEventRecord(open_ev, st);
  }
  void end(int cls, double b, double f, cudaStream_t st) {
    if (open_cls != cls || !open_ev) return;
    cudaEvent_t e = get();
    cudaEventRecord(e, st);
    recs.push_back({open_ev, e, cls, b, f});
    open_ev = nullptr;
    open_cls = -1;
  }
  // waits for the recorded events and folds them into the totals
  void collect() {
    if (!recs.empty()) cudaEventSynchronize(recs.back().b);
    for (auto& r : recs) {
      float t = 0;
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.cls] += t;
      bytes[r.cls] += r.bytes;
      flops[r.cls] += r.flops;
      launches[r.cls] += 1;
    }
    recs.clear();
    next = 0;
  }
  void reset() {
    collect();
    for (int c = 0; c < PROF_NCLASS; ++c) ms[c] = bytes[c] = flops[c] = 0, launches[c] = 0;
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace mcs
