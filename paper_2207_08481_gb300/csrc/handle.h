// Internal definition of the libmcs handle (shared by the C-ABI translation units).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mcs.h"
#include "kernels.h"
#include "meshing.h"
#include "profiler.h"
#include "reference.h"

namespace mcs {

struct McsError : std::runtime_error {
  int code;
  McsError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// Records the thread-local message returned by mcs_last_error.
void set_last_error(const char* msg);

inline void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    int code = (e == cudaErrorMemoryAllocation) ? MCS_ERR_OOM : MCS_ERR_CUDA;
    throw McsError(code, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

}  // namespace mcs

using namespace mcs;


struct mcs_handle {
  using McsError = mcs::McsError;
  int d = 0, k = 0;
  double nu = 1.0;
  mcs_options opt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  HostMesh mesh;
  RefTables ref;
  Sizes sz{};
  ElemSizes es{};
  Layout L{};
  double total_adet = 0;
  int ncol = 0;
  std::vector<int32_t> colour;          // per interior rank
  std::vector<int64_t> colour_off;      // host offsets into colour_list
  std::vector<int32_t> fpos;            // interior rank -> position in colour order
  int nlev = 0;
  std::vector<int> level_N;
  int64_t np1 = 0;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  // device data
  DevMesh dm{};
  DevTables dt{};
  KOp K{nullptr, nullptr, nullptr};   // A_T: FP64 (MCS_FP64) or float pairs (MCS_MIXED)
  PrecData<float> pf{};
  PrecData<double> pd{};
  bool condensed = false;
  bool tuned = false;                 // opt.tune: launch shapes chosen (by timing or from the cache)
  std::string tune_cache;             // copy of opt.tune_cache (opt.tune_cache points here or is NULL)
  bool outflow = false;               // Gamma_Ntilde marked (phantom uhat slots, no pressure mean)
  // Krylov work
  double *kv[12] = {nullptr};  // Krylov vectors; kv[10] is the iterate the captured graph updates,
                               // kv[11] the previous iterate of a refinement cycle (error estimate)
  cudaStream_t cap_stream = nullptr;   // non-default stream for graph capture
  cudaGraphExec_t gexec = nullptr;     // two MinRes iterations
  uint64_t graph_kernels = 0;          // kernel nodes of gexec
  bool use_graphs = true;
  double* scratch = nullptr;
  double* ydd = nullptr;            // [4][ndof] double-double row sums of the refinement residual
  MinresScalars* S = nullptr;
  MinresScalars* S_host = nullptr;  // pinned
  double* cond_scratch = nullptr;
  int64_t cond_scratch_doubles = 0;
  std::unique_ptr<Profiler> prof;

  template <class T>
  T* dalloc(int64_t n) {
    if (n <= 0) n = 1;
    void* p = nullptr;
    cuda_check(cudaMalloc(&p, sizeof(T) * n), "cudaMalloc");
    allocs.push_back(p);
    bytes += (int64_t)sizeof(T) * n;
    return (T*)p;
  }
  template <class T>
  T* upload(const std::vector<T>& v) {
    T* p = dalloc<T>((int64_t)v.size());
    if (!v.empty()) cuda_check(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice), "upload");
    return p;
  }
  ~mcs_handle() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (void* p : allocs) cudaFree(p);
    if (S_host) cudaFreeHost(S_host);
  }
};

