// Element condensation without any device allocation (mcs_condense_noalloc).
//
// Some callers cannot let the library allocate device memory at call time: applications that
// have handed the whole device to their own memory pool or run under a hard memory budget, and
// code paths that must not block on the allocator (cudaMalloc and cudaFree can synchronise the
// device).  For them this entry point forms the condensed element matrices A_T of a range of
// elements into a buffer the caller owns, using as workspace only a fixed file-scope device array
// that every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "handle.h"

namespace {

// Workspace of the resident blocks: 4 MiB of doubles per device.
constexpr int64_t kScratchDoubles = int64_t(1) << 19;
static __device__ __align__(256) double g_condense_scratch[kScratchDoubles];

// Device address of g_condense_scratch, looked up once per device with that device current.
// In host code the symbol's name is only a host-side stand-in, so kernels receive this address.
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

double* scratch_address(int dev) {
  if (dev < 0 || dev >= kMaxDevices) throw McsError(MCS_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cuda_check(cudaGetSymbolAddress(&p, g_condense_scratch), "cudaGetSymbolAddress");
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  return g_scratch_addr[dev];
}

struct BlockSyncNA {
  __device__ void operator()() const { __syncthreads(); }
};

// Per-block workspace: the element workspace of condense_element, then coordinates and signs.
int64_t slot_doubles(const ElemSizes& s) { return (elem_work_doubles(s) + 24 + 31) / 32 * 32; }

// A_T (full n_A x n_A, FP64, orientation signs applied) of elements T0 .. T0+count-1 into AT.
// Block b works in scratch[b*slot .. (b+1)*slot); every entry it reads there was written
// earlier by the same block for the same element, so nothing has to start at zero.
__global__ void __launch_bounds__(256) k_condense_noalloc(ElemSizes s, DevTables t, DevMesh m, double nu,
                                                          int64_t T0, int64_t count, double* AT, double* scratch,
                                                          int64_t slot) {
  const int lane = threadIdx.x, nl = blockDim.x, d = s.d;
  double* base = scratch + (int64_t)blockIdx.x * slot;
  ElemWork w = elem_work_carve(s, base);
  double* Xs = base + elem_work_doubles(s);
  int* sg = (int*)(Xs + 16);
  ElemTables et{t.B0, t.Rf, t.Bh, t.Ccon, t.Adiv, t.nhat, t.Wmom};
  const int nA2 = s.n_A * s.n_A;
  for (int64_t e = blockIdx.x; e < count; e += gridDim.x) {
    const int64_t T = T0 + e;
    if (lane < (d + 1) * d) {
      int v = lane / d, a = lane % d;
      Xs[lane] = m.coords[(int64_t)m.elems[T * (d + 1) + v] * d + a];
    }
    if (lane <= d) sg[lane] = m.signs[T * (d + 1) + lane];
    __syncthreads();
    condense_element(s, et, Xs, sg, nu, w, lane, nl, BlockSyncNA());
    double* out = AT + e * nA2;
    for (int q = lane; q < nA2; q += nl) out[q] = w.A[q];
    __syncthreads();
  }
}

}  // namespace

extern "C" int mcs_condense_noalloc(mcs_handle* h, int64_t T0, int64_t count, double* AT_out) {
  try {
    if (!h || !AT_out) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    if (T0 < 0 || count < 0 || T0 + count > h->mesh.ne) throw McsError(MCS_ERR_INVALID_ARG, "element range");
    if (h->outflow) throw McsError(MCS_ERR_UNSUPPORTED, "mcs_condense_noalloc with an outflow boundary");
    if (count == 0) return MCS_OK;
    int dev = 0;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != h->device) throw McsError(MCS_ERR_INVALID_ARG, "current device differs from the handle's device");
    const int64_t slot = slot_doubles(h->es);
    if (slot > kScratchDoubles)
      throw McsError(MCS_ERR_UNSUPPORTED, "element workspace (" + std::to_string(slot * 8) +
                                              " bytes) exceeds the 4 MiB static scratch of mcs_condense_noalloc");
    double* scratch = scratch_address(dev);
    int64_t blocks = kScratchDoubles / slot;
    if (blocks > count) blocks = count;
    const int threads = h->d == 2 ? 128 : 256;
    k_condense_noalloc<<<(unsigned)blocks, threads, 0, h->stream>>>(h->es, h->dt, h->dm, h->nu, T0, count, AT_out,
                                                                   scratch, slot);
    note_launch();
    cuda_check(cudaGetLastError(), "k_condense_noalloc");
    return MCS_OK;
  } catch (const McsError& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return MCS_ERR_INVALID_ARG;
  }
}
