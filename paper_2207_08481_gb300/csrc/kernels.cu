// Device kernels of libmcs (sm_103a).  See kernels.h for the roles.
#include <algorithm>
#include <atomic>
#include <cuda_runtime.h>

#include <cstdio>

#include "kernels.h"
#include "profiler.h"

namespace mcs {

#define MCS_WARP 32

// Copy n entries (n * sizeof(R) a multiple of 16, both pointers 16-byte aligned) with 16-byte loads.
template <class R>
__device__ __forceinline__ void vcopy16(R* dst, const R* __restrict__ src, int n, int tid, int nth) {
  const int nv = n * (int)sizeof(R) / 16;
  uint4* d = reinterpret_cast<uint4*>(dst);
  const uint4* sv = reinterpret_cast<const uint4*>(src);
  for (int i = tid; i < nv; i += nth) d[i] = sv[i];
}

// Asynchronous 16-byte global -> shared copies (no register staging; completion by
// cp.async.wait_all, a hardware wait).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
// L2 policy for data read once per pass (element slabs, facet blocks): evict first, so the
// vectors the pass gathers stay resident in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async16_hint(void* smem_dst, const void* gmem_src, uint64_t pol) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem_src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem_dst, const void* gmem_src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem_src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// 1D bulk copy (TMA, cp.async.bulk) global -> shared completing on an mbarrier of this CTA, with an L2
// cache policy; dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                              uint64_t pol) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(d),
      "l"(src), "r"(bytes), "r"(b), "l"(pol)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}
// Waits for the phase `parity` of bar to complete, at most about limit_ns nanoseconds (and at most
// 2^24 polls); false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;   // the common case: no timer read
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

struct WarpSync {
  __device__ void operator()() const { __syncwarp(); }
};

// ============================================================================ condensation
struct BlockSync {
  __device__ void operator()() const { __syncthreads(); }
};

// Condensation of element T by the whole block (a1-a4 except D_F), workspace at base.
// LO: 0 = k >= 2, 1 = lowest-order variant, -1 = decided per element from s.lowest.
template <class R, int LO>
__device__ __forceinline__ void condense_one(const ElemSizes& s, const DevTables& t, const DevMesh& m, double nu,
                                             const KOp& K, R* Fs, R* G, R* Aoi, double* base, int64_t T) {
  const int lane = threadIdx.x, nl = blockDim.x;
  // slot layout: coordinates and signs (24 doubles), then the element workspace; the bubble
  // condensation's work and staging reuse the rows of Bt and Ct, which are dead once A_T is formed
  double* Xs = base;                                       // (d+1)*d coords
  int* sg = (int*)(Xs + 16);
  ElemWork w = elem_work_carve(s, base + 24);
  double* bw = w.Bt;                                       // bubble work
  double* Adt = bw + s.n_bub * s.n_bub + s.n_bub * s.n_c;  // staging (FP64)
  double* Gt = Adt + s.n_c * s.n_c;
  double* Ait = Gt + s.n_bub * s.n_c;
  ElemTables et{t.B0, t.Rf, t.Bh, t.Ccon, t.Adiv, t.nhat, t.Wmom};
  const int d = s.d;
  if (lane < (d + 1) * d) {
    int v = lane / d, a = lane % d;
    Xs[lane] = m.coords[(int64_t)m.elems[T * (d + 1) + v] * d + a];
  }
  if (lane <= d) sg[lane] = m.signs[T * (d + 1) + lane];
  __syncthreads();
  if constexpr (LO == 0) condense_element_t<false>(s, et, Xs, sg, nu, w, lane, nl, BlockSync());
  else if constexpr (LO == 1) condense_element_t<true>(s, et, Xs, sg, nu, w, lane, nl, BlockSync());
  else condense_element(s, et, Xs, sg, nu, w, lane, nl, BlockSync());
  const int nA = s.n_A;
  if (m.fout) {
    // uhat of an outflow facet is 0 (Gamma_Ntilde): its slots are phantom dofs, rows and columns of
    // the identity (the facet has this one element, so the assembled diagonal is 1)
    bool out[4] = {false, false, false, false};
    for (int f = 0; f <= d; ++f) {
      const int32_t rk = m.elem_rank[T * (d + 1) + f];
      out[f] = rk >= 0 && m.fout[rk] != 0;
    }
    if (out[0] || out[1] || out[2] || out[3]) {
      for (int q = lane; q < nA * nA; q += nl) {
        const int i = q / nA, j = q - i * nA;
        const bool pi = i >= s.n_u && out[(i - s.n_u) / s.nhF], pj = j >= s.n_u && out[(j - s.n_u) / s.nhF];
        if (pi || pj) w.A[q] = (i == j) ? 1.0 : 0.0;
      }
      __syncthreads();
    }
  }
  if (K.AT) {  // full A_T (FP64, symmetric: row-major = column-major)
    double* out = K.AT + T * (int64_t)nA * nA;
    for (int q = lane; q < nA * nA; q += nl) out[q] = w.A[q];
  }
  if (K.Ahi) {  // packed lower triangle as float pairs, hi = fl(a), lo = fl(a - hi)
    const int pp = packed_pad(s);
    float* oh = K.Ahi + T * (int64_t)pp;
    float* ol = K.Alo + T * (int64_t)pp;
    for (int i = lane; i < nA; i += nl)
      for (int j = 0; j <= i; ++j) {
        const double a = w.A[i * nA + j];
        const float hi = (float)a;
        oh[i * (i + 1) / 2 + j] = hi;
        ol[i * (i + 1) / 2 + j] = (float)(a - (double)hi);
      }
  }
  __syncthreads();
  bubble_condense(s, w.A, bw, Adt, Gt, Ait, lane, nl, BlockSync());
  const int nc = s.n_c, no = s.n_bub, mF = s.mF, fss = fs_stride(s), slab = slab_pad(s);
  // slabs of the interior facets into the facet stream (boundary facets carry no dofs)
  for (int q = lane; q < nc * nc; q += nl) {   // q = (f*nc + c)*mF + tt: contiguous slab writes
    const int f = q / (nc * mF), rem = q - f * nc * mF, c = rem / mF, tt = rem - c * mF;
    const int i = f * mF + tt;                 // row of A^d_T
    const int32_t rk = m.elem_rank[T * (d + 1) + f];
    if (rk < 0) continue;
    const int side = m.fel[2 * (int64_t)rk] == (int32_t)T ? 0 : 1;
    Fs[(int64_t)m.fpos[rk] * fss + side * slab + c * mF + tt] = (R)Adt[i * nc + c];
  }
  for (int q = lane; q < no * nc; q += nl) G[T * g_stride(s) + q] = (R)Gt[q];
  for (int q = lane; q < no * no; q += nl) Aoi[T * a_stride(s) + q] = (R)Ait[q];
  __syncthreads();
}

// One thread block per element (grid-stride).  Workspace in dynamic shared memory when
// it fits, else in a global scratch slot per resident block.
template <class R, bool SMEM, int LO>
__global__ void __launch_bounds__(256, 2) k_condense(ElemSizes s, DevTables t, DevMesh m, double nu, KOp K, R* Fs,
                                                  R* G, R* Aoi, double* gscratch, int64_t slot_doubles) {
  extern __shared__ double smem[];
  double* base = SMEM ? smem : gscratch + (int64_t)blockIdx.x * slot_doubles;
  for (int64_t T = blockIdx.x; T < m.ne; T += gridDim.x) condense_one<R, LO>(s, t, m, nu, K, Fs, G, Aoi, base, T);
}

// Several problems (any d, k) in one persistent launch: the blocks walk the concatenated element
// lists (problem p owns the global indices first[p] .. first[p+1]-1) with a grid stride, so costly
// and cheap elements interleave.  Workspace: a global scratch slot per block, sized for the
// largest element.
template <class R>
__global__ void __launch_bounds__(256) k_condense_batch(const CondenseItem<R>* __restrict__ items, int nitems,
                                                        int64_t total, double* gscratch, int64_t slot_doubles) {
  double* base = gscratch + (int64_t)blockIdx.x * slot_doubles;
  int p = 0;
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    while (p + 1 < nitems && items[p + 1].first <= g) ++p;   // g increases: the problem index only grows
    const CondenseItem<R>& it = items[p];
    condense_one<R, -1>(it.s, it.t, it.m, it.nu, it.K, it.Fs, it.G, it.Aoi, base, g - it.first);
  }
}

// Doubles of the bubble condensation's work and staging, which condense_one places over the rows of
// Bt and Ct ((n_A + n_cc) * raw_stride doubles); the host checks that they fit there.
static int64_t bubble_doubles(const ElemSizes& s) {
  return 2 * (int64_t)s.n_bub * s.n_bub + 2 * (int64_t)s.n_bub * s.n_c + (int64_t)s.n_c * s.n_c;
}
static bool bubble_fits(const ElemSizes& s) {
  return bubble_doubles(s) <= (int64_t)(s.n_A + s.n_cc) * raw_stride(s);
}
static int64_t condense_slot_doubles(const ElemSizes& s) {
  const int64_t v = 24 + elem_work_doubles(s);
  return (v + 31) / 32 * 32;
}

static int condense_threads(const ElemSizes& s) { return s.d == 2 ? 128 : 256; }

template <class R, int LO>
static cudaError_t launch_condense_t(const ElemSizes& s, const DevTables& t, const DevMesh& m, double nu, KOp K,
                                     R* Fs, R* G, R* Aoi, double* scratch, int64_t scratch_doubles, cudaStream_t st);

template <class R>
cudaError_t launch_condense(const ElemSizes& s, const DevTables& t, const DevMesh& m, double nu, KOp K, R* Fs,
                            R* G, R* Aoi, double* scratch, int64_t scratch_doubles, cudaStream_t st) {
  return s.lowest ? launch_condense_t<R, 1>(s, t, m, nu, K, Fs, G, Aoi, scratch, scratch_doubles, st)
                  : launch_condense_t<R, 0>(s, t, m, nu, K, Fs, G, Aoi, scratch, scratch_doubles, st);
}

template <class R, int LO>
static cudaError_t launch_condense_t(const ElemSizes& s, const DevTables& t, const DevMesh& m, double nu, KOp K,
                                     R* Fs, R* G, R* Aoi, double* scratch, int64_t scratch_doubles, cudaStream_t st) {
  const int64_t slot = condense_slot_doubles(s);
  if (!bubble_fits(s)) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int threads = condense_threads(s);
  const int64_t bytes = slot * 8;
  prof_begin(PROF_CONDENSE, st);
  if (bytes <= maxsm) {
    size_t sm = (size_t)bytes;
    // the opt-in maximum, never lowered: other threads may launch this kernel with other sizes
    cudaFuncSetAttribute(k_condense<R, true, LO>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_condense<R, true, LO>, threads, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)nsm * per_sm;
    if (blocks > m.ne) blocks = m.ne;
    k_condense<R, true, LO><<<(unsigned)blocks, threads, sm, st>>>(s, t, m, nu, K, Fs, G, Aoi, nullptr, slot);
    note_launch();
  } else {
    int64_t blocks = scratch_doubles / slot;
    if (blocks < 1) return cudaErrorMemoryAllocation;
    if (blocks > m.ne) blocks = m.ne;
    k_condense<R, false, LO><<<(unsigned)blocks, threads, 0, st>>>(s, t, m, nu, K, Fs, G, Aoi, scratch, slot);
    note_launch();
  }
  {
    // FP64 flops of the element condensation (products and factorisations, see element.cuh)
    const double nA = s.n_A, nr = s.n_raw, nc = s.n_cc, no = s.n_bub, ncp = s.n_c;
    const double f = 2.0 * (nA * (nA + 1) / 2 * nr + nc * nA * nr + nc * (nc + 1) / 2 * nr + nc * nc * nc / 6 +
                            nc * nc * nA / 2 + nA * (nA + 1) / 2 * nc + no * no * no / 6 + no * no * ncp +
                            ncp * ncp * no + no * no * no) +
                     2.0 * nA * nr * s.n_s0;
    const double out = (double)m.ne * ((K.AT ? nA * nA * 8 : 0.0) + (K.Ahi ? 8.0 * packed_pad(s) : 0.0) +
                                       (double)(g_stride(s) + a_stride(s)) * sizeof(R)) +
                       (double)m.nint * 2.0 * slab_pad(s) * sizeof(R);
    prof_end(PROF_CONDENSE, out, f * (double)m.ne, st);
  }
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_condense_batch(const CondenseItem<R>* items_dev, const CondenseItem<R>* items_host, int nitems,
                                  double* scratch, int64_t scratch_doubles, cudaStream_t st) {
  int64_t slot = 0, total = 0;
  for (int i = 0; i < nitems; ++i) {
    if (!bubble_fits(items_host[i].s)) return cudaErrorInvalidValue;
    slot = std::max<int64_t>(slot, condense_slot_doubles(items_host[i].s));
    total += items_host[i].m.ne;
  }
  if (total == 0) return cudaSuccess;
  int64_t blocks = scratch_doubles / slot;
  if (blocks < 1) return cudaErrorMemoryAllocation;
  if (blocks > total) blocks = total;
  prof_begin(PROF_CONDENSE, st);
  k_condense_batch<R><<<(unsigned)blocks, 256, 0, st>>>(items_dev, nitems, total, scratch, slot);
  note_launch();
  prof_end(PROF_CONDENSE, 0.0, 0.0, st);
  return cudaGetLastError();
}
template cudaError_t launch_condense_batch<float>(const CondenseItem<float>*, const CondenseItem<float>*, int,
                                                  double*, int64_t, cudaStream_t);
template cudaError_t launch_condense_batch<double>(const CondenseItem<double>*, const CondenseItem<double>*, int,
                                                   double*, int64_t, cudaStream_t);
int64_t condense_slot_bytes(const ElemSizes& s) { return condense_slot_doubles(s) * 8; }

// Global workspace of the condensation when one element's does not fit in shared memory: a slot per
// resident block, up to 8 blocks per SM, fewer where that would exceed 2 GiB (3D k = 5, 6: 2.8 and
// 6 MB per element).
int64_t condense_scratch_doubles(const ElemSizes& s, int nsm) {
  const int64_t slot = condense_slot_doubles(s);
  int64_t per_sm = 8;
  while (per_sm > 1 && slot * nsm * per_sm * 8 > (int64_t(2) << 30)) --per_sm;
  return slot * (int64_t)nsm * per_sm;
}

// ---------------------------------------------------------------- facet blocks
template <class R>
__global__ void k_facet_blocks(ElemSizes s, DevMesh m, R* Fs) {
  extern __shared__ double sm2[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int mF = s.mF;
  double* A = sm2 + (int64_t)wib * 2 * mF * mF;
  double* I = A + mF * mF;
  for (int64_t r = (int64_t)blockIdx.x * wpb + wib; r < m.nint; r += (int64_t)gridDim.x * wpb) {
    for (int q = lane; q < mF * mF; q += 32) {
      int i = q / mF, j = q % mF;
      double v = 0;
      const R* blk = Fs + (int64_t)m.fpos[r] * fs_stride(s);
      for (int side = 0; side < 2; ++side) {
        const int f = m.floc[r * 2 + side];
        v += (double)blk[side * slab_pad(s) + (f * mF + j) * mF + i];
      }
      A[q] = v;
      I[q] = (i == j) ? 1.0 : 0.0;
    }
    __syncwarp();
    // Gauss-Jordan (SPD: no pivoting needed)
    for (int c = 0; c < mF; ++c) {
      double piv = A[c * mF + c];
      __syncwarp();
      for (int j = lane; j < mF; j += 32) {
        A[c * mF + j] /= piv;
        I[c * mF + j] /= piv;
      }
      __syncwarp();
      for (int q = lane; q < mF * mF; q += 32) {
        int rr = q / mF, j = q % mF;
        if (rr == c) continue;
        double f = A[rr * mF + c];
        I[q] -= f * I[c * mF + j];
      }
      __syncwarp();
      for (int q = lane; q < mF * mF; q += 32) {
        int rr = q / mF, j = q % mF;
        if (rr == c || j == c) continue;
        A[q] -= A[rr * mF + c] * A[c * mF + j];
      }
      __syncwarp();
      for (int rr = lane; rr < mF; rr += 32)
        if (rr != c) A[rr * mF + c] = 0.0;
      __syncwarp();
    }
    R* Dinv = Fs + (int64_t)m.fpos[r] * fs_stride(s) + 2 * slab_pad(s);
    for (int q = lane; q < mF * mF; q += 32) Dinv[q] = (R)(0.5 * (I[q] + I[(q % mF) * mF + q / mF]));
    __syncwarp();
  }
}

template <class R>
cudaError_t launch_facet_blocks(const ElemSizes& s, const DevMesh& m, R* Fs, cudaStream_t st) {
  if (m.nint == 0) return cudaSuccess;
  int wpb = 4;   // warps per block, each with two m_F x m_F FP64 work matrices (fewer for large m_F)
  while (wpb > 1 && (size_t)wpb * 2 * s.mF * s.mF * sizeof(double) > 200 * 1024) --wpb;
  size_t sm = (size_t)wpb * 2 * s.mF * s.mF * sizeof(double);
  cudaFuncSetAttribute(k_facet_blocks<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  int64_t blocks = (m.nint + wpb - 1) / wpb;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  prof_begin(PROF_FACET_BLOCKS, st);
  k_facet_blocks<R><<<(unsigned)blocks, wpb * 32, sm, st>>>(s, m, Fs);
  note_launch();
  prof_end(PROF_FACET_BLOCKS, (double)m.nint * (2.0 * s.mF * s.mF + s.mF * s.mF) * sizeof(R), 0.0, st);
  return cudaGetLastError();
}

// ============================================================================ K apply (FP64)
template <class S>
__device__ __forceinline__ int64_t local_to_global(const S& s, const Layout& L, const int32_t* er, int64_t T, int i) {
  // local A index (u_d (f, j) | u_o | uhat (f, t)) -> global index, -1 if on a Dirichlet facet
  const int nfd = (s.d + 1) * s.nF;
  if (i < nfd) {
    int f = i / s.nF;
    int32_t rk = er[f];
    return rk < 0 ? -1 : (int64_t)rk * s.nF + (i - f * s.nF);
  }
  if (i < s.n_u) return L.off_o + T * s.n_bub + (i - nfd);
  int q = i - s.n_u, f = q / s.nhF;
  int32_t rk = er[f];
  return rk < 0 ? -1 : L.off_h + (int64_t)rk * s.nhF + (q - f * s.nhF);
}

// y = K x element by element: the blocks A_T of EB elements are staged in shared memory with
// coalesced loads (full symmetric storage), then one thread per row forms the product.  When
// one block does not fit in shared memory (3D, k = 4) STAGED is false and the rows are read
// from global memory directly (thread i reads column entries i of consecutive rows: coalesced).
template <class S, bool STAGED>
__global__ void __launch_bounds__(256) k_apply_K(S s, DevTables t, DevMesh m, Layout L,
                                                 const double* __restrict__ AT, const double* __restrict__ x,
                                                 double* y, int EB, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ double sk[];
  const int nA = s.n_A, np_ = s.n_p, nu_ = s.n_u, d = s.d, nfd = (s.d + 1) * s.nF;
  const int per = nA + np_, nA2 = nA * nA;
  const int64_t Tb = (int64_t)blockIdx.x * EB;
  const double* As = STAGED ? sk : AT + Tb * nA2;   // [EB][nA*nA]
  double* xs = STAGED ? sk + EB * nA2 : sk;           // [EB][nA + np]
  int* er = (int*)(xs + EB * per);   // [EB][4]
  float* sg = (float*)(er + EB * 4); // [EB][4]
  const int tid = threadIdx.x;
  const int64_t T0 = (int64_t)blockIdx.x * EB;
  const int nvalid = (int)((m.ne - T0) < EB ? (m.ne - T0) : EB);
  if (tid < EB * 4) {
    int e = tid >> 2, f = tid & 3;
    int64_t T = T0 + e;
    bool ok = e < nvalid && f <= d;
    er[tid] = ok ? m.elem_rank[T * (d + 1) + f] : -1;
    sg[tid] = ok ? (float)m.signs[T * (d + 1) + f] : 0.f;
  }
  if (STAGED) {
    const double2* src = reinterpret_cast<const double2*>(AT + T0 * nA2);
    double2* dst = reinterpret_cast<double2*>(sk);
    const int cnt = nvalid * nA2;
    if ((nA2 & 1) == 0) {
      for (int q = tid; q < cnt / 2; q += blockDim.x) dst[q] = src[q];
    } else {
      for (int q = tid; q < cnt; q += blockDim.x) sk[q] = AT[T0 * nA2 + q];
    }
  }
  __syncthreads();
  for (int q = tid; q < nvalid * per; q += blockDim.x) {
    const int e = q / per, i = q - e * per;
    const int64_t T = T0 + e;
    double v;
    if (i < nA) {
      int64_t g = local_to_global(s, L, er + e * 4, T, i);
      v = g < 0 ? 0.0 : x[g];
    } else {
      v = x[L.off_p + T * np_ + (i - nA)];
    }
    xs[q] = v;
  }
  __syncthreads();
  // the n_A rows of every element first, then the n_p pressure rows (warps do not mix the two kinds)
  for (int q = tid; q < nvalid * per; q += blockDim.x) {
    int e, i;
    if (q < nvalid * nA) {
      e = q / nA;
      i = q - e * nA;
    } else {
      const int qq = q - nvalid * nA;
      e = qq / np_;
      i = nA + (qq - e * np_);
    }
    const int64_t T = T0 + e;
    const double* xe = xs + e * per;
    if (i < nA) {
      const double* A = As + e * nA2 + i;
      double v0 = 0.0, v1 = 0.0;
      int j = 0;
#pragma unroll 8
      for (; j + 1 < nA; j += 2) {
        v0 += A[j * nA] * xe[j];
        v1 += A[(j + 1) * nA] * xe[j + 1];
      }
      if (j < nA) v0 += A[j * nA] * xe[j];
      double v = v0 + v1;
      if (i < nu_) {
        double sgn = i < nfd ? (double)sg[e * 4 + i / s.nF] : 1.0;
        double bt = 0.0;
        for (int p = 0; p < np_; ++p) bt += t.Bp[p * nu_ + i] * xe[nA + p];
        v -= sgn * bt;
      }
      int64_t g = local_to_global(s, L, er + e * 4, T, i);
      if (g < 0) continue;
      if (i >= nfd && i < nu_) y[g] = v;     // bubble: owned by T
      else atomicAdd(&y[g], v);             // facet dof: exactly two contributions into 0
    } else {
      const int jp = i - nA;
      double v = 0.0;
      for (int c = 0; c < nu_; ++c) {
        double sgn = c < nfd ? (double)sg[e * 4 + c / s.nF] : 1.0;
        v += t.Bp[jp * nu_ + c] * sgn * xe[c];
      }
      y[L.off_p + T * np_ + jp] = -v;
    }
  }
}

// Double-float helpers (Dekker / Knuth error-free transformations): the product of two floats
// is split exactly into p + e with one fma; sums are accumulated with TwoSum.
struct DF {
  float hi, lo, c;  // value hi + lo, plus first-order corrections c
};
__device__ __forceinline__ void df_mac(DF& a, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  const float e = __fmaf_rn(xh, yh, -p);
  const float s = __fadd_rn(a.hi, p);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(err, e));
  a.c = __fmaf_rn(xh, yl, a.c);
  a.c = __fmaf_rn(xl, yh, a.c);
}
// The conversions between double and float pairs with integer operations on the IEEE bit patterns, so
// that the apply spends no FP64-pipe instruction on them (FP64 runs at a small fraction of the FP32 rate
// on this GPU).  Values outside the range the bit manipulation covers take the conversion instructions.
// float -> double, exact.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if ((u << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32));
  if (ex == 0u || ex == 255u) return (double)f;   // subnormal, inf, nan
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                          ((unsigned long long)(ex + 896u) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// v = h + l with h the significand of v rounded to 24 bits (to nearest, ties away from zero) and l the
// remainder rounded to float: |v - h - l| <= 2^-48 |v|.
__device__ __forceinline__ void split_ff(double v, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ffull);
  if ((b << 1) == 0ull) {   // +-0
    h = l = __uint_as_float((unsigned)(b >> 32));
    return;
  }
  if (ex < 949 || ex > 1149) {   // h or the scale of l would leave the normal float range
    h = (float)v;
    l = (float)(v - (double)h);
    return;
  }
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long m = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;   // 53-bit significand
  unsigned long long mh = (m + 0x10000000ull) >> 29;                                 // 24 bits, rounded
  const int r = (int)((long long)m - (long long)(mh << 29));                         // |r| <= 2^28, exact
  int eh = ex;
  if (mh == 0x1000000ull) {   // rounded up into the next binade
    mh = 0x800000ull;
    ++eh;
  }
  h = __uint_as_float(sgn | ((unsigned)(eh - 896) << 23) | (unsigned)(mh & 0x7fffffull));
  const float scale = __uint_as_float((unsigned)(ex - 948) << 23);   // 2^(ex - 1075)
  const float lr = (float)r * scale;
  l = sgn ? -lr : lr;
}
// hi + (lo + c) as a double: lo + c rounded in FP32 (both are O(2^-24) of hi), then one FP64 add.
__device__ __forceinline__ double df_value(const DF& a) { return f2d_bits(a.hi) + f2d_bits(__fadd_rn(a.lo, a.c)); }

// y = K x with A_T as packed-lower float pairs and double-float arithmetic (mixed form).  The block
// stages the pairs of EB elements with hi and lo of each entry side by side (one 8-byte shared load per
// entry), and x split into float pairs the same way.
template <class S>
__global__ void __launch_bounds__(256) k_apply_K_df(S s, DevTables t, DevMesh m, Layout L,
                                                    const float* __restrict__ Ahi, const float* __restrict__ Alo,
                                                    const double* __restrict__ x, double* y, int EB, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) float skf[];
  const int nA = s.n_A, np_ = s.n_p, nu_ = s.n_u, d = s.d, nfd = (s.d + 1) * s.nF;
  const int per = nA + np_, pp = packed_pad(s);
  float2* Ap = reinterpret_cast<float2*>(skf);    // [EB][pp] (hi, lo)
  float2* Xp = Ap + (size_t)EB * pp;              // [EB][per] (hi, lo)
  int* er = reinterpret_cast<int*>(Xp + (size_t)EB * per);   // [EB][4]
  float* sg = reinterpret_cast<float*>(er + EB * 4);         // [EB][4]
  const int tid = threadIdx.x;
  const int64_t T0 = (int64_t)blockIdx.x * EB;
  const int nvalid = (int)((m.ne - T0) < EB ? (m.ne - T0) : EB);
  if (tid < EB * 4) {
    int e = tid >> 2, f = tid & 3;
    int64_t T = T0 + e;
    bool ok = e < nvalid && f <= d;
    er[tid] = ok ? m.elem_rank[T * (d + 1) + f] : -1;
    sg[tid] = ok ? (float)m.signs[T * (d + 1) + f] : 0.f;
  }
  {
    // the block's elements are contiguous in Ahi / Alo; pp is a multiple of 4 (16-byte chunks)
    const float4* hs = reinterpret_cast<const float4*>(Ahi + T0 * pp);
    const float4* ls = reinterpret_cast<const float4*>(Alo + T0 * pp);
    float4* dst = reinterpret_cast<float4*>(Ap);
    const int nq = nvalid * pp / 4;
    for (int q = tid; q < nq; q += blockDim.x) {
      const float4 h = __ldg(hs + q), l = __ldg(ls + q);
      dst[2 * q] = make_float4(h.x, l.x, h.y, l.y);
      dst[2 * q + 1] = make_float4(h.z, l.z, h.w, l.w);
    }
  }
  __syncthreads();
  for (int q = tid; q < nvalid * per; q += blockDim.x) {
    const int e = q / per, i = q - e * per;
    const int64_t T = T0 + e;
    double v;
    if (i < nA) {
      int64_t g = local_to_global(s, L, er + e * 4, T, i);
      v = g < 0 ? 0.0 : x[g];
    } else {
      v = x[L.off_p + T * np_ + (i - nA)];
    }
    float h, l;
    split_ff(v, h, l);
    Xp[q] = make_float2(h, l);
  }
  __syncthreads();
  // threads take the n_A rows of every element first, then the n_p pressure rows of every element, so
  // that the warps do not mix the two kinds of rows
  for (int q = tid; q < nvalid * per; q += blockDim.x) {
    int e, i;
    if (q < nvalid * nA) {
      e = q / nA;
      i = q - e * nA;
    } else {
      const int qq = q - nvalid * nA;
      e = qq / np_;
      i = nA + (qq - e * np_);
    }
    const int64_t T = T0 + e;
    const float2* xe = Xp + (size_t)e * per;
    DF acc{0.f, 0.f, 0.f};
    if (i < nA) {
      const float2* ap = Ap + (size_t)e * pp;
      // one loop over the row, the packed index chosen per entry (row part j <= i, column part
      // j > i), so the lanes of a warp, which hold rows of different lengths, do not diverge
      const int row = i * (i + 1) / 2;
      int colidx = row + i;               // j(j+1)/2 + i for j = i
#pragma unroll 4
      for (int j = 0; j < nA; ++j) {
        const int idx = j <= i ? row + j : colidx;
        const float2 a = ap[idx], xv = xe[j];
        df_mac(acc, a.x, a.y, xv.x, xv.y);
        if (j >= i) colidx += j + 1;      // next: (j+1)(j+2)/2 + i
      }
      if (i < nu_) {  // (B^T x_p)_i = -s_i sum_j Bhat[j][i] x_p[j]
        const float sgn = i < nfd ? sg[e * 4 + i / s.nF] : 1.f;
        for (int p = 0; p < np_; ++p) {
          const float2 xv = xe[nA + p];
          df_mac(acc, -sgn * t.Bp_hi[p * nu_ + i], -sgn * t.Bp_lo[p * nu_ + i], xv.x, xv.y);
        }
      }
      const double v = df_value(acc);
      int64_t g = local_to_global(s, L, er + e * 4, T, i);
      if (g < 0) continue;
      if (i >= nfd && i < nu_) y[g] = v;     // bubble: owned by T
      else atomicAdd(&y[g], v);             // facet dof: exactly two contributions into 0
    } else {
      const int jp = i - nA;
      for (int c = 0; c < nu_; ++c) {
        const float sgn = c < nfd ? sg[e * 4 + c / s.nF] : 1.f;
        const float2 xv = xe[c];
        df_mac(acc, -sgn * t.Bp_hi[jp * nu_ + c], -sgn * t.Bp_lo[jp * nu_ + c], xv.x, xv.y);
      }
      y[L.off_p + T * np_ + jp] = df_value(acc);
    }
  }
}

// The double-float apply for elements whose packed pairs do not fit in shared memory (3D k >= 5): one
// block per element, the packed lower triangle streamed through shared memory in chunks of whole
// rows [r0, r1) (one contiguous range of the packed storage each); a thread owns rows i = tid + 256 m
// and adds, per chunk, the row part A_ij x_j (j <= i, i in the chunk) and the column part A_ji x_j
// (j in the chunk, j > i).  The same products as k_apply_K_df, summed in another order.
template <int MAXR>
__global__ void __launch_bounds__(256) k_apply_K_df_chunk(ElemSizes s, DevTables t, DevMesh m, Layout L,
                                                          const float* __restrict__ Ahi,
                                                          const float* __restrict__ Alo,
                                                          const double* __restrict__ x, double* y, int chunk,
                                                          const int* stop) {
  if (stop && *stop) return;
  extern __shared__ float skc[];
  const int nA = s.n_A, np_ = s.n_p, nu_ = s.n_u, d = s.d, nfd = (s.d + 1) * s.nF;
  const int per = nA + np_, pp = packed_pad(s);
  float* ch = skc;                   // [chunk] hi
  float* cl = ch + chunk;            // [chunk] lo
  float* xh = cl + chunk;            // [per]
  float* xl = xh + per;              // [per]
  int* er = (int*)(xl + per);        // [4]
  float* sg = (float*)(er + 4);      // [4]
  const int tid = threadIdx.x;
  for (int64_t T = blockIdx.x; T < m.ne; T += gridDim.x) {
    if (tid < 4) {
      er[tid] = tid <= d ? m.elem_rank[T * (d + 1) + tid] : -1;
      sg[tid] = tid <= d ? (float)m.signs[T * (d + 1) + tid] : 0.f;
    }
    __syncthreads();
    for (int q = tid; q < per; q += blockDim.x) {
      double v;
      if (q < nA) {
        const int64_t g = local_to_global(s, L, er, T, q);
        v = g < 0 ? 0.0 : x[g];
      } else {
        v = x[L.off_p + T * np_ + (q - nA)];
      }
      float h, l;
      split_ff(v, h, l);
      xh[q] = h;
      xl[q] = l;
    }
    DF acc[MAXR];
#pragma unroll
    for (int u = 0; u < MAXR; ++u) acc[u] = DF{0.f, 0.f, 0.f};
    const float* Ah = Ahi + T * (int64_t)pp;
    const float* Al = Alo + T * (int64_t)pp;
    int r0 = 0;
    while (r0 < nA) {
      int r1 = r0 + 1;   // rows [r0, r1) with at most `chunk` packed entries (one row always fits)
      while (r1 < nA && (r1 + 1) * (r1 + 2) / 2 - r0 * (r0 + 1) / 2 <= chunk) ++r1;
      const int base = r0 * (r0 + 1) / 2, cnt = r1 * (r1 + 1) / 2 - base;
      __syncthreads();   // the previous chunk is consumed (and x is staged)
      for (int q = tid; q < cnt; q += blockDim.x) {
        ch[q] = Ah[base + q];
        cl[q] = Al[base + q];
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < MAXR; ++u) {
        const int i = tid + u * blockDim.x;
        if (i >= nA) continue;
        if (i >= r0 && i < r1) {            // row part of row i
          const int o = i * (i + 1) / 2 - base;
          for (int j = 0; j <= i; ++j) df_mac(acc[u], ch[o + j], cl[o + j], xh[j], xl[j]);
        }
        for (int j = (i + 1 > r0 ? i + 1 : r0); j < r1; ++j) {   // column part: A_ji, j > i
          const int o = j * (j + 1) / 2 - base + i;
          df_mac(acc[u], ch[o], cl[o], xh[j], xl[j]);
        }
      }
      r0 = r1;
    }
#pragma unroll
    for (int u = 0; u < MAXR; ++u) {
      const int i = tid + u * blockDim.x;
      if (i >= nA) continue;
      if (i < nu_) {  // (B^T x_p)_i = -s_i sum_j Bhat[j][i] x_p[j]
        const float sgn = i < nfd ? sg[i / s.nF] : 1.f;
        for (int p = 0; p < np_; ++p)
          df_mac(acc[u], -sgn * t.Bp_hi[p * nu_ + i], -sgn * t.Bp_lo[p * nu_ + i], xh[nA + p], xl[nA + p]);
      }
      const double v = df_value(acc[u]);
      const int64_t g = local_to_global(s, L, er, T, i);
      if (g < 0) continue;
      if (i >= nfd && i < nu_) y[g] = v;     // bubble: owned by T
      else atomicAdd(&y[g], v);             // facet dof: exactly two contributions into 0
    }
    for (int jp = tid; jp < np_; jp += blockDim.x) {
      DF a{0.f, 0.f, 0.f};
      for (int c = 0; c < nu_; ++c) {
        const float sgn = c < nfd ? sg[c / s.nF] : 1.f;
        df_mac(a, -sgn * t.Bp_hi[jp * nu_ + c], -sgn * t.Bp_lo[jp * nu_ + c], xh[c], xl[c]);
      }
      y[L.off_p + T * np_ + jp] = df_value(a);
    }
    __syncthreads();
  }
}

__global__ void k_zero_facet(const Layout L, double* y, const int* stop) {
  if (stop && *stop) return;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < L.n_dd; i += stride) y[i] = 0.0;
  for (i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n_hat; i += stride) y[L.off_h + i] = 0.0;
}

static int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

cudaError_t launch_apply_K(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L,
                           KOp K, const double* x, double* y, const int* stop, cudaStream_t st) {
  k_zero_facet<<<sm_count() * 4, 256, 0, st>>>(L, y, stop);
  note_launch();
  const int per = s.n_A + s.n_p;
  // algorithmic: packed symmetric A_T, x read once, y written once; flops: full row products
  const double alg_bytes = (double)m.ne * s.n_A * (s.n_A + 1) / 2 * 8.0 + 16.0 * L.ndof;
  const double alg_flops = 2.0 * (double)m.ne * ((double)s.n_A * s.n_A + 2.0 * s.n_u * s.n_p);
  if (K.Ahi && (2 * (size_t)packed_pad(s) + 2 * per) * sizeof(float) > 160 * 1024) {
    // packed pairs of one element beyond shared memory: streamed in row chunks of 12,288 entries
    const int chunk = 12288;
    const size_t sm = (2 * (size_t)chunk + 2 * per) * sizeof(float) + 64;
    int64_t blocks = (int64_t)sm_count() * 2;
    if (blocks > m.ne) blocks = m.ne;
    if (s.n_A > 512) return cudaErrorInvalidValue;
    static std::atomic<bool> set{false};
    if (!set.load(std::memory_order_acquire)) {
      cudaFuncSetAttribute(k_apply_K_df_chunk<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      set.store(true, std::memory_order_release);
    }
    prof_begin(PROF_APPLY, st);
    k_apply_K_df_chunk<2><<<(unsigned)blocks, 256, sm, st>>>(s, t, m, L, K.Ahi, K.Alo, x, y, chunk, stop);
    note_launch();
    prof_end(PROF_APPLY, alg_bytes, alg_flops, st);
    return cudaGetLastError();
  }
  if (K.Ahi) {
    const size_t per_bytes = (2 * (size_t)packed_pad(s) + 2 * per) * sizeof(float) + 4 * (sizeof(int) + sizeof(float));
    // one (element, row) per thread in one pass: as many elements as fill 256 threads, within 64 KB
    int EB = 256 / per;
    while (EB > 1 && (size_t)EB * per_bytes > 64 * 1024) --EB;
    if (K.eb > 0 && (size_t)K.eb * per_bytes <= 160 * 1024) EB = K.eb;   // autotuned
    if (EB < 1) EB = 1;
    const int threads = EB * per <= 128 ? 128 : 256;
    const size_t sm = (size_t)EB * per_bytes + 64;
    const int64_t blocks = (m.ne + EB - 1) / EB;
    dispatch_sizes(s, [&](auto sz) {
      static std::atomic<bool> set{false};
      if (!set.load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(k_apply_K_df<decltype(sz)>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        set.store(true, std::memory_order_release);
      }
      prof_begin(PROF_APPLY, st);
      k_apply_K_df<decltype(sz)><<<(unsigned)blocks, threads, sm, st>>>(sz, t, m, L, K.Ahi, K.Alo, x, y, EB, stop);
      note_launch();
      prof_end(PROF_APPLY, alg_bytes, alg_flops, st);
    });
    return cudaGetLastError();
  }
  const size_t small_bytes = (size_t)per * sizeof(double) + 4 * (sizeof(int) + sizeof(float));
  const size_t per_bytes = (size_t)s.n_A * s.n_A * sizeof(double) + small_bytes;
  const bool staged = per_bytes + 64 <= 200 * 1024;
  int EB = staged ? (int)((40 * 1024) / per_bytes) : 1;
  if (EB < 1) EB = 1;
  if (EB > 16) EB = 16;
  if (staged && K.eb > 0 && (size_t)K.eb * per_bytes + 64 <= 160 * 1024) EB = K.eb;   // autotuned
  const int threads = EB * per <= 128 ? 128 : 256;
  size_t sm = (size_t)EB * (staged ? per_bytes : small_bytes) + 64;
  int64_t blocks = (m.ne + EB - 1) / EB;
  dispatch_sizes(s, [&](auto sz) {
    static std::atomic<bool> set{false};
    if (!set.load(std::memory_order_acquire)) {
      cudaFuncSetAttribute(k_apply_K<decltype(sz), true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      set.store(true, std::memory_order_release);
    }
    prof_begin(PROF_APPLY, st);
    if (staged)
      k_apply_K<decltype(sz), true><<<(unsigned)blocks, threads, sm, st>>>(sz, t, m, L, K.AT, x, y, EB, stop);
    else
      k_apply_K<decltype(sz), false><<<(unsigned)blocks, threads, sm, st>>>(sz, t, m, L, K.AT, x, y, EB, stop);
    note_launch();
    prof_end(PROF_APPLY, alg_bytes, alg_flops, st);
  });
  return cudaGetLastError();
}

// ============================================================================ refinement residual
// Double-double arithmetic (error-free transformations: TwoProd with one fma, Knuth's TwoSum).
// Every operation is an explicitly rounded intrinsic so the compiler cannot contract or reorder.
struct DDv {
  double hi, lo;
};
__device__ __forceinline__ void dd_mac(DDv& a, double u, double v) {
  const double p = __dmul_rn(u, v);
  const double e = __fma_rn(u, v, -p);
  const double sum = __dadd_rn(a.hi, p);
  const double bb = __dsub_rn(sum, a.hi);
  const double err = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(sum, bb)), __dsub_rn(p, bb));
  a.hi = sum;
  a.lo = __dadd_rn(a.lo, __dadd_rn(err, e));
}
__device__ __forceinline__ DDv dd_add(DDv a, DDv b) {
  const double sum = __dadd_rn(a.hi, b.hi);
  const double bb = __dsub_rn(sum, a.hi);
  const double err = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(sum, bb)), __dsub_rn(b.hi, bb));
  return DDv{sum, __dadd_rn(err, __dadd_rn(a.lo, b.lo))};
}

// The rows of K_T x_T in double-double.  A block takes EB elements: their A_T (lower triangle,
// as doubles: FP64 storage, or the exact sums hi + lo of the float pairs of the mixed form) and
// their x_T are staged in shared memory, then one thread per (element, local row) accumulates
// with one TwoProd and one TwoSum per entry.  Contributions to a facet dof go to the slot of
// the element's side (s_{T,f} = +1: slot 0, -1: slot 1), so no sum is rounded before
// k_residual_combine.
template <class S, bool PACKED>
__global__ void __launch_bounds__(256) k_residual_rows(S s, DevTables t, DevMesh m, Layout L,
                                                       const double* __restrict__ AT, const float* __restrict__ Ahi,
                                                       const float* __restrict__ Alo, const double* __restrict__ x,
                                                       double* __restrict__ Y, int EB) {
  extern __shared__ double srd[];
  const int nA = s.n_A, np_ = s.n_p, nu_ = s.n_u, d = s.d, nfd = (s.d + 1) * s.nF;
  const int per = nA + np_, pl = nA * (nA + 1) / 2, pp = packed_pad(s);
  double* Ap = srd;               // [EB][pl] lower triangle, row-major
  double* xs = Ap + EB * pl;      // [EB][per]
  const int64_t nd = L.ndof;
  const int tid = threadIdx.x;
  for (int64_t T0 = (int64_t)blockIdx.x * EB; T0 < m.ne; T0 += (int64_t)gridDim.x * EB) {
    const int nvalid = (int)((m.ne - T0) < EB ? (m.ne - T0) : EB);
    for (int q = tid; q < nvalid * pl; q += blockDim.x) {
      const int e = q / pl, l = q - e * pl;
      const int64_t T = T0 + e;
      if (PACKED) {
        Ap[q] = (double)Ahi[T * pp + l] + (double)Alo[T * pp + l];
      } else {
        const int r = (int)((sqrtf(8.f * l + 1.f) - 1.f) * 0.5f);
        int rr = r;
        if (rr * (rr + 1) / 2 > l) --rr;
        else if ((rr + 1) * (rr + 2) / 2 <= l) ++rr;
        Ap[q] = AT[T * (int64_t)nA * nA + (int64_t)rr * nA + (l - rr * (rr + 1) / 2)];
      }
    }
    for (int q = tid; q < nvalid * per; q += blockDim.x) {
      const int e = q / per, j = q - e * per;
      const int64_t T = T0 + e;
      double v;
      if (j < nA) {
        const int64_t g = local_to_global(s, L, m.elem_rank + T * (d + 1), T, j);
        v = g < 0 ? 0.0 : x[g];
      } else {
        v = x[L.off_p + T * np_ + (j - nA)];
      }
      xs[q] = v;
    }
    __syncthreads();
    for (int q = tid; q < nvalid * per; q += blockDim.x) {
      const int e = q / per, i = q - e * per;
      const int64_t T = T0 + e;
      const int8_t* sg = m.signs + T * (d + 1);
      const double* xe = xs + e * per;
      const double* A = Ap + e * pl;
      DDv acc{0.0, 0.0};
      int64_t g;
      int slot = 0;
      if (i < nA) {
        const int row = i * (i + 1) / 2;
        for (int j = 0; j <= i; ++j) dd_mac(acc, A[row + j], xe[j]);
        for (int j = i + 1; j < nA; ++j) dd_mac(acc, A[j * (j + 1) / 2 + i], xe[j]);
        if (i < nu_) {  // (B^T x_p)_i = -s_i sum_p Bhat[p][i] x_p[p]
          const double sgn = i < nfd ? (double)sg[i / s.nF] : 1.0;
          for (int p = 0; p < np_; ++p) dd_mac(acc, -sgn * t.Bp[p * nu_ + i], xe[nA + p]);
        }
        g = local_to_global(s, L, m.elem_rank + T * (d + 1), T, i);
        if (g < 0) continue;
        if (i < nfd) slot = sg[i / s.nF] > 0 ? 0 : 1;
        else if (i >= nu_) slot = sg[(i - nu_) / s.nhF] > 0 ? 0 : 1;
      } else {
        const int jp = i - nA;
        for (int c = 0; c < nu_; ++c) {
          const double sgn = c < nfd ? (double)sg[c / s.nF] : 1.0;
          dd_mac(acc, -sgn * t.Bp[jp * nu_ + c], xe[c]);
        }
        g = L.off_p + T * np_ + jp;
      }
      Y[(2 * slot) * nd + g] = acc.hi;
      Y[(2 * slot + 1) * nd + g] = acc.lo;
    }
    __syncthreads();
  }
}

// The rows of K_T x_T in double-double for elements whose A_T does not fit in shared memory (3D
// k >= 5): one block per element, a thread per row i = tid + 256 u.  FP64 storage (full symmetric):
// A_ij read as A[j][i] straight from global memory (lanes of consecutive i read consecutive
// addresses); float pairs (packed lower): streamed through shared memory in chunks of whole rows as
// exact doubles hi + lo, row part and column part as in k_apply_K_df_chunk.  Output slots as in
// k_residual_rows.
template <bool PACKED, int MAXR>
__global__ void __launch_bounds__(256) k_residual_rows_big(ElemSizes s, DevTables t, DevMesh m, Layout L,
                                                           const double* __restrict__ AT,
                                                           const float* __restrict__ Ahi,
                                                           const float* __restrict__ Alo,
                                                           const double* __restrict__ x, double* __restrict__ Y,
                                                           int chunk) {
  extern __shared__ double srb[];
  const int nA = s.n_A, np_ = s.n_p, nu_ = s.n_u, d = s.d, nfd = (s.d + 1) * s.nF;
  const int per = nA + np_, pp = packed_pad(s);
  const int64_t nd = L.ndof;
  double* xs = srb;                  // [per]
  double* cb = xs + per;             // [chunk] (PACKED)
  const int tid = threadIdx.x;
  for (int64_t T = blockIdx.x; T < m.ne; T += gridDim.x) {
    const int8_t* sg = m.signs + T * (d + 1);
    for (int q = tid; q < per; q += blockDim.x) {
      double v;
      if (q < nA) {
        const int64_t g = local_to_global(s, L, m.elem_rank + T * (d + 1), T, q);
        v = g < 0 ? 0.0 : x[g];
      } else {
        v = x[L.off_p + T * np_ + (q - nA)];
      }
      xs[q] = v;
    }
    __syncthreads();
    DDv acc[MAXR];
#pragma unroll
    for (int u = 0; u < MAXR; ++u) acc[u] = DDv{0.0, 0.0};
    if (!PACKED) {
      const double* A = AT + T * (int64_t)nA * nA;
#pragma unroll
      for (int u = 0; u < MAXR; ++u) {
        const int i = tid + u * blockDim.x;
        if (i >= nA) continue;
        for (int j = 0; j < nA; ++j) dd_mac(acc[u], A[(int64_t)j * nA + i], xs[j]);
      }
    } else {
      const float* Ah = Ahi + T * (int64_t)pp;
      const float* Al = Alo + T * (int64_t)pp;
      int r0 = 0;
      while (r0 < nA) {
        int r1 = r0 + 1;
        while (r1 < nA && (r1 + 1) * (r1 + 2) / 2 - r0 * (r0 + 1) / 2 <= chunk) ++r1;
        const int base = r0 * (r0 + 1) / 2, cnt = r1 * (r1 + 1) / 2 - base;
        __syncthreads();
        for (int q = tid; q < cnt; q += blockDim.x) cb[q] = (double)Ah[base + q] + (double)Al[base + q];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < MAXR; ++u) {
          const int i = tid + u * blockDim.x;
          if (i >= nA) continue;
          if (i >= r0 && i < r1) {
            const int o = i * (i + 1) / 2 - base;
            for (int j = 0; j <= i; ++j) dd_mac(acc[u], cb[o + j], xs[j]);
          }
          for (int j = (i + 1 > r0 ? i + 1 : r0); j < r1; ++j) dd_mac(acc[u], cb[j * (j + 1) / 2 - base + i], xs[j]);
        }
        r0 = r1;
      }
    }
#pragma unroll
    for (int u = 0; u < MAXR; ++u) {
      const int i = tid + u * blockDim.x;
      if (i >= nA) continue;
      if (i < nu_) {  // (B^T x_p)_i = -s_i sum_p Bhat[p][i] x_p[p]
        const double sgn = i < nfd ? (double)sg[i / s.nF] : 1.0;
        for (int p = 0; p < np_; ++p) dd_mac(acc[u], -sgn * t.Bp[p * nu_ + i], xs[nA + p]);
      }
      const int64_t g = local_to_global(s, L, m.elem_rank + T * (d + 1), T, i);
      if (g < 0) continue;
      int slot = 0;
      if (i < nfd) slot = sg[i / s.nF] > 0 ? 0 : 1;
      else if (i >= nu_) slot = sg[(i - nu_) / s.nhF] > 0 ? 0 : 1;
      Y[(2 * slot) * nd + g] = acc[u].hi;
      Y[(2 * slot + 1) * nd + g] = acc[u].lo;
    }
    for (int jp = tid; jp < np_; jp += blockDim.x) {
      DDv a{0.0, 0.0};
      for (int c = 0; c < nu_; ++c) {
        const double sgn = c < nfd ? (double)sg[c / s.nF] : 1.0;
        dd_mac(a, -sgn * t.Bp[jp * nu_ + c], xs[c]);
      }
      const int64_t g = L.off_p + T * np_ + jp;
      Y[g] = a.hi;
      Y[nd + g] = a.lo;
    }
    __syncthreads();
  }
}

// r_g = F_g - (slot 0 + slot 1 for facet dofs, slot 0 otherwise), in double-double, rounded once.
__global__ void k_residual_combine(Layout L, const double* F, const double* __restrict__ Y, double* r) {
  const int64_t nd = L.ndof;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nd; g += (int64_t)gridDim.x * blockDim.x) {
    DDv y{Y[g], Y[nd + g]};
    const bool facet = g < L.off_o || (g >= L.off_h && g < L.off_p);
    if (facet) y = dd_add(y, DDv{Y[2 * nd + g], Y[3 * nd + g]});
    const DDv v = dd_add(DDv{F[g], 0.0}, DDv{-y.hi, -y.lo});
    r[g] = __dadd_rn(v.hi, v.lo);
  }
}

cudaError_t launch_residual_dd(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, KOp K,
                               const double* F, const double* x, double* Y, double* r, cudaStream_t st) {
  const int bs = 256;
  const int per = s.n_A + s.n_p;
  const size_t per_bytes = ((size_t)s.n_A * (s.n_A + 1) / 2 + per) * sizeof(double);
  if (per_bytes > 160 * 1024) {
    // one element's A_T beyond shared memory
    if (s.n_A > 512) return cudaErrorInvalidValue;
    const int chunk = 12288;
    const size_t sm = ((size_t)per + (K.Ahi ? chunk : 0)) * sizeof(double) + 16;
    int64_t g = (int64_t)sm_count() * 2;
    if (g > m.ne) g = m.ne;
    static std::atomic<bool> set{false};
    if (!set.load(std::memory_order_acquire)) {
      cudaFuncSetAttribute(k_residual_rows_big<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(k_residual_rows_big<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      set.store(true, std::memory_order_release);
    }
    if (K.Ahi)
      k_residual_rows_big<true, 2><<<(unsigned)g, bs, sm, st>>>(s, t, m, L, nullptr, K.Ahi, K.Alo, x, Y, chunk);
    else
      k_residual_rows_big<false, 2><<<(unsigned)g, bs, sm, st>>>(s, t, m, L, K.AT, nullptr, nullptr, x, Y, chunk);
    note_launch();
    k_residual_combine<<<sm_count() * 8, bs, 0, st>>>(L, F, Y, r);
    note_launch();
    return cudaGetLastError();
  }
  int EB = bs / per;
  while (EB > 1 && (size_t)EB * per_bytes > 48 * 1024) --EB;
  if (EB < 1) EB = 1;
  const size_t sm = (size_t)EB * per_bytes;
  int64_t g = (m.ne + EB - 1) / EB;
  if (g > (int64_t)sm_count() * 32) g = (int64_t)sm_count() * 32;
  dispatch_sizes(s, [&](auto sz) {
    using SZ = decltype(sz);
    static std::atomic<bool> set{false};
    if (!set.load(std::memory_order_acquire)) {
      cudaFuncSetAttribute(k_residual_rows<SZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(k_residual_rows<SZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      set.store(true, std::memory_order_release);
    }
    if (K.Ahi)
      k_residual_rows<SZ, true><<<(unsigned)g, bs, sm, st>>>(sz, t, m, L, nullptr, K.Ahi, K.Alo, x, Y, EB);
    else
      k_residual_rows<SZ, false><<<(unsigned)g, bs, sm, st>>>(sz, t, m, L, K.AT, nullptr, nullptr, x, Y, EB);
    note_launch();
  });
  k_residual_combine<<<sm_count() * 8, bs, 0, st>>>(L, F, Y, r);
  note_launch();
  return cudaGetLastError();
}


// ---------------------------------------------------------------- mass and load
__global__ void k_mass_u(ElemSizes s, DevTables t, DevMesh m, Layout L, const double* c, double* F) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int d = s.d, nu_ = s.n_u;
  for (int64_t T = (int64_t)blockIdx.x * wpb + wib; T < m.ne; T += (int64_t)gridDim.x * wpb) {
    const int32_t* er = m.elem_rank + T * (d + 1);
    double J[9], G[9];
    const int32_t* ev = m.elems + T * (d + 1);
    for (int a = 0; a < d; ++a)
      for (int i = 0; i < d; ++i) J[a * d + i] = m.coords[(int64_t)ev[i + 1] * d + a] - m.coords[(int64_t)ev[0] * d + a];
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double v = 0;
        for (int q = 0; q < d; ++q) v += J[q * d + a] * J[q * d + b];
        G[a * d + b] = v;
      }
    const double inv = 1.0 / m.adet[T];
    for (int i = lane; i < nu_; i += 32) {
      int64_t gi = local_to_global(s, L, er, T, i);
      if (gi < 0) continue;
      double si = (i < (d + 1) * s.nF) ? (double)m.signs[T * (d + 1) + i / s.nF] : 1.0;
      double v = 0;
      for (int j = 0; j < nu_; ++j) {
        int64_t gj = local_to_global(s, L, er, T, j);
        if (gj < 0) continue;
        double sj = (j < (d + 1) * s.nF) ? (double)m.signs[T * (d + 1) + j / s.nF] : 1.0;
        double mij = 0;
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) mij += G[a * d + b] * t.Mu[((a * d + b) * nu_ + i) * nu_ + j];
        v += mij * sj * c[gj];
      }
      v *= si * inv;
      if (i >= (d + 1) * s.nF) F[gi] = v;
      else atomicAdd(&F[gi], v);
    }
  }
}

cudaError_t launch_mass_u(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L,
                          const double* c, double* F, cudaStream_t st) {
  cudaMemsetAsync(F, 0, sizeof(double) * L.ndof, st);
  k_mass_u<<<sm_count() * 8, 128, 0, st>>>(s, t, m, L, c, F);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_load_points(ElemSizes s, DevTables t, DevMesh m, double* xq) {
  const int d = s.d;
  int64_t n = m.ne * t.nq_load;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < n; id += (int64_t)gridDim.x * blockDim.x) {
    int64_t T = id / t.nq_load;
    int q = (int)(id % t.nq_load);
    const int32_t* ev = m.elems + T * (d + 1);
    for (int a = 0; a < d; ++a) {
      double v = m.coords[(int64_t)ev[0] * d + a];
      for (int i = 0; i < d; ++i)
        v += (m.coords[(int64_t)ev[i + 1] * d + a] - m.coords[(int64_t)ev[0] * d + a]) * t.xq_load[q * d + i];
      xq[id * d + a] = v;
    }
  }
}

// ---------------------------------------------------------------- stress recovery
// Per element (one block): the condensation workspace is rebuilt (condense_element), the local
// velocity coefficients are gathered from x with the orientation signs of the facet-BDM dofs removed,
// and recover_element evaluates sigma_h and omega_h at the reference points (eq. projection).
template <bool SMEM>
__global__ void __launch_bounds__(256) k_recover(ElemSizes s, DevTables t, DevMesh m, Layout L, double nu,
                                                 const double* __restrict__ x, int nq, const double* __restrict__ psi,
                                                 double* sig, double* om, double* gscratch, int64_t slot) {
  extern __shared__ double smr[];
  const int lane = threadIdx.x, nl = blockDim.x, d = s.d, nA = s.n_A, nfd = (s.d + 1) * s.nF;
  double* base = SMEM ? smr : gscratch + (int64_t)blockIdx.x * slot;
  ElemWork w = elem_work_carve(s, base);
  double* Xs = base + elem_work_doubles(s);
  int* sg = (int*)(Xs + 16);
  double* a = Xs + 24;
  double* wk = a + nA;
  ElemTables et{t.B0, t.Rf, t.Bh, t.Ccon, t.Adiv, t.nhat, t.Wmom};
  const int64_t per = (int64_t)nq * d * d;
  for (int64_t T = blockIdx.x; T < m.ne; T += gridDim.x) {
    if (lane < (d + 1) * d) {
      const int v = lane / d, c = lane % d;
      Xs[lane] = m.coords[(int64_t)m.elems[T * (d + 1) + v] * d + c];
    }
    if (lane <= d) sg[lane] = m.signs[T * (d + 1) + lane];
    __syncthreads();
    condense_element(s, et, Xs, sg, nu, w, lane, nl, BlockSync());
    for (int i = lane; i < nA; i += nl) {
      const int64_t g = local_to_global(s, L, m.elem_rank + T * (d + 1), T, i);
      const double sgi = i < nfd ? (double)sg[i / s.nF] : (is_rot_dof(s, i) ? (double)sg[(i - s.n_u) / s.nhF] : 1.0);
      a[i] = g < 0 ? 0.0 : x[g] * sgi;
    }
    __syncthreads();
    recover_element(s, w, Xs, a, nq, psi, wk, sig + T * per, om ? om + T * per : nullptr, lane, nl, BlockSync());
  }
}

int64_t recover_slot_doubles(const ElemSizes& s) {
  return ((int64_t)elem_work_doubles(s) + 24 + s.n_A + s.n_cc + 2 * s.n_raw + 31) / 32 * 32;
}

cudaError_t launch_recover(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, double nu,
                           const double* x, int nq, const double* psi, double* sig, double* om, double* scratch,
                           int64_t scratch_doubles, cudaStream_t st) {
  const int64_t slot = recover_slot_doubles(s);
  int dev = 0, nsm = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int threads = s.d == 2 ? 128 : 256;
  if (slot * 8 <= maxsm) {
    const size_t sm = (size_t)slot * 8;
    cudaFuncSetAttribute(k_recover<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_recover<true>, threads, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)nsm * per_sm;
    if (blocks > m.ne) blocks = m.ne;
    k_recover<true><<<(unsigned)blocks, threads, sm, st>>>(s, t, m, L, nu, x, nq, psi, sig, om, nullptr, slot);
    note_launch();
  } else {
    int64_t blocks = scratch_doubles / slot;
    if (blocks < 1) return cudaErrorMemoryAllocation;
    if (blocks > m.ne) blocks = m.ne;
    k_recover<false><<<(unsigned)blocks, threads, 0, st>>>(s, t, m, L, nu, x, nq, psi, sig, om, scratch, slot);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_load_points(const ElemSizes& s, const DevTables& t, const DevMesh& m, double* xq,
                               cudaStream_t st) {
  k_load_points<<<sm_count() * 8, 256, 0, st>>>(s, t, m, xq);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_load(ElemSizes s, DevTables t, DevMesh m, Layout L, const double* fq, double* F) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int d = s.d, nu_ = s.n_u;
  for (int64_t T = (int64_t)blockIdx.x * wpb + wib; T < m.ne; T += (int64_t)gridDim.x * wpb) {
    const int32_t* er = m.elem_rank + T * (d + 1);
    const int32_t* ev = m.elems + T * (d + 1);
    double J[9];
    for (int a = 0; a < d; ++a)
      for (int i = 0; i < d; ++i) J[a * d + i] = m.coords[(int64_t)ev[i + 1] * d + a] - m.coords[(int64_t)ev[0] * d + a];
    for (int i = lane; i < nu_; i += 32) {
      int64_t gi = local_to_global(s, L, er, T, i);
      if (gi < 0) continue;
      double v = 0;
      for (int q = 0; q < t.nq_load; ++q) {
        const double* f = fq + (T * t.nq_load + q) * d;
        // (J^T f) . phi_hat
        for (int b = 0; b < d; ++b) {
          double jf = 0;
          for (int a = 0; a < d; ++a) jf += J[a * d + b] * f[a];
          v += t.wq_load[q] * jf * t.phi_load[(q * nu_ + i) * d + b];
        }
      }
      double si = (i < (d + 1) * s.nF) ? (double)m.signs[T * (d + 1) + i / s.nF] : 1.0;
      v *= si;
      if (i >= (d + 1) * s.nF) F[gi] = v;
      else atomicAdd(&F[gi], v);
    }
  }
}

cudaError_t launch_load(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L,
                        const double* fq, double* F, cudaStream_t st) {
  cudaMemsetAsync(F, 0, sizeof(double) * L.ndof, st);
  k_load<<<sm_count() * 8, 128, 0, st>>>(s, t, m, L, fq, F);
  note_launch();
  return cudaGetLastError();
}

// ============================================================================ preconditioner (precision R)
// gather the coupling vector x_T (facet-major) of element T from an external-layout vector
// index of coupling dof t (facet-major: u_d modes, then uhat modes) of interior facet rk
template <class R, class S>
__device__ __forceinline__ int64_t coup_idx(const S& s, const Layout& L, int32_t rk, int t) {
  if (L.fstride) return (int64_t)rk * L.fstride + t;
  return (t < s.nF) ? (int64_t)rk * s.nF + t : L.off_h + (int64_t)rk * s.nhF + (t - s.nF);
}
template <class R, class S>
__device__ __forceinline__ R coup_get(const S& s, const Layout& L, const R* x, int32_t rk, int t) {
  if (rk < 0) return (R)0;
  return x[coup_idx<R>(s, L, rk, t)];
}

// b (preconditioner layout PL, precision R) = a (external layout L); padding entries are zero
template <class R>
__global__ void k_to_prec(ElemSizes s, Layout L, Layout PL, const double* __restrict__ a, R* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < PL.ndof;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (i < PL.n_dd) {
      const int64_t rk = i / PL.fstride;
      const int t = (int)(i - rk * PL.fstride);
      v = t < s.nF ? a[rk * s.nF + t] : (t < s.mF ? a[L.off_h + rk * s.nhF + (t - s.nF)] : 0.0);
    } else if (i < PL.off_p) {
      v = a[L.off_o + (i - PL.off_o)];
    } else {
      v = a[L.off_p + (i - PL.off_p)];
    }
    b[i] = (R)v;
  }
}
// b (external layout L, FP64) = a (preconditioner layout PL)
template <class R>
__global__ void k_from_prec(ElemSizes s, Layout L, Layout PL, const R* __restrict__ a, double* __restrict__ b,
                            const int* stop) {
  if (stop && *stop) return;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L.ndof;
       j += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    if (j < L.n_dd) {
      const int64_t rk = j / s.nF;
      i = rk * PL.fstride + (j - rk * s.nF);
    } else if (j < L.off_h) {
      i = PL.off_o + (j - L.off_o);
    } else if (j < L.off_p) {
      const int64_t q = j - L.off_h, rk = q / s.nhF;
      i = rk * PL.fstride + s.nF + (q - rk * s.nhF);
    } else {
      i = PL.off_p + (j - L.off_p);
    }
    b[j] = (double)a[i];
  }
}

// ---------------------------------------------------------------- element-level preconditioner kernels
// Prologue of one Ahat^{-1} application (bubble elimination, eq. factorSsigma):
//   rin_o = r_o - (B^T z_p)_o                          (WITH_BT; else rin_o = r_o)
//   tb   += (B^T z_p)_c + (G^T rin_o)_c                 (two contributions per facet dof, into zero)
// B = -Bhat diag(sign) (reading R18), z_p read from zp (pressure layout of the full vector).
template <class R, class S, bool WITH_BT, bool STAGE = true>
__global__ void __launch_bounds__(256) k_elem_prologue(S s, DevTables t, DevMesh m, Layout L,
                                                       const R* __restrict__ G, const R* __restrict__ r,
                                                       const R* __restrict__ zp, R* rin, R* tb, int EB,
                                                       const int* stop) {
  if (stop && *stop) return;
  extern __shared__ unsigned char sraw[];
  const int d = s.d, nc = s.n_c, no = s.n_bub, nu_ = s.n_u, np_ = s.n_p, nfd = (s.d + 1) * s.nF;
  const int gs = g_stride(s);
  // STAGE: G of the EB elements in shared memory; else (one element's G beyond shared memory) read from
  // global memory, column c of row o at o*nc + c (lanes of consecutive c: consecutive addresses)
  R* Gst = (R*)sraw;             // [EB][gs] (STAGE)
  R* ro = Gst + (STAGE ? EB * gs : 0);   // [EB][no]
  R* bt = ro + EB * no;          // [EB][nu]
  R* zz = bt + EB * nu_;         // [EB][np]
  const int64_t T0 = (int64_t)blockIdx.x * EB;
  const int nvalid = (int)((m.ne - T0) < EB ? (m.ne - T0) : EB);
  const int tid = threadIdx.x;
  const R* Gs = STAGE ? Gst : G + T0 * gs;
  if (STAGE) vcopy16<R>(Gst, G + T0 * gs, nvalid * gs, tid, blockDim.x);
  for (int q = tid; q < nvalid * no; q += blockDim.x) ro[q] = r[L.off_o + T0 * no + q];
  if (WITH_BT)
    for (int q = tid; q < nvalid * np_; q += blockDim.x) zz[q] = zp[L.off_p + T0 * np_ + q];
  __syncthreads();
  if (WITH_BT) {
    // the B table in the preconditioner's precision (float: its leading part)
    const R* Bt = sizeof(R) == 4 ? (const R*)(const void*)t.Bp_hi : (const R*)(const void*)t.Bp;
    for (int q = tid; q < nvalid * nu_; q += blockDim.x) {
      const int e = q / nu_, i = q - e * nu_;
      const int64_t T = T0 + e;
      R sg = i < nfd ? (R)m.signs[T * (d + 1) + i / s.nF] : (R)1;
      R v = 0;
      for (int j = 0; j < np_; ++j) v += Bt[j * nu_ + i] * zz[e * np_ + j];
      bt[q] = -sg * v;
    }
    __syncthreads();
    for (int q = tid; q < nvalid * no; q += blockDim.x) {
      const int e = q / no, o = q - e * no;
      ro[q] -= bt[e * nu_ + nfd + o];
    }
    __syncthreads();
  }
  for (int q = tid; q < nvalid * no; q += blockDim.x) rin[L.off_o + T0 * no + q] = ro[q];
  for (int q = tid; q < nvalid * nc; q += blockDim.x) {
    const int e = q / nc, c = q - e * nc;
    const int64_t T = T0 + e;
    const int f = c / s.mF, tt = c - f * s.mF;
    const int32_t rk = m.elem_rank[T * (d + 1) + f];
    if (rk < 0) continue;
    R v = 0;
    const R* g = Gs + e * gs + c;
    const R* rv = ro + e * no;
#pragma unroll 4
    for (int o = 0; o < no; ++o) v += g[o * nc] * rv[o];
    if (WITH_BT && tt < s.nF) v += bt[e * nu_ + f * s.nF + tt];
    atomicAdd(&tb[coup_idx<R>(s, L, rk, tt)], v);
  }
}

// Epilogue of one Ahat^{-1} application (back substitution, eq. factorSsigma):
//   x_o = A_oo^{-1} rin_o - G x_c
// WITH_P (first application of eq. mhatinvfactor): also z_p = Shat_p^{-1}(r_p - B a), a = (x_c, x_o),
// Shat_p = M_p = nu^{-1}(p, q)  ->  z_p = nu/|det J| (r_p - B a).
template <class R, class S, bool WITH_P, bool STAGE = true>
__global__ void __launch_bounds__(256) k_elem_epilogue(S s, DevTables t, DevMesh m, Layout L, double nu,
                                                       const R* __restrict__ G, const R* __restrict__ Aoi,
                                                       const R* __restrict__ rin, const R* __restrict__ r, R* x,
                                                       R* zp, int EB, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ unsigned char sraw[];
  const int d = s.d, nc = s.n_c, no = s.n_bub, nu_ = s.n_u, np_ = s.n_p, nfd = (s.d + 1) * s.nF, mF = s.mF;
  const int gs = g_stride(s), as_ = a_stride(s);
  // STAGE: G and A_oo^{-1} of the EB elements in shared memory; else read from global memory (one
  // element), A_oo^{-1} by columns (it is symmetric), G by rows
  R* Gst = (R*)sraw;             // [EB][gs] (STAGE)
  R* Ast = Gst + (STAGE ? EB * gs : 0);  // [EB][as] (STAGE)
  R* xc = Ast + (STAGE ? EB * as_ : 0);  // [EB][nc]
  R* ro = xc + EB * nc;          // [EB][no]
  R* xo = ro + EB * no;          // [EB][no]
  const int64_t T0 = (int64_t)blockIdx.x * EB;
  const int nvalid = (int)((m.ne - T0) < EB ? (m.ne - T0) : EB);
  const int tid = threadIdx.x;
  const R* Gs = STAGE ? Gst : G + T0 * gs;
  const R* As = STAGE ? Ast : Aoi + T0 * as_;
  if (STAGE) {
    vcopy16<R>(Gst, G + T0 * gs, nvalid * gs, tid, blockDim.x);
    vcopy16<R>(Ast, Aoi + T0 * as_, nvalid * as_, tid, blockDim.x);
  }
  for (int q = tid; q < nvalid * no; q += blockDim.x) ro[q] = rin[L.off_o + T0 * no + q];
  for (int q = tid; q < nvalid * nc; q += blockDim.x) {
    const int e = q / nc, c = q - e * nc;
    const int64_t T = T0 + e;
    const int f = c / mF;
    xc[q] = coup_get<R>(s, L, x, m.elem_rank[T * (d + 1) + f], c - f * mF);
  }
  __syncthreads();
  for (int q = tid; q < nvalid * no; q += blockDim.x) {
    const int e = q / no, o = q - e * no;
    R v = 0;
    const R* a = As + e * as_ + (STAGE ? o * no : o);   // row o, or column o of the symmetric inverse
    const int ast = STAGE ? 1 : no;
    const R* rv = ro + e * no;
#pragma unroll 4
    for (int p = 0; p < no; ++p) v += a[p * ast] * rv[p];
    const R* g = Gs + e * gs + o * nc;
    const R* xv = xc + e * nc;
#pragma unroll 4
    for (int c = 0; c < nc; ++c) v -= g[c] * xv[c];
    xo[q] = v;
    x[L.off_o + T0 * no + q] = v;
  }
  if (WITH_P) {
    __syncthreads();
    // in the precision of the preconditioner: the B table as R (float: its leading part)
    const R* Bt = sizeof(R) == 4 ? (const R*)(const void*)t.Bp_hi : (const R*)(const void*)t.Bp;
    for (int q = tid; q < nvalid * np_; q += blockDim.x) {
      const int e = q / np_, j = q - e * np_;
      const int64_t T = T0 + e;
      R v = 0;  // sum_i Bhat[j][i] sign_i a_i over the velocity dofs
      const R* Bj = Bt + j * nu_;
      for (int f = 0; f <= d; ++f) {
        const R sg = (R)m.signs[T * (d + 1) + f];
        const R* xf = xc + e * nc + f * mF;
        R vf = 0;
        for (int i = 0; i < s.nF; ++i) vf += Bj[f * s.nF + i] * xf[i];
        v += sg * vf;
      }
      for (int o = 0; o < no; ++o) v += Bj[nfd + o] * xo[e * no + o];
      const int64_t gp = L.off_p + T * np_ + j;
      zp[gp] = (R)(nu / m.adet[T]) * (r[gp] + v);
    }
  }
}

// Facet-centric block step over the facet records rec[0..n) (colour order):
//   r_F = b_F - tb_F - sum_{T in F} (A^d_T x_T)|_F,
// UPDATE: x_F += D_F^{-1} r_F (block Gauss-Seidel within one colour); else rr_F = r_F.
// Vectors are in the preconditioner layout (L.fstride > 0): the m_F coupling values of a facet
// are one 16-byte-aligned segment, fetched with 16-byte copies.  Persistent blocks walk batches
// of FB facets.  Everything a batch needs (A^d slabs of both elements, D_F^{-1}, the segments of
// all facets of both elements, b, tb) is fetched with asynchronous copies into one of two
// shared-memory stages while the previous batch is computed; the 64-byte facet records are read
// one batch ahead.  Slabs and D_F^{-1} are read once per pass and carry an L2 evict-first hint.
// Facets of one colour share no element, so the copies of batch i+1 never read values that
// batch i updates.
template <class R, class S, bool UPDATE>
__global__ void __launch_bounds__(256) k_facet_step(S s, DevMesh m, Layout L, const R* __restrict__ Fs,
                                                    const R* __restrict__ b,
                                                    const R* __restrict__ tb, R* x, R* rr,
                                                    const int4* __restrict__ rec, int64_t n, int FB,
                                                    const int* stop, int* dbg, int64_t fs_avail,
                                                    int smem_bytes) {
  if (stop && *stop) return;
  // diagnostics: returns false (and records the first failure) for an access outside its buffer
  // or a 16-byte copy off its alignment
  auto ok = [&](int code, int64_t off, int64_t len, int64_t size, const void* addr, bool a16) -> bool {
    if (!dbg) return true;
    const bool good = off >= 0 && off + len <= size && (!a16 || (reinterpret_cast<uintptr_t>(addr) & 15) == 0);
    if (!good && atomicCAS(dbg, 0, code) == 0) {
      dbg[1] = (int)blockIdx.x;
      dbg[2] = (int)(off & 0x7fffffff);
      dbg[3] = (int)(size & 0x7fffffff);
    }
    return good;
  };
  extern __shared__ __align__(16) unsigned char sraw[];
  const int mF = s.mF, dp1 = s.d + 1, slab = slab_pad(s), fss = fs_stride(s);
  const int fs = facet_stride(s, (int)sizeof(R));   // equals L.fstride
  const int xe = dp1 * fs;                          // gathered values per (facet, side)
  // stage layout (both stages identical, 16-byte aligned pieces)
  unsigned char* sbase = sraw;
  const int rec_b = FB * 16 * (int)sizeof(int);
  const int fsb = FB * fss * (int)sizeof(R);        // the batch's facet-stream blocks
  const int xt_b = FB * 2 * xe * (int)sizeof(R);
  const int bb_b = FB * fs * (int)sizeof(R);
  const int stage_b = rec_b + fsb + xt_b + 2 * bb_b;
  R* yS = (R*)(sbase + 2 * stage_b);       // [FB][2][mF]
  R* rF = yS + FB * 2 * mF;                // [FB][mF]
  auto RC = [&](int st) { return (int*)(sbase + st * stage_b); };
  auto FSB = [&](int st) { return (R*)(sbase + st * stage_b + rec_b); };
  auto XT = [&](int st) { return (R*)(sbase + st * stage_b + rec_b + fsb); };
  auto BS = [&](int st) { return (R*)(sbase + st * stage_b + rec_b + fsb + xt_b); };
  auto TS = [&](int st) { return (R*)(sbase + st * stage_b + rec_b + fsb + xt_b + bb_b); };
  constexpr int V = 16 / (int)sizeof(R);
  const int cf = fss / V, cslab = 2 * slab / V, cx = fs / V;
  const int tid = threadIdx.x;
  const int64_t nb = (n + FB - 1) / FB;
  const uint64_t pol = l2_evict_first_policy();

  auto load_records = [&](int st, int64_t bi) {
    int* rc = RC(st);
    for (int q = tid; q < FB * 4; q += blockDim.x) {
      const int fb = q >> 2;
      int4 v = make_int4(-1, -1, -1, -1);
      if (bi * FB + fb < n) v = rec[(bi * FB + fb) * 4 + (q & 3)];
      reinterpret_cast<int4*>(rc)[q] = v;
    }
  };
  auto issue = [&](int st, int64_t bi) {
    const int* rc = RC(st);
    R* Fb = FSB(st);
    R* xT = XT(st);
    R* bS = BS(st);
    R* tS = TS(st);
    // the batch's stream blocks are one contiguous range (without D_F^{-1} for the residual pass)
    const int nvalid = (int)((n - bi * FB) < FB ? (n - bi * FB) : FB);
    const R* src = Fs + bi * FB * (int64_t)fss;
    for (int q = tid; q < nvalid * cf; q += blockDim.x) {
      if (!UPDATE && q % cf >= cslab) continue;
      R* dst = Fb + q * V;
      const R* sp = src + (int64_t)q * V;
      if (!ok(1, (const unsigned char*)dst - sraw, 16, smem_bytes, dst, true)) continue;
      if (!ok(2, bi * FB * (int64_t)fss + (int64_t)q * V, V, fs_avail, sp, true)) continue;
      cp_async16_hint(dst, sp, pol);
    }
    for (int q = tid; q < FB * 2 * dp1 * cx; q += blockDim.x) {
      const int seg = q / cx, ch = q - seg * cx;          // seg = (fb*2 + side)*dp1 + f
      const int fsd = seg / dp1, f = seg - fsd * dp1, fb = fsd >> 1, side = fsd & 1;
      const int* r_ = rc + fb * 16;
      const int32_t g = r_[0] >= 0 ? r_[5 + side * dp1 + f] : -1;
      R* dst = xT + seg * fs + ch * V;
      if (!ok(3, (const unsigned char*)dst - sraw, 16, smem_bytes, dst, true)) continue;
      if (g >= 0) {
        if (!ok(4, (int64_t)g * fs + ch * V, V, L.ndof, x + (int64_t)g * fs + ch * V, true)) continue;
        cp_async16(dst, x + (int64_t)g * fs + ch * V);
      } else {
        *reinterpret_cast<int4*>(dst) = make_int4(0, 0, 0, 0);
      }
    }
    for (int q = tid; q < FB * cx; q += blockDim.x) {
      const int fb = q / cx, ch = q - fb * cx;
      const int r = rc[fb * 16];
      R* db = bS + fb * fs + ch * V;
      R* dt = tS + fb * fs + ch * V;
      if (!ok(5, (const unsigned char*)dt - sraw, 16, smem_bytes, dt, true)) continue;
      if (r >= 0) {
        if (!ok(6, (int64_t)r * fs + ch * V, V, L.ndof, b + (int64_t)r * fs + ch * V, true)) continue;
        cp_async16(db, b + (int64_t)r * fs + ch * V);
        if (tb) cp_async16(dt, tb + (int64_t)r * fs + ch * V);
        else *reinterpret_cast<int4*>(dt) = make_int4(0, 0, 0, 0);
      } else {
        *reinterpret_cast<int4*>(db) = make_int4(0, 0, 0, 0);
        *reinterpret_cast<int4*>(dt) = make_int4(0, 0, 0, 0);
      }
    }
  };

  int64_t bi = blockIdx.x;
  int st = 0;
  if (bi < nb) {
    load_records(0, bi);
    __syncthreads();
    issue(0, bi);
  }
  cp_async_commit();
  while (bi < nb) {
    const int64_t nbi = bi + gridDim.x;
    const int ns = st ^ 1;
    if (nbi < nb) load_records(ns, nbi);
    __syncthreads();
    if (nbi < nb) issue(ns, nbi);
    cp_async_commit();
    cp_async_wait_group<1>();
    __syncthreads();
    // ---- compute batch bi from stage st
    const int* rc = RC(st);
    const R* Fb = FSB(st);
    const R* xT = XT(st);
    const R* bS = BS(st);
    const R* tS = TS(st);
    for (int q = tid; q < FB * 2 * mF; q += blockDim.x) {
      const int fsd = q / mF, t = q - fsd * mF;
      const R* A = Fb + (fsd >> 1) * fss + (fsd & 1) * slab + t;
      const R* xv = xT + fsd * xe;
      R v0 = 0, v1 = 0;
#pragma unroll
      for (int f = 0; f < dp1; ++f) {
        const R* Af = A + f * mF * mF;
        const R* xf = xv + f * fs;
        int tt = 0;
#pragma unroll
        for (; tt + 1 < mF; tt += 2) {
          v0 += Af[tt * mF] * xf[tt];
          v1 += Af[(tt + 1) * mF] * xf[tt + 1];
        }
        if (tt < mF) v0 += Af[tt * mF] * xf[tt];
      }
      yS[q] = v0 + v1;
    }
    __syncthreads();
    for (int q = tid; q < FB * mF; q += blockDim.x) {
      const int fb = q / mF, t = q - fb * mF;
      const int r = rc[fb * 16];
      const R v = bS[fb * fs + t] - tS[fb * fs + t] - yS[(fb * 2) * mF + t] - yS[(fb * 2 + 1) * mF + t];
      if (UPDATE) rF[q] = v;
      else if (r >= 0 && ok(7, (int64_t)r * fs + t, 1, L.ndof, rr, false)) rr[(int64_t)r * fs + t] = v;
    }
    if (UPDATE) {
      __syncthreads();
      for (int q = tid; q < FB * mF; q += blockDim.x) {
        const int fb = q / mF, t = q - fb * mF;
        const int r = rc[fb * 16];
        if (r < 0) continue;
        const R* Dr = Fb + fb * fss + 2 * slab + t * mF;
        const R* rv = rF + fb * mF;
        R v = 0;
        for (int j = 0; j < mF; ++j) v += Dr[j] * rv[j];
        // x_F before the update is the facet's own segment in the gathered values of side 0
        const int f0 = rc[fb * 16 + 3];
        if (!ok(8, (int64_t)r * fs + t, 1, L.ndof, x, false) || !ok(9, f0, 1, dp1, x, false)) continue;
        x[(int64_t)r * fs + t] = xT[(fb * 2) * xe + f0 * fs + t] + v;
      }
    }
    __syncthreads();
    st = ns;
    bi = nbi;
  }
  cp_async_wait_all();
}

// xbar = E^d^T rr (rr + rr2 when rr2 is given): one warp per P1 vertex; the lanes take the (incident facet, mode) pairs and the
// d sums are combined by a fixed butterfly, so the result does not depend on scheduling.
template <class R>
__global__ void k_embed_T(ElemSizes s, Layout L, const R* Eb, const int32_t* vf_ptr, const int32_t* vf_idx,
                          int64_t nP1, const R* rr, const R* rr2, R* xb, const int* stop) {
  if (stop && *stop) return;
  const int d = s.d, mF = s.mF, lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = w0; v < nP1; v += ws) {
    const int32_t e0 = vf_ptr[v], ne = vf_ptr[v + 1] - e0;
    R acc[3] = {0, 0, 0};
    for (int q = lane; q < ne * mF; q += 32) {
      const int ei = q / mF, t = q - ei * mF;
      const int32_t rk = vf_idx[2 * (e0 + ei)], w = vf_idx[2 * (e0 + ei) + 1];
      const int64_t ci = coup_idx<R>(s, L, rk, t);
      const R r = rr2 ? rr[ci] + rr2[ci] : rr[ci];   // rr2: the residual kept as two partial sums
      const R* B = Eb + (((int64_t)rk * d + w) * mF + t) * d;   // layout [nint][d (w)][mF][d (a)]
      for (int a = 0; a < d; ++a) acc[a] += B[a] * r;
    }
    for (int a = 0; a < d; ++a) {
      R x = acc[a];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) xb[v * d + a] = x;
    }
  }
}

// x_F += E^d_F xbar  (facet vertices' P1 ranks in fvr [nint][d])
template <class R>
__global__ void k_embed(ElemSizes s, Layout L, const R* Eb, const int32_t* fvr, int64_t nint, const R* xb, R* x,
                        const int* stop) {
  if (stop && *stop) return;
  const int d = s.d, mF = s.mF;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nint * mF;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t rk = q / mF;
    int t = (int)(q % mF);
    R v = 0;
    for (int w = 0; w < d; ++w) {
      int32_t vr = fvr[rk * d + w];
      if (vr < 0) continue;
      const R* B = Eb + ((rk * d + w) * mF + t) * d;   // layout [nint][d (w)][mF][d (a)]
      for (int a = 0; a < d; ++a) v += B[a] * xb[(int64_t)vr * d + a];
    }
    x[coup_idx<R>(s, L, (int32_t)rk, t)] += v;
  }
}

// ---- GMG kernels ----
// l1-Jacobi sweep xn = x + D (b - A x) (first: from x = 0, xn = D b).
template <class R>
__global__ void k_jacobi(Ell A, const R* dinv, const R* b, const R* x, R* xn, int first, const int* stop) {
  if (stop && *stop) return;
  const int64_t n = A.n;
  const R* va = (const R*)A.val;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (first) {
      xn[i] = dinv[i] * b[i];
      continue;
    }
    R ax = 0;
    for (int k = 0; k < A.k; ++k) ax += va[k * n + i] * x[A.col[k * n + i]];
    xn[i] = x[i] + dinv[i] * (b[i] - ax);
  }
}
// Two l1-Jacobi sweeps from x = 0 in one pass: x1 = D b, x2 = x1 + D (b - A x1).
template <class R>
__global__ void k_jacobi2_from_b(Ell A, const R* dinv, const R* b, R* xn, const int* stop) {
  if (stop && *stop) return;
  const int64_t n = A.n;
  const R* va = (const R*)A.val;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    R ax = 0;
    for (int k = 0; k < A.k; ++k) {
      const int32_t j = A.col[k * n + i];
      ax += va[k * n + i] * (dinv[j] * b[j]);
    }
    xn[i] = dinv[i] * b[i] + dinv[i] * (b[i] - ax);
  }
}
template <class R>
__global__ void k_residual_ell(Ell A, const R* b, const R* x, R* r, const int* stop) {
  if (stop && *stop) return;
  const int64_t n = A.n;
  const R* va = (const R*)A.val;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    R ax = 0;
    for (int k = 0; k < A.k; ++k) ax += va[k * n + i] * x[A.col[k * n + i]];
    r[i] = b[i] - ax;
  }
}
// y = M x (add: y += M x)
template <class R>
__global__ void k_spmv_ell(Ell M, const R* x, R* y, int add, const int* stop) {
  if (stop && *stop) return;
  const int64_t n = M.n;
  const R* va = (const R*)M.val;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    R v = 0;
    for (int k = 0; k < M.k; ++k) v += va[k * n + i] * x[M.col[k * n + i]];
    y[i] = add ? y[i] + v : v;
  }
}
template <class R>
__global__ void k_coarse(int64_t n, const double* Ci, const R* b, R* x, const int* stop) {
  if (stop && *stop) return;
  // one warp per row
  const int lane = threadIdx.x & 31;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double v = 0;
    for (int64_t j = lane; j < n; j += 32) v += Ci[i * n + j] * (double)b[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) x[i] = (R)v;
  }
}

template <class R>
static void vcycle(PrecData<R>& P, int l, const int* stop, cudaStream_t st) {
  const int bs = 256;
  const GmgLevel& G = P.lev[l];
  auto grid = [&](int64_t n) { return (unsigned)((n + bs - 1) / bs < 4096 ? (n + bs - 1) / bs : 4096); };
  if (G.n == 0) return;
  if (l == 0) {
    unsigned g = (unsigned)((G.n * 32 + bs - 1) / bs);
    if (g > 4096) g = 4096;
    k_coarse<R><<<g, bs, 0, st>>>(G.n, P.coarse_inv, P.pb[0], P.px[0], stop);
    note_launch();
    return;
  }

  const R* di = (const R*)G.dl1inv;
  const GmgLevel& Gc = P.lev[l - 1];
  R* x = P.px[l];
  R* xt = P.ptmp[l];
  // pre-smoothing from x = 0: two sweeps per pass, a last single sweep if their number is odd
  int sw = 0;
  if (P.gmg_smooth >= 2) {
    k_jacobi2_from_b<R><<<grid(G.n), bs, 0, st>>>(G.A, di, P.pb[l], x, stop);
    note_launch();
    sw = 2;
  }
  for (; sw < P.gmg_smooth; ++sw) {
    k_jacobi<R><<<grid(G.n), bs, 0, st>>>(G.A, di, P.pb[l], x, xt, sw == 0, stop);
    note_launch();
    R* tmp = x; x = xt; xt = tmp;
  }
  // b_{l-1} = R (b - A x)
  k_residual_ell<R><<<grid(G.n), bs, 0, st>>>(G.A, P.pb[l], x, P.pr[l], stop);
  note_launch();
  k_spmv_ell<R><<<grid(Gc.n), bs, 0, st>>>(G.Rt, P.pr[l], P.pb[l - 1], 0, stop);
  note_launch();
  vcycle(P, l - 1, stop, st);
  // x += P x_{l-1}, post-smoothing
  k_spmv_ell<R><<<grid(G.n), bs, 0, st>>>(G.P, P.px[l - 1], x, 1, stop);
  note_launch();
  for (int s2 = 0; s2 < P.gmg_smooth; ++s2) {
    k_jacobi<R><<<grid(G.n), bs, 0, st>>>(G.A, di, P.pb[l], x, xt, 0, stop);
    note_launch();
    R* tmp = x; x = xt; xt = tmp;
  }
  if (x != P.px[l]) cudaMemcpyAsync(P.px[l], x, sizeof(R) * G.n, cudaMemcpyDeviceToDevice, st);
}

// Diagnostics mode: synchronise after a preconditioner launch and report a failure by name.
template <class R>
static void dbg_sync(const PrecData<R>& P, cudaStream_t st, const char* what) {
  if (!P.debug) return;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "mcs diagnostics: %s failed: %s\n", what, cudaGetErrorString(e));
    std::fflush(stderr);
    return;
  }
  int hv[4] = {0, 0, 0, 0};
  cudaMemcpy(hv, P.dbg, sizeof(hv), cudaMemcpyDeviceToHost);
  if (hv[0]) {
    std::fprintf(stderr, "mcs diagnostics: %s: check %d failed (block %d, offset %d, size %d)\n", what, hv[0], hv[1],
                 hv[2], hv[3]);
    std::fflush(stderr);
  }
}

// Warp-per-facet variant of the facet step (same arithmetic): every warp walks its own facets
// (records f, f + W, ... of the colour range, W = number of warps) through a private two-stage
// cp.async pipeline, so no block-wide barrier is needed.  Per facet: lanes (row, part) form the
// 2 m_F slab-row dot products in L = 32 / (2 m_F) parts joined by shuffles, lanes t < m_F form r_F
// and D_F^{-1} r_F (r broadcast by shuffles).  Stage layout per warp (16-byte aligned): stream
// block [fs_stride], gathered segments [2][d+1][fs], b [fs], tb [fs].
template <class S, class R>
__host__ __device__ inline int warp_stage_elems(const S& s) {
  const int fs = facet_stride(s, (int)sizeof(R));
  return fs_stride(s) + 2 * (s.d + 1) * fs + 2 * fs;
}
template <class R, class S, bool UPDATE>
__global__ void __launch_bounds__(256) k_facet_step_warp(S s, Layout L, const R* __restrict__ Fs,
                                                         const R* __restrict__ b, const R* __restrict__ tb, R* x,
                                                         R* rr, const int* __restrict__ rec, int64_t n,
                                                         const int* stop, int* err) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char swr[];
  const int mF = s.mF, dp1 = s.d + 1, slab = slab_pad(s), fss = fs_stride(s), nc = s.n_c;
  const int fs = facet_stride(s, (int)sizeof(R));
  const int se = warp_stage_elems<S, R>(s);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  R* wbase = reinterpret_cast<R*>(swr) + (size_t)wib * 2 * se;
  // the two mbarriers of this warp's stages follow all warps' stages
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<R*>(swr) + (size_t)(blockDim.x >> 5) * 2 * se) + 2 * wib;
  const unsigned sbytes = (unsigned)((UPDATE ? fss : 2 * slab) * (int)sizeof(R));   // stream bytes per facet
  if (lane == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    mbar_init_fence();
  }
  __syncwarp();
  unsigned phases = 0u;   // bit st: parity of the next phase of stage st's mbarrier
  constexpr int V = 16 / (int)sizeof(R);
  const int cx = fs / V;
  const int rows = 2 * mF;
  const int LP = rows <= 16 ? 2 : 1;            // lanes per row
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t f0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const uint64_t pol = l2_evict_first_policy();

  auto issue = [&](int st, int64_t f, int myrec) {
    R* Sb = wbase + st * se;
    R* Xs = Sb + fss;
    R* Bs = Xs + 2 * dp1 * fs;
    R* Ts = Bs + fs;
    const R* src = Fs + f * fss;
    // record fields to every lane first (all 32 lanes shuffle, outside the lane-dependent loops)
    int gseg[8];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) gseg[k2] = __shfl_sync(0xffffffffu, myrec, 5 + k2);
    const int r = __shfl_sync(0xffffffffu, myrec, 0);
    // the facet's stream block (contiguous, 16-byte aligned): one bulk copy on the stage's mbarrier
    if (lane == 0) {
      mbar_expect_tx(bars + st, sbytes);
      bulk_copy_g2s(Sb, src, sbytes, bars + st, pol);
    }
    for (int q = lane; q < 2 * dp1 * cx; q += 32) {
      const int seg = q / cx, ch = q - seg * cx;   // seg = side*dp1 + local facet
      const int g = gseg[seg];
      R* dst = Xs + seg * fs + ch * V;
      if (g >= 0) cp_async16(dst, x + (int64_t)g * fs + ch * V);
      else *reinterpret_cast<int4*>(dst) = make_int4(0, 0, 0, 0);
    }
    for (int q = lane; q < 2 * cx; q += 32) {
      const int which = q / cx, ch = q - which * cx;
      R* dst = (which ? Ts : Bs) + ch * V;
      const R* sp = which ? tb : b;
      if (sp) cp_async16(dst, sp + (int64_t)r * fs + ch * V);
      else *reinterpret_cast<int4*>(dst) = make_int4(0, 0, 0, 0);
    }
  };
  // the shuffles in issue() need every lane, so all lanes run the loop the same number of times
  int st = 0;
  // records two facets ahead: the load of the next-but-one record overlaps this facet's work
  int rec_a = (f0 < n && lane < 16) ? rec[f0 * 16 + lane] : -1;            // facet f
  int rec_b = (f0 + W < n && lane < 16) ? rec[(f0 + W) * 16 + lane] : -1;  // facet f + W
  if (f0 < n) issue(0, f0, rec_a);
  cp_async_commit();
  for (int64_t f = f0; f < n; f += W) {
    const int rec_cur = rec_a;
    const int64_t fn = f + W;
    if (fn < n) issue(st ^ 1, fn, rec_b);
    cp_async_commit();
    rec_a = rec_b;
    rec_b = (fn + W < n && lane < 16) ? rec[(fn + W) * 16 + lane] : -1;
    cp_async_wait_group<1>();
    // bounded wait for the stream block (about a second): on expiry the error flag is set, the
    // other stage's copy is waited for (bounded too) and the warp stops
    bool got = true;
    if (lane == 0) got = mbar_wait_bounded(bars + st, (phases >> st) & 1u, 1000000000ull);
    got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
    if (!got) {
      if (lane == 0) {
        atomicExch(err, 1);
        if (fn < n) mbar_wait_bounded(bars + (st ^ 1), (phases >> (st ^ 1)) & 1u, 1000000000ull);
      }
      cp_async_wait_all();
      __syncwarp();
      return;
    }
    __syncwarp();
    phases ^= 1u << st;
    const R* Sb = wbase + st * se;
    const R* Xs = Sb + fss;
    const R* Bs = Xs + 2 * dp1 * fs;
    const R* Ts = Bs + fs;
    // slab-row dot products: lane -> (row = side*mF + t, part)
    R y = 0;
    const int row = lane / LP, part = lane - row * LP;
    if (row < rows) {
      const int side = row >= mF ? 1 : 0, t = row - side * mF;
      const R* A = Sb + side * slab + t;
      const R* xv = Xs + side * dp1 * fs;
      for (int c = part; c < nc; c += LP) {
        const int fl = c / mF, tt = c - fl * mF;
        y += A[c * mF] * xv[fl * fs + tt];
      }
    }
    if (LP == 2) y += __shfl_xor_sync(0xffffffffu, y, 1);
    // r_F on lanes t < mF
    const R y0 = __shfl_sync(0xffffffffu, y, (lane < mF ? lane : 0) * LP);
    const R y1 = __shfl_sync(0xffffffffu, y, ((lane < mF ? lane : 0) + mF) * LP);
    const R rv = lane < mF ? Bs[lane] - Ts[lane] - y0 - y1 : (R)0;
    const int r = __shfl_sync(0xffffffffu, rec_cur, 0);
    if (UPDATE) {
      const int f0l = __shfl_sync(0xffffffffu, rec_cur, 3);   // local index of the facet in side 0
      const R* Dr = Sb + 2 * slab + (lane < mF ? lane : 0) * mF;
      R v = 0;
      for (int j = 0; j < mF; ++j) v += Dr[j] * __shfl_sync(0xffffffffu, rv, j);
      if (lane < mF && r >= 0) x[(int64_t)r * fs + lane] = Xs[f0l * fs + lane] + v;
    } else {
      if (lane < mF && r >= 0) rr[(int64_t)r * fs + lane] = rv;
    }
    __syncwarp();
    st ^= 1;
  }
  cp_async_wait_all();
}

// Facet step for facet blocks too large to stage in shared memory (3D k >= 5): one block per facet
// (grid stride over the records), the gathered segments, b and tb in shared memory, the two slabs and
// D_F^{-1} read from global memory directly (slab column c, row t at c*mF + t: lanes of consecutive
// t read consecutive addresses; D_F^{-1} is symmetric, so its column t is read for row t).  Same
// arithmetic as k_facet_step.  Shared memory: [2][d+1][fs] segments, b, tb, [P][2 m_F] partial sums.
template <class R, class S, bool UPDATE>
__global__ void __launch_bounds__(256) k_facet_step_direct(S s, Layout L, const R* __restrict__ Fs,
                                                           const R* __restrict__ b, const R* __restrict__ tb, R* x,
                                                           R* rr, const int* __restrict__ rec, int64_t n,
                                                           const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char sdr[];
  const int mF = s.mF, dp1 = s.d + 1, slab = slab_pad(s), fss = fs_stride(s), nc = s.n_c;
  const int fs = facet_stride(s, (int)sizeof(R));
  const int rows = 2 * mF;
  const int P = blockDim.x / rows > 0 ? blockDim.x / rows : 1;   // parts per row
  R* Xs = reinterpret_cast<R*>(sdr);          // [2][d+1][fs]
  R* Bs = Xs + 2 * dp1 * fs;                  // [fs]
  R* Ts = Bs + fs;                            // [fs]
  R* Yp = Ts + fs;                            // [P][rows]
  R* Rv = Yp + P * rows;                      // [mF] r_F
  const int tid = threadIdx.x;
  for (int64_t f = blockIdx.x; f < n; f += gridDim.x) {
    const int* rc = rec + f * 16;
    const int r = rc[0];
    for (int q = tid; q < 2 * dp1 * fs; q += blockDim.x) {
      const int seg = q / fs, t = q - seg * fs;          // seg = side*dp1 + local facet
      const int g = rc[5 + seg];
      Xs[q] = (g >= 0 && t < mF) ? x[(int64_t)g * fs + t] : (R)0;
    }
    for (int q = tid; q < fs; q += blockDim.x) {
      Bs[q] = (r >= 0 && q < mF) ? b[(int64_t)r * fs + q] : (R)0;
      Ts[q] = (r >= 0 && q < mF && tb) ? tb[(int64_t)r * fs + q] : (R)0;
    }
    __syncthreads();
    const R* blk = Fs + f * (int64_t)fss;
    for (int q = tid; q < P * rows; q += blockDim.x) {
      const int part = q / rows, row = q - part * rows;
      const int side = row >= mF ? 1 : 0, t = row - side * mF;
      const R* A = blk + side * slab + t;
      const R* xv = Xs + side * dp1 * fs;
      R y = 0;
      for (int c = part; c < nc; c += P) {
        const int fl = c / mF, tt = c - fl * mF;
        y += A[(int64_t)c * mF] * xv[fl * fs + tt];
      }
      Yp[q] = y;
    }
    __syncthreads();
    for (int t = tid; t < mF; t += blockDim.x) {
      R y = 0;
      for (int part = 0; part < P; ++part) y += Yp[part * rows + t] + Yp[part * rows + mF + t];
      const R v = Bs[t] - Ts[t] - y;
      if (UPDATE) Rv[t] = v;
      else if (r >= 0) rr[(int64_t)r * fs + t] = v;
    }
    if (UPDATE) {
      __syncthreads();
      const R* Di = blk + 2 * slab;
      const int f0 = rc[3];                      // local index of the facet in side 0
      for (int t = tid; t < mF; t += blockDim.x) {
        R v = 0;
        for (int j = 0; j < mF; ++j) v += Di[j * mF + t] * Rv[j];
        if (r >= 0) x[(int64_t)r * fs + t] = Xs[f0 * fs + t] + v;
      }
    }
    __syncthreads();
  }
}

// Forward colour sweep with a maintained residual (the sweeps of the multiplicative ASP before the
// coarse correction, which start from x = 0).  Besides x the sweep keeps, per interior facet H and side
// s, a partial residual q_s[H]: q_0 starts as b - tb and q_1 as 0, and every block update subtracts
// A^d_T[H, F] delta_F from the slot of H's element T, so that r_F = q_0[F] + q_1[F] equals
// b_F - tb_F - sum_{T ni F} A^d_T[F, :] x_T at every step.  After the block solve delta = D_F^{-1} r_F
// the facet pushes -A^d_T[H, F] delta = -(A^d_T[F, H])^T delta into the slot of every facet H of both
// its elements; A^d_T[F, H] are the columns of its own slabs, already in shared memory, so the sweep
// reads the same stream as the row-product form and forms no row products.  Facets of one colour share
// no element, so each (H, side) slot has one writer per launch and is read by no other facet of the
// launch.  After the last forward colour q_0 + q_1 is the residual, which the coarse correction needs.
// Record field [13]: bit side*(d+1) + f set when element rec[1 + side] is side 1 of the facet
// H = rec[5 + side*(d+1) + f].  One warp per facet as in k_facet_step_warp, with a two-stage pipeline:
// the stream block by one bulk copy on an mbarrier (bounded wait), the q segments of the 2(d+1) facets of
// both elements and x_F by cp.async; the records are loaded two facets ahead.  xin = nullptr: x = 0
// before the launch (the first sweep).
template <class S, class R>
__host__ __device__ inline int push_stage_elems(const S& s) {
  const int fs = facet_stride(s, (int)sizeof(R));
  return fs_stride(s) + 2 * (s.d + 1) * fs + fs;
}
template <class R, class S>
__global__ void __launch_bounds__(256) k_facet_push_warp(S s, const R* __restrict__ Fs, const R* xin, R* x, R* q0,
                                                         R* q1, const int* __restrict__ rec, int64_t n,
                                                         const int* stop, int* err) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char swq[];
  const int mF = s.mF, dp1 = s.d + 1, slab = slab_pad(s), fss = fs_stride(s), nc = s.n_c;
  const int fs = facet_stride(s, (int)sizeof(R));
  const int se = push_stage_elems<S, R>(s);
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // per warp: two stages and a scratch of 32 entries (r_F, then delta), then all warps' mbarriers
  R* wbase = reinterpret_cast<R*>(swq) + (size_t)wib * (2 * se + 32);
  R* Rs = wbase + 2 * se;
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<R*>(swq) + (size_t)nw * (2 * se + 32)) + 2 * wib;
  const unsigned sbytes = (unsigned)(fss * (int)sizeof(R));
  if (lane == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    mbar_init_fence();
  }
  __syncwarp();
  unsigned phases = 0u;   // bit st: parity of the next phase of stage st's mbarrier
  constexpr int V = 16 / (int)sizeof(R);
  const int cx = fs / V;
  const int nseg = 2 * dp1;
  const int64_t W = (int64_t)gridDim.x * nw;
  const int64_t f0 = (int64_t)blockIdx.x * nw + wib;
  const uint64_t pol = l2_evict_first_policy();
  const bool vec = ((mF * (int)sizeof(R)) & 15) == 0;   // slab columns and D_F^{-1} rows on 16-byte boundaries
  // the lane's slab columns c = 32u + lane (2 n_c <= 128): offset in the stage, segment, mode
  int c_off[4], c_seg[4], c_tp[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = 32 * u + lane;
    const bool act = c < 2 * nc;
    const int side = (act && c >= nc) ? 1 : 0;
    const int cc = act ? c - side * nc : 0;
    const int fl = cc / mF;
    c_off[u] = side * slab + cc * mF;
    c_seg[u] = act ? side * dp1 + fl : -1;
    c_tp[u] = cc - fl * mF;
  }
  // sum_{t < mF} a[t] b[t] in the order t = 0, 1, ... (b a register array when REG)
  auto dot_m = [&](const R* a, const R* bv) -> R {
    R acc = 0;
    if (vec) {
#pragma unroll
      for (int t0 = 0; t0 < 16; t0 += V) {
        if (t0 < mF) {
          if constexpr (sizeof(R) == 4) {
            const float4 A = *reinterpret_cast<const float4*>(a + t0);
            const float4 B = *reinterpret_cast<const float4*>(bv + t0);
            acc += A.x * B.x;
            acc += A.y * B.y;
            acc += A.z * B.z;
            acc += A.w * B.w;
          } else {
            const double2 A = *reinterpret_cast<const double2*>(a + t0);
            const double2 B = *reinterpret_cast<const double2*>(bv + t0);
            acc += A.x * B.x;
            acc += A.y * B.y;
          }
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < 16; ++t)
        if (t < mF) acc += a[t] * bv[t];
    }
    return acc;
  };

  // stage: [stream block | q segments of the 2(d+1) facets of both elements | x_F]
  auto issue = [&](int st, int64_t f, int myrec) {
    R* Sb = wbase + st * se;
    R* Qs = Sb + fss;
    R* Xs = Qs + nseg * fs;
    int gseg[8];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) gseg[k2] = __shfl_sync(0xffffffffu, myrec, 5 + k2);
    const int bits = __shfl_sync(0xffffffffu, myrec, 13);
    const int r = __shfl_sync(0xffffffffu, myrec, 0);
    if (lane == 0) {
      mbar_expect_tx(bars + st, sbytes);
      bulk_copy_g2s(Sb, Fs + f * fss, sbytes, bars + st, pol);
    }
    for (int q = lane; q < nseg * cx; q += 32) {
      const int seg = q / cx, ch = q - seg * cx;   // seg = side*dp1 + local facet
      const int g = gseg[seg];
      R* dst = Qs + seg * fs + ch * V;
      if (g >= 0) cp_async16(dst, (((bits >> seg) & 1) ? q1 : q0) + (int64_t)g * fs + ch * V);
      else *reinterpret_cast<int4*>(dst) = make_int4(0, 0, 0, 0);
    }
    for (int q = lane; q < cx; q += 32) {
      R* dst = Xs + q * V;
      if (xin && r >= 0) cp_async16(dst, xin + (int64_t)r * fs + q * V);
      else *reinterpret_cast<int4*>(dst) = make_int4(0, 0, 0, 0);
    }
  };
  int st = 0;
  int rec_a = (f0 < n && lane < 16) ? rec[f0 * 16 + lane] : -1;            // facet f
  int rec_b = (f0 + W < n && lane < 16) ? rec[(f0 + W) * 16 + lane] : -1;  // facet f + W
  if (f0 < n) issue(0, f0, rec_a);
  cp_async_commit();
  for (int64_t f = f0; f < n; f += W) {
    const int rec_cur = rec_a;
    const int64_t fn = f + W;
    if (fn < n) issue(st ^ 1, fn, rec_b);
    cp_async_commit();
    rec_a = rec_b;
    rec_b = (fn + W < n && lane < 16) ? rec[(fn + W) * 16 + lane] : -1;
    cp_async_wait_group<1>();
    bool got = true;
    if (lane == 0) got = mbar_wait_bounded(bars + st, (phases >> st) & 1u, 1000000000ull);
    got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
    if (!got) {
      if (lane == 0) {
        atomicExch(err, 1);
        if (fn < n) mbar_wait_bounded(bars + (st ^ 1), (phases >> (st ^ 1)) & 1u, 1000000000ull);
      }
      cp_async_wait_all();
      __syncwarp();
      return;
    }
    __syncwarp();
    phases ^= 1u << st;
    const R* Sb = wbase + st * se;
    const R* Qs = Sb + fss;
    const R* Xs = Qs + nseg * fs;
    const int r = __shfl_sync(0xffffffffu, rec_cur, 0);
    const int fl0 = __shfl_sync(0xffffffffu, rec_cur, 3);
    const int fl1 = __shfl_sync(0xffffffffu, rec_cur, 4);
    const int bits = __shfl_sync(0xffffffffu, rec_cur, 13);
    // r_F on lanes t < mF (the facet's own q slots are the segments of its local facets in both
    // elements) into the scratch, then delta = D_F^{-1} r_F (row t on lane t) into the scratch
    if (lane < mF) {
      R rv = Qs[fl0 * fs + lane];
      if (fl1 >= 0) rv += Qs[(dp1 + fl1) * fs + lane];
      Rs[lane] = rv;
    }
    __syncwarp();
    if (lane < mF) {
      const R v = dot_m(Sb + 2 * slab + lane * mF, Rs);
      Rs[16 + lane] = v;
      if (r >= 0) x[(int64_t)r * fs + lane] = Xs[lane] + v;
    }
    __syncwarp();
    R dl[16];   // delta on every lane (m_F <= 16)
#pragma unroll
    for (int t = 0; t < 16; ++t) dl[t] = t < mF ? Rs[16 + t] : (R)0;
    // push: the lane's columns of the slabs against delta
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int seg = c_seg[u] < 0 ? 0 : c_seg[u];
      const int H = __shfl_sync(0xffffffffu, rec_cur, 5 + seg);
      if (c_seg[u] < 0 || H < 0) continue;
      const R* col = Sb + c_off[u];
      R val = 0;
      if (vec) {
#pragma unroll
        for (int t0 = 0; t0 < 16; t0 += V) {
          if (t0 < mF) {
            if constexpr (sizeof(R) == 4) {
              const float4 a = *reinterpret_cast<const float4*>(col + t0);
              val += a.x * dl[t0];
              val += a.y * dl[t0 + 1];
              val += a.z * dl[t0 + 2];
              val += a.w * dl[t0 + 3];
            } else {
              const double2 a = *reinterpret_cast<const double2*>(col + t0);
              val += a.x * dl[t0];
              val += a.y * dl[t0 + 1];
            }
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (t < mF) val += col[t] * dl[t];
      }
      R* qd = ((bits >> seg) & 1) ? q1 : q0;
      qd[(int64_t)H * fs + c_tp[u]] = Qs[seg * fs + c_tp[u]] - val;
    }
    __syncwarp();
    st ^= 1;
  }
  cp_async_wait_all();
}

// q_0 = b - tb, q_1 = 0 (entries of all facet slots): the partial residuals before a forward sweep from
// x = 0.
template <class R>
__global__ void k_push_init(int64_t nint, int fs, const R* __restrict__ b, const R* __restrict__ tb, R* q0, R* q1,
                            const int* stop) {
  if (stop && *stop) return;
  const int64_t total = nint * fs;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    q0[i] = b[i] - (tb ? tb[i] : (R)0);
    q1[i] = (R)0;
  }
}

template <class R>
int facet_push_warps(const ElemSizes& s) {
  if (2 * s.mF > 32) return 0;
  if ((size_t)fs_stride(s) * sizeof(R) < 4096) return 0;   // small blocks: the batched row-product kernel
  for (int nw = 8; nw >= 2; nw /= 2)
    if ((size_t)nw * (2 * push_stage_elems<ElemSizes, R>(s) + 32) * sizeof(R) + (size_t)nw * 2 * sizeof(uint64_t) <=
        100 * 1024)
      return nw;
  return 0;
}
template int facet_push_warps<float>(const ElemSizes&);
template int facet_push_warps<double>(const ElemSizes&);

template <class R>
static cudaError_t facet_push(const ElemSizes& s, const DevMesh& m, const Layout& L, PrecData<R>& P, const R* xin,
                              R* x, int64_t first, int64_t n, const int* stop, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (L.fstride != facet_stride(s, (int)sizeof(R)) || P.push_warps <= 0 || !P.q0 || !P.q1)
    return cudaErrorInvalidValue;
  const int nw = P.push_warps;
  const size_t wsm =
      (size_t)nw * (2 * push_stage_elems<ElemSizes, R>(s) + 32) * sizeof(R) + (size_t)nw * 2 * sizeof(uint64_t);
  const int* ri = reinterpret_cast<const int*>(m.frec + first * 4);
  const R* fs0 = P.Fs + first * (int64_t)fs_stride(s);
  dispatch_sizes(s, [&](auto sz) {
    using SZ = decltype(sz);
    // occupancy cached per shared-memory size (the run-time-size instantiation serves several (d, k))
    static std::atomic<int64_t> cached{0};   // (wsm << 8) | blocks per SM
    int64_t c = cached.load(std::memory_order_acquire);
    if ((c >> 8) != (int64_t)wsm) {
      cudaFuncSetAttribute(k_facet_push_warp<R, SZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_facet_push_warp<R, SZ>, nw * 32, wsm);
      c = ((int64_t)wsm << 8) | (int64_t)(occ > 0 ? (occ < 255 ? occ : 255) : 1);
      cached.store(c, std::memory_order_release);
    }
    int64_t blocks = (int64_t)sm_count() * (c & 255);
    const int64_t need = (n + nw - 1) / nw;
    if (blocks > need) blocks = need;
    prof_begin(PROF_FACET_PUSH, st);
    note_launch();
    k_facet_push_warp<R, SZ><<<(unsigned)blocks, nw * 32, wsm, st>>>(sz, fs0, xin, x, P.q0, P.q1, ri, n, stop,
                                                                      P.err);
    // algorithmic bytes per facet as for the row-product update (the stream block, b, tb, x_F read and
    // written; here q_0, q_1 of the facet stand for b, tb); the q segments of the neighbours, like the
    // gathered x there, are L2-resident vectors
    const double per = 2.0 * s.mF * s.n_c + (double)s.mF * s.mF + 4.0 * s.mF;
    prof_end(PROF_FACET_PUSH, (double)n * per * sizeof(R), 2.0 * (double)n * (2.0 * s.mF * s.n_c + s.mF * s.mF), st);
  });
  dbg_sync(P, st, "k_facet_push_warp");
  return cudaGetLastError();
}

template <class R>
static size_t facet_step_smem(const ElemSizes& s, int FB, bool update) {
  (void)update;
  const int fs = facet_stride(s, (int)sizeof(R));
  const size_t stage = (size_t)FB * 16 * sizeof(int) + (size_t)FB * fs_stride(s) * sizeof(R) +
                       (size_t)FB * 2 * (s.d + 1) * fs * sizeof(R) + 2 * (size_t)FB * fs * sizeof(R);
  return 2 * stage + (size_t)FB * 3 * s.mF * sizeof(R) + 16;
}

template <class R>
static cudaError_t facet_step(const ElemSizes& s, const DevMesh& m, const Layout& L, PrecData<R>& P, const R* b,
                              const R* tb, R* x, R* rr, int64_t first, int64_t n, bool update,
                              const int* stop, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (L.fstride != facet_stride(s, (int)sizeof(R))) return cudaErrorInvalidValue;  // preconditioner layout only
  const int4* rec0 = m.frec + first * 4;
  const R* fs0 = P.Fs + first * (int64_t)fs_stride(s);
  {
    // warp-per-facet kernel for large facet blocks (at least 4 KB of stream per facet: 3D; measured
    // faster there, slower than the batched block kernel for the 1.4 KB blocks of 2D k = 3), when the
    // 2 m_F rows fit a warp and the stages of 8 (else 4) warps fit in 100 KB
    int nwarp = 0;
    size_t wsm = 0;
    if ((size_t)fs_stride(s) * sizeof(R) >= 4096 && 2 * s.mF <= 32) {
      for (int w = 8; w >= 4; w /= 2) {
        const size_t b_ = (size_t)w * 2 * warp_stage_elems<ElemSizes, R>(s) * sizeof(R) + (size_t)w * 2 * sizeof(uint64_t);
        if (b_ <= 100 * 1024) {
          nwarp = w;
          wsm = b_;
          break;
        }
      }
    }
    if (nwarp > 0) {
      bool done = false;
      dispatch_sizes(s, [&](auto sz) {
        using SZ = decltype(sz);
        // occupancy cached per (update, shared-memory size)
        static std::atomic<int64_t> cached[2];   // (wsm << 8) | blocks per SM
        const int ui = update ? 1 : 0;
        int64_t c = cached[ui].load(std::memory_order_acquire);
        if ((c >> 8) != (int64_t)wsm) {
          cudaFuncSetAttribute(k_facet_step_warp<R, SZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               200 * 1024);
          cudaFuncSetAttribute(k_facet_step_warp<R, SZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               200 * 1024);
          int occ = 0;
          if (update)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_facet_step_warp<R, SZ, true>, nwarp * 32, wsm);
          else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_facet_step_warp<R, SZ, false>, nwarp * 32, wsm);
          c = ((int64_t)wsm << 8) | (int64_t)(occ > 0 ? (occ < 255 ? occ : 255) : 1);
          cached[ui].store(c, std::memory_order_release);
        }
        int64_t blocks = (int64_t)sm_count() * (c & 255);
        const int64_t need = (n + nwarp - 1) / nwarp;
        if (blocks > need) blocks = need;
        const int cls = update ? PROF_FACET_GS : PROF_FACET_RES;
        prof_begin(cls, st);
        note_launch();
        const int* ri = reinterpret_cast<const int*>(rec0);
        if (update)
          k_facet_step_warp<R, SZ, true><<<(unsigned)blocks, nwarp * 32, wsm, st>>>(sz, L, fs0, b, tb, x, rr, ri, n,
                                                                                      stop, P.err);
        else
          k_facet_step_warp<R, SZ, false><<<(unsigned)blocks, nwarp * 32, wsm, st>>>(sz, L, fs0, b, tb, x, rr, ri, n,
                                                                                       stop, P.err);
        const double per = update ? (2.0 * s.mF * s.n_c + (double)s.mF * s.mF + 4.0 * s.mF)
                                  : (2.0 * s.mF * s.n_c + 3.0 * s.mF);
        prof_end(cls, (double)n * per * sizeof(R),
                 2.0 * (double)n * (2.0 * s.mF * s.n_c + (update ? s.mF * s.mF : 0)), st);
        done = true;
      });
      if (done && !P.debug) return cudaGetLastError();
      if (done) {
        dbg_sync(P, st, update ? "k_facet_step_warp (update)" : "k_facet_step_warp (residual)");
        return cudaGetLastError();
      }
    }
  }
  if (facet_step_smem<R>(s, 1, update) > 200 * 1024) {
    // one facet's stages do not fit: the unstaged kernel
    const int fs = facet_stride(s, (int)sizeof(R));
    const int rows = 2 * s.mF, parts = 256 / rows > 0 ? 256 / rows : 1;
    const size_t sm = ((size_t)(2 * (s.d + 1) + 2) * fs + (size_t)parts * rows + s.mF) * sizeof(R) + 16;
    int64_t blocks = (int64_t)sm_count() * 8;
    if (blocks > n) blocks = n;
    const int* ri = reinterpret_cast<const int*>(rec0);
    const int cls = update ? PROF_FACET_GS : PROF_FACET_RES;
    prof_begin(cls, st);
    note_launch();
    if (update)
      k_facet_step_direct<R, ElemSizes, true><<<(unsigned)blocks, 256, sm, st>>>(s, L, fs0, b, tb, x, rr, ri, n, stop);
    else
      k_facet_step_direct<R, ElemSizes, false><<<(unsigned)blocks, 256, sm, st>>>(s, L, fs0, b, tb, x, rr, ri, n, stop);
    const double per = update ? (2.0 * s.mF * s.n_c + (double)s.mF * s.mF + 4.0 * s.mF) : (2.0 * s.mF * s.n_c + 3.0 * s.mF);
    prof_end(cls, (double)n * per * sizeof(R), 2.0 * (double)n * (2.0 * s.mF * s.n_c + (update ? s.mF * s.mF : 0)), st);
    dbg_sync(P, st, update ? "k_facet_step_direct (update)" : "k_facet_step_direct (residual)");
    return cudaGetLastError();
  }
  // small batches (at most 40 KB of stages, at least 4 facets) in narrow blocks, so that several
  // blocks share an SM and their barriers overlap; else up to 96 KB
  int FB = 128 / (2 * s.mF);
  if (FB < 1) FB = 1;
  while (FB > 1 && facet_step_smem<R>(s, FB, update) > 40 * 1024) --FB;
  int threads = 128;
  if (FB < 4) {
    FB = 256 / (2 * s.mF);
    if (FB < 1) FB = 1;
    while (FB > 1 && facet_step_smem<R>(s, FB, update) > 96 * 1024) --FB;
    threads = 256;
  }
  const bool tuned = P.fb > 0 && P.fthreads > 0 && facet_step_smem<R>(s, P.fb, update) <= 160 * 1024;
  if (tuned) {
    FB = P.fb;
    threads = P.fthreads;
  }
  const size_t sm = facet_step_smem<R>(s, FB, update);
  const int64_t nb = (n + FB - 1) / FB;
  const int4* rec = m.frec + first * 4;
  const R* fsrc = P.Fs + first * (int64_t)fs_stride(s);
  const int64_t fs_avail = (L.nint - first) * (int64_t)fs_stride(s);
  dispatch_sizes(s, [&](auto sz) {
    using SZ = decltype(sz);
    static std::atomic<int> per_sm[2];
    const int ui = update ? 1 : 0;
    if (!per_sm[ui].load(std::memory_order_acquire)) {
      cudaFuncSetAttribute(k_facet_step<R, SZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(k_facet_step<R, SZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      int occ = 0;
      if (update) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_facet_step<R, SZ, true>, threads, sm);
      else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_facet_step<R, SZ, false>, threads, sm);
      per_sm[ui].store(occ > 0 ? occ : 1, std::memory_order_release);
    }
    int occ_now = per_sm[ui].load(std::memory_order_acquire);
    if (tuned) {   // the cached occupancy belongs to the formula's shape
      occ_now = 0;
      if (update) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_now, k_facet_step<R, SZ, true>, threads, sm);
      else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_now, k_facet_step<R, SZ, false>, threads, sm);
      if (occ_now < 1) occ_now = 1;
    }
    int64_t blocks = (int64_t)sm_count() * occ_now;
    if (blocks > nb) blocks = nb;
    const int cls = update ? PROF_FACET_GS : PROF_FACET_RES;
    prof_begin(cls, st);
    note_launch();
    if (update)
      k_facet_step<R, SZ, true><<<(unsigned)blocks, threads, sm, st>>>(sz, m, L, fsrc, b, tb, x, rr, rec, n, FB, stop,
                                                                        P.dbg, fs_avail, (int)sm);
    else
      k_facet_step<R, SZ, false><<<(unsigned)blocks, threads, sm, st>>>(sz, m, L, fsrc, b, tb, x, rr, rec, n, FB, stop,
                                                                         P.dbg, fs_avail, (int)sm);
    // algorithmic bytes per facet: the facet's rows of A^d from both elements, D_F^{-1}, b, tb,
    // x_F read and written (update) or rr_F written (residual)
    const double per = update ? (2.0 * s.mF * s.n_c + (double)s.mF * s.mF + 4.0 * s.mF)
                              : (2.0 * s.mF * s.n_c + 3.0 * s.mF);
    prof_end(cls, (double)n * per * sizeof(R), 2.0 * (double)n * (2.0 * s.mF * s.n_c + (update ? s.mF * s.mF : 0)), st);
  });
  dbg_sync(P, st, update ? "k_facet_step (update)" : "k_facet_step (residual)");
  return cudaGetLastError();
}

static int elem_batch(size_t per_elem_bytes) {
  int EB = (int)((32 * 1024) / per_elem_bytes);
  if (EB < 1) EB = 1;
  if (EB > 32) EB = 32;
  return EB;
}

template <class R, bool WITH_BT>
static void elem_prologue(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, PrecData<R>& P,
                          const R* r, const R* zp, R* rin, R* tb, const int* stop, cudaStream_t st) {
  const size_t per = (size_t)(g_stride(s) + s.n_bub + s.n_u + s.n_p) * sizeof(R);
  const bool stage = per + 16 <= 190 * 1024;   // else G is read from global memory, one element per block
  const int EB = stage ? elem_batch(per) : 1;
  const size_t sm = (stage ? per * EB : (size_t)(s.n_bub + s.n_u + s.n_p) * sizeof(R)) + 16;
  const int64_t blocks = (m.ne + EB - 1) / EB;
  dispatch_sizes(s, [&](auto sz) {
    using SZ = decltype(sz);
    static std::atomic<bool> set{false};
    if (!set.load(std::memory_order_acquire)) {
      cudaFuncSetAttribute(k_elem_prologue<R, SZ, WITH_BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      set.store(true, std::memory_order_release);
    }
    prof_begin(PROF_PROLOGUE, st);
    if (stage)
      k_elem_prologue<R, SZ, WITH_BT><<<(unsigned)blocks, 256, sm, st>>>(sz, t, m, L, P.G, r, zp, rin, tb, EB, stop);
    else
      k_elem_prologue<R, SZ, WITH_BT, false><<<(unsigned)blocks, 256, sm, st>>>(sz, t, m, L, P.G, r, zp, rin, tb, EB,
                                                                                  stop);
    note_launch();
    prof_end(PROF_PROLOGUE, (double)m.ne * (s.n_bub * s.n_c + 2 * s.n_bub + s.n_c + (WITH_BT ? s.n_p : 0)) * sizeof(R),
             2.0 * (double)m.ne * s.n_bub * s.n_c, st);
  });
}

template <class R, bool WITH_P>
static void elem_epilogue(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, double nu,
                          PrecData<R>& P, const R* rin, const R* r, R* x, R* zp, const int* stop, cudaStream_t st) {
  const size_t per = (size_t)(g_stride(s) + a_stride(s) + s.n_c + 2 * s.n_bub) * sizeof(R);
  const bool stage = per + 16 <= 190 * 1024;   // else G and A_oo^{-1} are read from global memory
  const int EB = stage ? elem_batch(per) : 1;
  const size_t sm = (stage ? per * EB : (size_t)(s.n_c + 2 * s.n_bub) * sizeof(R)) + 16;
  const int64_t blocks = (m.ne + EB - 1) / EB;
  dispatch_sizes(s, [&](auto sz) {
    using SZ = decltype(sz);
    static std::atomic<bool> set{false};
    if (!set.load(std::memory_order_acquire)) {
      cudaFuncSetAttribute(k_elem_epilogue<R, SZ, WITH_P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      set.store(true, std::memory_order_release);
    }
    prof_begin(PROF_EPILOGUE, st);
    if (stage)
      k_elem_epilogue<R, SZ, WITH_P><<<(unsigned)blocks, 256, sm, st>>>(sz, t, m, L, nu, P.G, P.Aoi, rin, r, x, zp, EB,
                                                                         stop);
    else
      k_elem_epilogue<R, SZ, WITH_P, false><<<(unsigned)blocks, 256, sm, st>>>(sz, t, m, L, nu, P.G, P.Aoi, rin, r, x,
                                                                                zp, EB, stop);
    note_launch();
    prof_end(PROF_EPILOGUE, (double)m.ne * (s.n_bub * s.n_c + s.n_bub * s.n_bub + 2 * s.n_bub + s.n_c +
                                             (WITH_P ? 2 * s.n_p : 0)) * sizeof(R),
             2.0 * (double)m.ne * (s.n_bub * s.n_c + s.n_bub * s.n_bub), st);
  });
}

// Additive ASP, facet part: rr_F = b_F - tb_F and x_F = D_F^{-1} rr_F for every interior facet
// (block Jacobi from x = 0); one thread per (facet record, mode).
template <class R, class S>
__global__ void k_facet_jacobi(S s, DevMesh m, Layout L, const R* __restrict__ Fs, const R* __restrict__ b,
                               const R* __restrict__ tb, R* x, R* rr, int64_t n, const int* stop) {
  if (stop && *stop) return;
  const int mF = s.mF, fss = fs_stride(s), slab = slab_pad(s);
  const int64_t fs = L.fstride;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * mF; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / mF;
    const int t = (int)(q - i * mF);
    const int64_t r = m.frec[i * 4].x;
    const R* Di = Fs + i * fss + 2 * slab + t * mF;
    const R* bf = b + r * fs;
    const R* tf = tb + r * fs;
    R v = 0;
    for (int j = 0; j < mF; ++j) v += Di[j] * (bf[j] - tf[j]);
    x[r * fs + t] = v;
    rr[r * fs + t] = bf[t] - tf[t];
  }
}

// Multiplicative ASP on A^d (Sec. 5.2 / 6.1): x_c from the right-hand side b_c - tb_c.
template <class R>
static void asp_core(const ElemSizes& s, const DevMesh& m, const Layout& L, PrecData<R>& P, const R* b, const R* tb,
                     R* x, const int* stop, cudaStream_t st) {
  const int bs = 256;
  const unsigned g = (unsigned)(sm_count() * 8);
  cudaMemsetAsync(x, 0, sizeof(R) * L.n_dd, st);
  if (L.n_hat) cudaMemsetAsync(x + L.off_h, 0, sizeof(R) * L.n_hat, st);
  const int64_t* co = P.colour_off;
  if (P.multiplicative && P.push_warps > 0 && P.q0 && P.q1) {
    // forward sweeps with the maintained residual (from x = 0: q_0 = b - tb, q_1 = 0), then rr = q_0 + q_1
    if (L.nint > 0) {
      k_push_init<R><<<g, bs, 0, st>>>(L.nint, L.fstride, b, tb, P.q0, P.q1, stop);
      note_launch();
      dbg_sync(P, st, "k_push_init");
    }
    for (int sw = 0; sw < P.smooth; ++sw)
      for (int c = 0; c < P.ncol; ++c)
        facet_push<R>(s, m, L, P, sw == 0 ? nullptr : x, x, co[c], co[c + 1] - co[c], stop, st);   // sweep 0: x_F = 0
    // the residual rr = q_0 + q_1 is summed where E^d^T reads it
  } else if (P.multiplicative) {
    for (int sw = 0; sw < P.smooth; ++sw)
      for (int c = 0; c < P.ncol; ++c)
        facet_step<R>(s, m, L, P, b, tb, x, nullptr, co[c], co[c + 1] - co[c], true, stop, st);
    facet_step<R>(s, m, L, P, b, tb, x, P.rr, 0, L.nint, false, stop, st);
  } else if (L.nint > 0) {  // additive: block Jacobi, and the coarse correction of the same residual
    dispatch_sizes(s, [&](auto sz) {
      k_facet_jacobi<R, decltype(sz)><<<g, bs, 0, st>>>(sz, m, L, P.Fs, b, tb, x, P.rr, L.nint, stop);
      note_launch();
    });
    dbg_sync(P, st, "k_facet_jacobi");
  }
  const int top = P.nlev - 1;
  prof_begin(PROF_GMG, st);
  {
    int64_t ge = (P.nP1 * 32 + bs - 1) / bs;  // a warp per P1 vertex
    if (ge > (int64_t)sm_count() * 32) ge = (int64_t)sm_count() * 32;
    if (ge < 1) ge = 1;
    const bool push = P.multiplicative && P.push_warps > 0 && P.q0 && P.q1;
    k_embed_T<R><<<(unsigned)ge, bs, 0, st>>>(s, L, P.Eb, P.vf_ptr, P.vf_idx, P.nP1, push ? P.q0 : P.rr,
                                             push ? P.q1 : nullptr, P.pb[top], stop);
  }
  note_launch();
  dbg_sync(P, st, "k_embed_T");
  vcycle<R>(P, top, stop, st);
  dbg_sync(P, st, "V-cycle");
  k_embed<R><<<g, bs, 0, st>>>(s, L, P.Eb, P.fvr, L.nint, P.px[top], x, stop);
  note_launch();
  dbg_sync(P, st, "k_embed");
  prof_end(PROF_GMG, 0.0, 0.0, st);
  if (P.multiplicative)
    for (int sw = 0; sw < P.smooth; ++sw)
      for (int c = P.ncol - 1; c >= 0; --c)
        facet_step<R>(s, m, L, P, b, tb, x, nullptr, co[c], co[c + 1] - co[c], true, stop, st);
}

template <class R>
cudaError_t autotune_launches(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, PrecData<R>& P,
                              KOp& K, double* v1, double* v2, cudaStream_t st, char* report, int report_len) {
  const Layout PL = precond_layout(L, s, sizeof(R));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_ms = [&](auto&& fn) {
    fn();   // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) fn();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / 3.0f;
  };
  int pos = 0;
  auto rep = [&](const char* fmt, int a, int b, float ms) {
    if (report && pos < report_len - 64) pos += snprintf(report + pos, report_len - pos, fmt, a, b, ms);
  };
  // facet step candidates: only where the batched block kernel runs (2D; facet stream under 4 KB)
  const bool block_kernel = !((size_t)fs_stride(s) * sizeof(R) >= 4096 && 2 * s.mF <= 32) &&
                            facet_step_smem<R>(s, 1, true) <= 200 * 1024 && PL.nint > 0;
  if (block_kernel) {
    const int64_t n0 = P.colour_off[1] - P.colour_off[0];
    float best = 1e30f;
    int bfb = -1, bth = -1;
    const int fbs[] = {2, 3, 4, 6, 9, 12, 16, 24};
    for (int th : {128, 256})
      for (int fb : fbs) {
        if (2 * s.mF * fb > 2 * th || facet_step_smem<R>(s, fb, true) > 160 * 1024) continue;
        P.fb = fb;
        P.fthreads = th;
        const float ms = time_ms([&] { facet_step<R>(s, m, PL, P, P.b, P.t, P.x, nullptr, 0, n0, true, nullptr, st); });
        rep("facet FB=%d threads=%d %.4f ms; ", fb, th, ms);
        if (ms < best) { best = ms; bfb = fb; bth = th; }
      }
    P.fb = bfb;
    P.fthreads = bth;
  }
  // staged K apply candidates
  {
    const int per = s.n_A + s.n_p;
    const size_t per_bytes = K.Ahi ? (2 * (size_t)packed_pad(s) + 2 * per) * sizeof(float) + 32
                                   : (size_t)s.n_A * s.n_A * sizeof(double) + (size_t)per * 8 + 32;
    if (per_bytes <= 160 * 1024) {
      float best = 1e30f;
      int beb = -1;
      for (int eb : {1, 2, 3, 4, 5, 6, 8, 12}) {
        if ((size_t)eb * per_bytes > 160 * 1024 || eb * per > 1024) continue;
        K.eb = eb;
        const float ms = time_ms([&] { launch_apply_K(s, t, m, L, K, v1, v2, nullptr, st); });
        rep("apply EB=%d (%d) %.4f ms; ", eb, 0, ms);
        if (ms < best) { best = ms; beb = eb; }
      }
      K.eb = beb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError();
}
template cudaError_t autotune_launches<float>(const ElemSizes&, const DevTables&, const DevMesh&, const Layout&,
                                              PrecData<float>&, KOp&, double*, double*, cudaStream_t, char*, int);
template cudaError_t autotune_launches<double>(const ElemSizes&, const DevTables&, const DevMesh&, const Layout&,
                                               PrecData<double>&, KOp&, double*, double*, cudaStream_t, char*, int);

// z = Khat^{-1} r (eq. mhatinvfactor, two applications of Ahat^{-1}, reading R3).
template <class R>
cudaError_t launch_precond(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, double nu,
                           PrecData<R>& P, const double* r, double* z, const int* stop, cudaStream_t st) {
  const int bs = 256;
  const unsigned g = (unsigned)(sm_count() * 8);
  const Layout& LE = L;                                 // external layout of r and z
  const Layout PL = precond_layout(LE, s, sizeof(R));   // facet-interleaved internal layout
  // b = r in precision R, preconditioner layout
  k_to_prec<R><<<g, bs, 0, st>>>(s, LE, PL, r, P.b);
  note_launch();
  dbg_sync(P, st, "k_to_prec");
  // first Ahat^{-1}: a = Ahat^{-1} r_u  (a in P.zz), then z_p = Shat_p^{-1}(r_p - B a) (P.x, p part)
  cudaMemsetAsync(P.t, 0, sizeof(R) * PL.n_dd, st);
  elem_prologue<R, false>(s, t, m, PL, P, P.b, nullptr, P.zz, P.t, stop, st);
  dbg_sync(P, st, "k_elem_prologue");
  asp_core<R>(s, m, PL, P, P.b, P.t, P.zz, stop, st);
  elem_epilogue<R, true>(s, t, m, PL, nu, P, P.zz, P.b, P.zz, P.x, stop, st);
  dbg_sync(P, st, "k_elem_epilogue");
  // second Ahat^{-1}: z_u = Ahat^{-1}(r_u - B^T z_p)  (P.x velocity part)
  cudaMemsetAsync(P.t, 0, sizeof(R) * PL.n_dd, st);
  elem_prologue<R, true>(s, t, m, PL, P, P.b, P.x, P.x, P.t, stop, st);
  asp_core<R>(s, m, PL, P, P.b, P.t, P.x, stop, st);
  elem_epilogue<R, false>(s, t, m, PL, nu, P, P.x, P.b, P.x, nullptr, stop, st);
  k_from_prec<R><<<g, bs, 0, st>>>(s, LE, PL, P.x, z, stop);
  note_launch();
  dbg_sync(P, st, "k_from_prec");
  return cudaGetLastError();
}

// ============================================================================ Krylov helpers
// DIFF = false: a.b; DIFF = true: |a - b|^2 (the same fixed reduction order)
template <bool DIFF>
__global__ void k_dot(const double* a, const double* b, int64_t n, double* part, double* out, const int* stop,
                      unsigned int* counter) {
  if (stop && *stop) return;
  __shared__ double red[32];
  __shared__ bool last;
  double v = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (DIFF) {
      const double e = a[i] - b[i];
      v += e * e;
    } else {
      v += a[i] * b[i];
    }
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      part[blockIdx.x] = v;
      __threadfence();
      unsigned t = atomicAdd(counter, 1u);
      last = (t == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (last) {
    __threadfence();
    // fixed-order final sum over the block partials
    double w = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) w += ((volatile double*)part)[i];
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x < 32) {
      w = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      if (threadIdx.x == 0) {
        *out = w;
        *counter = 0;
      }
    }
  }
}

cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* scratch, double* out, const int* stop,
                       cudaStream_t st) {
  int blocks = sm_count() * 4;
  if (blocks > 1024) blocks = 1024;
  k_dot<false><<<blocks, 256, 0, st>>>(a, b, n, scratch, out, stop, (unsigned int*)(scratch + 1024));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_diff_sq(const double* a, const double* b, int64_t n, double* scratch, double* out,
                           cudaStream_t st) {
  int blocks = sm_count() * 4;
  if (blocks > 1024) blocks = 1024;
  k_dot<true><<<blocks, 256, 0, st>>>(a, b, n, scratch, out, nullptr, (unsigned int*)(scratch + 1024));
  note_launch();
  return cudaGetLastError();
}

__global__ void k_mean_sum(DevMesh m, Layout L, int n_p, const double* x, double* part, double* out, double total,
                           const int* stop, unsigned int* counter) {
  if (stop && *stop) return;
  __shared__ double red[32];
  __shared__ bool last;
  double v = 0;
  for (int64_t T = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; T < m.ne; T += (int64_t)gridDim.x * blockDim.x)
    v += m.adet[T] * x[L.off_p + T * n_p];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      part[blockIdx.x] = v;
      __threadfence();
      unsigned t = atomicAdd(counter, 1u);
      last = (t == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double w = 0;
    for (int i = 0; i < (int)gridDim.x; ++i) w += ((volatile double*)part)[i];
    *out = w / total;
    *counter = 0;
  }
}
__global__ void k_mean_sub(DevMesh m, Layout L, int n_p, double* x, const double* mean, const int* stop) {
  if (stop && *stop) return;
  const double mu = *mean;
  for (int64_t T = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; T < m.ne; T += (int64_t)gridDim.x * blockDim.x)
    x[L.off_p + T * n_p] -= mu;
}

cudaError_t launch_mean_zero(const DevMesh& m, const Layout& L, int n_p, double* x, double* scratch,
                             double total_adet, const int* stop, cudaStream_t st) {
  // p_h mean weighted by |T|: mode-0 coefficients weighted by |det J| (the constant mode)
  int blocks = sm_count() * 2;
  k_mean_sum<<<blocks, 256, 0, st>>>(m, L, n_p, x, scratch + 1040, scratch + 2070, total_adet, stop,
                                     (unsigned int*)(scratch + 2080));
  note_launch();
  k_mean_sub<<<blocks, 256, 0, st>>>(m, L, n_p, x, scratch + 2070, stop);
  note_launch();
  return cudaGetLastError();
}

// ---- MinRes scalars ----
__global__ void k_minres_init(MinresScalars* S) {
  double g = S->dot1 > 0 ? sqrt(S->dot1) : 0.0;
  if (S->g_first < 0) S->g_first = g;
  const double target = S->rtol * S->g_first;
  S->gamma = g;
  S->gamma_old = 1.0;
  S->eta = g;
  S->res0 = g;
  S->c = 1.0;
  S->c_old = 1.0;
  S->s = 0.0;
  S->s_old = 0.0;
  S->it = 0;
  S->status = 0;
  S->dot2 = 0.0;
  S->rtol_cycle = (g > 0) ? fmax(target / g, S->floor_rtol) : 1.0;
  S->stop = (g == 0.0 || g <= target || !(g == g)) ? 1 : 0;
  if (!(g == g)) S->status = -5;
}
cudaError_t launch_minres_init(MinresScalars* S, cudaStream_t st) {
  k_minres_init<<<1, 1, 0, st>>>(S);
  note_launch();
  return cudaGetLastError();
}
__global__ void k_minres_scalars(MinresScalars* S) {
  if (S->stop) return;
  const double delta = S->delta, gamma = S->gamma;
  const double gnew = S->dot1 > 0 ? sqrt(S->dot1) : 0.0;
  const double a0 = S->c * delta - S->c_old * S->s * gamma;
  const double a1 = sqrt(a0 * a0 + gnew * gnew);
  const double a2 = S->s * delta + S->c_old * S->c * gamma;
  const double a3 = S->s_old * gamma;
  S->c_old = S->c;
  S->s_old = S->s;
  S->c = a0 / a1;
  S->s = gnew / a1;
  S->a1 = a1;
  S->a2 = a2;
  S->a3 = a3;
  S->coef_x = S->c * S->eta;
  S->eta = -S->s * S->eta;
  S->gamma_old = gamma;
  S->gamma = gnew;
  S->it += 1;
  S->delta = 0;
  int halt = 0;
  if (!(S->eta == S->eta) || !(a1 == a1) || S->dot1 < 0) {
    S->status = -5;  // breakdown
    halt = 1;
  } else if (fabs(S->eta) <= S->rtol_cycle * S->res0 || gnew == 0.0) {
    S->status = 0;
    halt = 1;
  } else if (S->it >= S->maxit) {
    S->status = -4;
    halt = 1;
  }
  if (halt) S->dot2 = 1.0;  // commit flag, applied after the update
}
cudaError_t launch_minres_scalars(MinresScalars* S, cudaStream_t st) {
  k_minres_scalars<<<1, 1, 0, st>>>(S);
  note_launch();
  return cudaGetLastError();
}
__global__ void k_minres_commit(MinresScalars* S) {
  if (S->dot2 != 0.0) S->stop = 1;
}
__global__ void k_scale(int64_t n, const double* zin, double* z, const MinresScalars* S) {
  if (S->stop) return;
  const double ig = 1.0 / S->gamma;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = zin[i] * ig;
}
__global__ void k_lanczos(int64_t n, const double* Kz, const double* v, double* v_old, const MinresScalars* S) {
  if (S->stop) return;
  const double al = S->delta / S->gamma, be = S->gamma / S->gamma_old;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v_old[i] = Kz[i] - al * v[i] - be * v_old[i];
}
__global__ void k_update(int64_t n, const double* z, const double* w, double* w_old, double* x,
                         const MinresScalars* S) {
  if (S->stop) return;
  const double ia1 = 1.0 / S->a1, a2 = S->a2, a3 = S->a3, cx = S->coef_x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double wn = (z[i] - a3 * w_old[i] - a2 * w[i]) * ia1;
    w_old[i] = wn;
    x[i] += cx * wn;
  }
}
cudaError_t launch_minres_lanczos(MinresScalars* S, int64_t n, double* z, const double* Kz, const double* v,
                                  double* v_old, cudaStream_t st) {
  (void)z;
  k_lanczos<<<sm_count() * 8, 256, 0, st>>>(n, Kz, v, v_old, S);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_minres_update(MinresScalars* S, int64_t n, const double* z, double* w, double* w_old,
                                 double* x, cudaStream_t st) {
  k_update<<<sm_count() * 8, 256, 0, st>>>(n, z, w, w_old, x, S);
  note_launch();
  k_minres_commit<<<1, 1, 0, st>>>(S);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_minres_scale(MinresScalars* S, int64_t n, const double* zin, double* z, cudaStream_t st) {
  k_scale<<<sm_count() * 8, 256, 0, st>>>(n, zin, z, S);
  note_launch();
  return cudaGetLastError();
}
__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  k_axpby<<<sm_count() * 8, 256, 0, st>>>(n, a, x, b, y);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- explicit instantiations
template cudaError_t launch_condense<float>(const ElemSizes&, const DevTables&, const DevMesh&, double, KOp,
                                            float*, float*, float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_condense<double>(const ElemSizes&, const DevTables&, const DevMesh&, double, KOp,
                                             double*, double*, double*, double*, int64_t, cudaStream_t);
template cudaError_t launch_facet_blocks<float>(const ElemSizes&, const DevMesh&, float*, cudaStream_t);
template cudaError_t launch_facet_blocks<double>(const ElemSizes&, const DevMesh&, double*, cudaStream_t);
template cudaError_t launch_precond<float>(const ElemSizes&, const DevTables&, const DevMesh&, const Layout&, double,
                                           PrecData<float>&, const double*, double*, const int*, cudaStream_t);
template cudaError_t launch_precond<double>(const ElemSizes&, const DevTables&, const DevMesh&, const Layout&, double,
                                            PrecData<double>&, const double*, double*, const int*, cudaStream_t);

// ---------------------------------------------------------------- launch accounting
static std::atomic<uint64_t> g_launches{0};
thread_local bool g_capturing = false;

void note_launch() {
  if (!g_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------- profiler
thread_local Profiler* g_prof = nullptr;

void prof_begin(int cls, cudaStream_t st) {
  if (g_prof) g_prof->begin(cls, st);
}
void prof_end(int cls, double bytes, double flops, cudaStream_t st) {
  if (g_prof) g_prof->end(cls, bytes, flops, st);
}

}  // namespace mcs
