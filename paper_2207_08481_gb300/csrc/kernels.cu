// Device kernels of libmcs (sm_103a).  See kernels.h for the roles.
#include <cuda_runtime.h>

#include <cstdio>

#include "kernels.h"

namespace mcs {

#define MCS_WARP 32

struct WarpSync {
  __device__ void operator()() const { __syncwarp(); }
};

// ============================================================================ condensation
// One warp per element (grid-stride).  Workspace in dynamic shared memory when it
// fits, else in a global scratch slot per resident warp.
template <class R, bool SMEM>
__global__ void __launch_bounds__(128) k_condense(ElemSizes s, DevTables t, DevMesh m, double nu, double* AT, R* Ad,
                                                  R* G, R* Aoi, double* gscratch, int64_t slot_doubles) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * wpb + wib, nw = (int64_t)gridDim.x * wpb;
  double* base = SMEM ? smem + (int64_t)wib * slot_doubles : gscratch + gw * slot_doubles;
  ElemWork w = elem_work_carve(s, base);
  double* bw = base + elem_work_doubles(s);         // bubble work
  double* Xs = bw + s.n_bub * s.n_bub + s.n_bub * s.n_c;  // (d+1)*d coords
  int* sg = (int*)(Xs + 16);
  double* Adt = Xs + 24;                            // n_c*n_c + n_bub*n_c + n_bub*n_bub staging (FP64)
  double* Gt = Adt + s.n_c * s.n_c;
  double* Ait = Gt + s.n_bub * s.n_c;
  ElemTables et{t.B0, t.Rf, t.Bh, t.Ccon, t.Adiv, t.nhat};
  const int d = s.d;
  for (int64_t T = gw; T < m.ne; T += nw) {
    if (lane < (d + 1) * d) {
      int v = lane / d, a = lane % d;
      Xs[lane] = m.coords[(int64_t)m.elems[T * (d + 1) + v] * d + a];
    }
    if (lane <= d) sg[lane] = m.signs[T * (d + 1) + lane];
    __syncwarp();
    condense_element(s, et, Xs, sg, nu, w, lane, MCS_WARP, WarpSync());
    // packed lower triangle of A_T (FP64)
    const int nA = s.n_A;
    const int64_t np = (int64_t)nA * (nA + 1) / 2;
    double* out = AT + T * np;
    for (int64_t q = lane; q < np; q += MCS_WARP) {
      int i = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
      while ((int64_t)i * (i + 1) / 2 > q) --i;
      while ((int64_t)(i + 1) * (i + 2) / 2 <= q) ++i;
      int j = (int)(q - (int64_t)i * (i + 1) / 2);
      out[q] = w.A[i * nA + j];
    }
    __syncwarp();
    bubble_condense(s, w.A, bw, Adt, Gt, Ait, lane, MCS_WARP, WarpSync());
    const int nc = s.n_c, no = s.n_bub;
    for (int q = lane; q < nc * nc; q += MCS_WARP) Ad[T * nc * nc + q] = (R)Adt[q];
    for (int q = lane; q < no * nc; q += MCS_WARP) G[T * no * nc + q] = (R)Gt[q];
    for (int q = lane; q < no * no; q += MCS_WARP) Aoi[T * no * no + q] = (R)Ait[q];
    __syncwarp();
  }
}

static int64_t condense_slot_doubles(const ElemSizes& s) {
  int64_t v = elem_work_doubles(s) + s.n_bub * s.n_bub + s.n_bub * s.n_c + 24 + s.n_c * s.n_c + s.n_bub * s.n_c +
              s.n_bub * s.n_bub;
  return (v + 31) / 32 * 32;
}

template <class R>
cudaError_t launch_condense(const ElemSizes& s, const DevTables& t, const DevMesh& m, double nu, double* AT, R* Ad,
                            R* G, R* Aoi, double* scratch, int64_t scratch_doubles, cudaStream_t st) {
  const int64_t slot = condense_slot_doubles(s);
  int dev = 0, nsm = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int64_t bytes_per_warp = slot * 8;
  if (bytes_per_warp * 1 <= maxsm) {
    int wpb = 4;
    while (wpb > 1 && bytes_per_warp * wpb > maxsm) wpb >>= 1;
    size_t sm = (size_t)(bytes_per_warp * wpb);
    cudaFuncSetAttribute(k_condense<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_condense<R, true>, wpb * 32, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)nsm * per_sm;
    int64_t need = (m.ne + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    k_condense<R, true><<<(unsigned)blocks, wpb * 32, sm, st>>>(s, t, m, nu, AT, Ad, G, Aoi, nullptr, slot);
  } else {
    int64_t slots = scratch_doubles / slot;
    if (slots < 1) return cudaErrorMemoryAllocation;
    int wpb = 4;
    int64_t blocks = slots / wpb;
    if (blocks < 1) {
      wpb = 1;
      blocks = slots;
    }
    int64_t need = (m.ne + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    k_condense<R, false><<<(unsigned)blocks, wpb * 32, 0, st>>>(s, t, m, nu, AT, Ad, G, Aoi, scratch, slot);
  }
  return cudaGetLastError();
}

int64_t condense_scratch_doubles(const ElemSizes& s, int nsm) {
  return condense_slot_doubles(s) * (int64_t)nsm * 8;
}

// ---------------------------------------------------------------- facet blocks
template <class R>
__global__ void k_facet_blocks(ElemSizes s, DevMesh m, const R* Ad, R* Dinv) {
  extern __shared__ double sm2[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int mF = s.mF, nc = s.n_c;
  double* A = sm2 + (int64_t)wib * 2 * mF * mF;
  double* I = A + mF * mF;
  for (int64_t r = (int64_t)blockIdx.x * wpb + wib; r < m.nint; r += (int64_t)gridDim.x * wpb) {
    for (int q = lane; q < mF * mF; q += 32) {
      int i = q / mF, j = q % mF;
      double v = 0;
      for (int side = 0; side < 2; ++side) {
        int64_t T = m.fel[r * 2 + side];
        int f = m.floc[r * 2 + side];
        v += (double)Ad[T * nc * nc + (int64_t)(f * mF + i) * nc + f * mF + j];
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
    for (int q = lane; q < mF * mF; q += 32) Dinv[r * mF * mF + q] = (R)(0.5 * (I[q] + I[(q % mF) * mF + q / mF]));
    __syncwarp();
  }
}

template <class R>
cudaError_t launch_facet_blocks(const ElemSizes& s, const DevMesh& m, const R* Ad, R* Dinv, cudaStream_t st) {
  if (m.nint == 0) return cudaSuccess;
  int wpb = 4;
  size_t sm = (size_t)wpb * 2 * s.mF * s.mF * sizeof(double);
  cudaFuncSetAttribute(k_facet_blocks<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int64_t blocks = (m.nint + wpb - 1) / wpb;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  k_facet_blocks<R><<<(unsigned)blocks, wpb * 32, sm, st>>>(s, m, Ad, Dinv);
  return cudaGetLastError();
}

// ============================================================================ K apply (FP64)
__device__ __forceinline__ int64_t local_to_global(const ElemSizes& s, const Layout& L, const int32_t* er, int64_t T,
                                                   int i) {
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

__global__ void __launch_bounds__(128) k_apply_K(ElemSizes s, DevTables t, DevMesh m, Layout L, const double* AT,
                                                 const double* x, double* y, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ double sk[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int nA = s.n_A, np_ = s.n_p, nu_ = s.n_u, d = s.d;
  const int64_t npk = (int64_t)nA * (nA + 1) / 2;
  double* A = sk + (int64_t)wib * (npk + 2 * nA + np_ + 8);
  double* xa = A + npk;
  double* ya = xa + nA;
  double* xp = ya + nA;
  int* er = (int*)(xp + np_);
  for (int64_t T = (int64_t)blockIdx.x * wpb + wib; T < m.ne; T += (int64_t)gridDim.x * wpb) {
    const double* src = AT + T * npk;
    for (int64_t q = lane; q < npk; q += 32) A[q] = src[q];
    if (lane <= d) er[lane] = m.elem_rank[T * (d + 1) + lane];
    __syncwarp();
    for (int i = lane; i < nA; i += 32) {
      int64_t g = local_to_global(s, L, er, T, i);
      xa[i] = g < 0 ? 0.0 : x[g];
    }
    for (int j = lane; j < np_; j += 32) xp[j] = x[L.off_p + T * np_ + j];
    __syncwarp();
    // B = -Bhat diag(sign) on the u columns
    for (int i = lane; i < nA; i += 32) {
      double v = 0;
      for (int j = 0; j < nA; ++j) {
        int64_t q = (i >= j) ? (int64_t)i * (i + 1) / 2 + j : (int64_t)j * (j + 1) / 2 + i;
        v += A[q] * xa[j];
      }
      if (i < nu_) {
        double sgn = (i < (d + 1) * s.nF) ? (double)m.signs[T * (d + 1) + i / s.nF] : 1.0;
        double bt = 0;
        for (int j = 0; j < np_; ++j) bt += t.Bp[j * nu_ + i] * xp[j];
        v -= sgn * bt;
      }
      ya[i] = v;
    }
    for (int j = lane; j < np_; j += 32) {
      double v = 0;
      for (int i = 0; i < nu_; ++i) {
        double sgn = (i < (d + 1) * s.nF) ? (double)m.signs[T * (d + 1) + i / s.nF] : 1.0;
        v += t.Bp[j * nu_ + i] * sgn * xa[i];
      }
      y[L.off_p + T * np_ + j] = -v;
    }
    __syncwarp();
    for (int i = lane; i < nA; i += 32) {
      int64_t g = local_to_global(s, L, er, T, i);
      if (g < 0) continue;
      if (i >= (d + 1) * s.nF && i < nu_) y[g] = ya[i];   // bubble: owned by T
      else atomicAdd(&y[g], ya[i]);                       // facet dof: exactly two contributions into 0
    }
    __syncwarp();
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
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  }
  return n;
}

cudaError_t launch_apply_K(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L,
                           const double* AT, const double* x, double* y, const int* stop, cudaStream_t st) {
  k_zero_facet<<<sm_count() * 4, 256, 0, st>>>(L, y, stop);
  static int maxsm = 0;
  if (!maxsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  int wpb = 4;
  const int64_t npk = (int64_t)s.n_A * (s.n_A + 1) / 2;
  const int64_t per_warp = (npk + 2 * s.n_A + s.n_p + 8) * (int64_t)sizeof(double);
  while (wpb > 1 && per_warp * wpb > maxsm) wpb >>= 1;
  if (per_warp > maxsm) return cudaErrorInvalidConfiguration;
  size_t sm = (size_t)(per_warp * wpb);
  cudaFuncSetAttribute(k_apply_K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_apply_K, wpb * 32, sm);
  if (per < 1) per = 1;
  int64_t blocks = (int64_t)sm_count() * per;
  int64_t need = (m.ne + wpb - 1) / wpb;
  if (blocks > need) blocks = need;
  k_apply_K<<<(unsigned)blocks, wpb * 32, sm, st>>>(s, t, m, L, AT, x, y, stop);
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

cudaError_t launch_load_points(const ElemSizes& s, const DevTables& t, const DevMesh& m, double* xq,
                               cudaStream_t st) {
  k_load_points<<<sm_count() * 8, 256, 0, st>>>(s, t, m, xq);
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
  return cudaGetLastError();
}

// ============================================================================ preconditioner (precision R)
// gather the coupling vector x_T (facet-major) of element T from an external-layout vector
template <class R>
__device__ __forceinline__ R coup_get(const ElemSizes& s, const Layout& L, const R* x, int32_t rk, int t) {
  if (rk < 0) return (R)0;
  return (t < s.nF) ? x[(int64_t)rk * s.nF + t] : x[L.off_h + (int64_t)rk * s.nhF + (t - s.nF)];
}
template <class R>
__device__ __forceinline__ int64_t coup_idx(const ElemSizes& s, const Layout& L, int32_t rk, int t) {
  return (t < s.nF) ? (int64_t)rk * s.nF + t : L.off_h + (int64_t)rk * s.nhF + (t - s.nF);
}

__global__ void k_to_R_f(int64_t n, const double* a, float* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_to_R_d(int64_t n, const double* a, double* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}
template <class R>
__global__ void k_from_R(int64_t n, const R* a, double* b, const int* stop) {
  if (stop && *stop) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// tb[c] = sum_T (G_T^T r_o)_c over the coupling dofs (two contributions each, into zero)
template <class R>
__global__ void k_bubble_elim(ElemSizes s, DevMesh m, Layout L, const R* G, const R* r, R* tb, const int* stop) {
  if (stop && *stop) return;
  const int d = s.d, nc = s.n_c, no = s.n_bub;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < m.ne * nc;
       id += (int64_t)gridDim.x * blockDim.x) {
    int64_t T = id / nc;
    int c = (int)(id % nc);
    int f = c / s.mF, tt = c % s.mF;
    int32_t rk = m.elem_rank[T * (d + 1) + f];
    if (rk < 0) continue;
    const R* g = G + T * no * nc;
    const R* ro = r + L.off_o + T * no;
    R v = 0;
    for (int o = 0; o < no; ++o) v += g[o * nc + c] * ro[o];
    atomicAdd(&tb[coup_idx<R>(s, L, rk, tt)], v);
  }
}

// x_o = Aoo^{-1} r_o - G x_c
template <class R>
__global__ void k_bubble_back(ElemSizes s, DevMesh m, Layout L, const R* G, const R* Aoi, const R* r, R* x,
                              const int* stop) {
  if (stop && *stop) return;
  const int d = s.d, nc = s.n_c, no = s.n_bub;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < m.ne * no;
       id += (int64_t)gridDim.x * blockDim.x) {
    int64_t T = id / no;
    int o = (int)(id % no);
    const R* ai = Aoi + T * no * no + o * no;
    const R* ro = r + L.off_o + T * no;
    R v = 0;
    for (int p = 0; p < no; ++p) v += ai[p] * ro[p];
    const R* g = G + T * no * nc + o * nc;
    for (int c = 0; c < nc; ++c) {
      int f = c / s.mF;
      int32_t rk = m.elem_rank[T * (d + 1) + f];
      v -= g[c] * coup_get<R>(s, L, x, rk, c % s.mF);
    }
    x[L.off_o + T * no + o] = v;
  }
}

// Facet-centric block step: for facets in `list`, r_F = b_F - tb_F - sum_T (Ad_T x_T)|_F;
// UPDATE: x_F += Dinv_F r_F; else rr_F = r_F.
template <class R, bool UPDATE>
__global__ void __launch_bounds__(128) k_facet_step(ElemSizes s, DevMesh m, Layout L, const R* Ad, const R* Dinv,
                                                    const R* b, const R* tb, R* x, R* rr, const int32_t* list,
                                                    int64_t nlist, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ unsigned char sraw[];
  R* sh = (R*)sraw;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int d = s.d, nc = s.n_c, mF = s.mF;
  R* xT = sh + (int64_t)wib * (nc + 2 * mF);
  R* rF = xT + nc;
  R* yF = rF + mF;
  for (int64_t li = (int64_t)blockIdx.x * wpb + wib; li < nlist; li += (int64_t)gridDim.x * wpb) {
    const int64_t r = list ? list[li] : li;
    for (int t = lane; t < mF; t += 32) {
      int64_t g = coup_idx<R>(s, L, (int32_t)r, t);
      rF[t] = b[g] - (tb ? tb[g] : (R)0);
    }
    for (int side = 0; side < 2; ++side) {
      const int64_t T = m.fel[r * 2 + side];
      const int f = m.floc[r * 2 + side];
      __syncwarp();
      for (int c = lane; c < nc; c += 32) {
        int ff = c / mF;
        xT[c] = coup_get<R>(s, L, x, m.elem_rank[T * (d + 1) + ff], c % mF);
      }
      __syncwarp();
      const R* A = Ad + T * nc * nc + (int64_t)f * mF * nc;
      // each row t: lanes split the dot product
      for (int t = 0; t < mF; ++t) {
        R v = 0;
        for (int c = lane; c < nc; c += 32) v += A[(int64_t)t * nc + c] * xT[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) rF[t] -= v;
      }
    }
    __syncwarp();
    if (UPDATE) {
      const R* Di = Dinv + r * mF * mF;
      for (int t = lane; t < mF; t += 32) {
        R v = 0;
        for (int j = 0; j < mF; ++j) v += Di[t * mF + j] * rF[j];
        yF[t] = v;
      }
      __syncwarp();
      for (int t = lane; t < mF; t += 32) x[coup_idx<R>(s, L, (int32_t)r, t)] += yF[t];
    } else {
      for (int t = lane; t < mF; t += 32) rr[coup_idx<R>(s, L, (int32_t)r, t)] = rF[t];
    }
    __syncwarp();
  }
}

// xbar = E^d^T rr  (gather per P1 dof over incident facets)
template <class R>
__global__ void k_embed_T(ElemSizes s, Layout L, const R* Eb, const int32_t* vf_ptr, const int32_t* vf_idx,
                          int64_t nP1, const R* rr, R* xb, const int* stop) {
  if (stop && *stop) return;
  const int d = s.d, mF = s.mF, dd = d * d;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nP1 * d;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = q / d;
    int a = (int)(q % d);
    R acc = 0;
    for (int32_t e = vf_ptr[v]; e < vf_ptr[v + 1]; ++e) {
      int32_t rk = vf_idx[2 * e], w = vf_idx[2 * e + 1];
      const R* B = Eb + (int64_t)rk * mF * dd;
      for (int t = 0; t < mF; ++t) acc += B[t * dd + w * d + a] * rr[coup_idx<R>(s, L, rk, t)];
    }
    xb[q] = acc;
  }
}

// x_F += E^d_F xbar  (facet vertices' P1 ranks in fvr [nint][d])
template <class R>
__global__ void k_embed(ElemSizes s, Layout L, const R* Eb, const int32_t* fvr, int64_t nint, const R* xb, R* x,
                        const int* stop) {
  if (stop && *stop) return;
  const int d = s.d, mF = s.mF, dd = d * d;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nint * mF;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t rk = q / mF;
    int t = (int)(q % mF);
    const R* B = Eb + rk * mF * dd + t * dd;
    R v = 0;
    for (int w = 0; w < d; ++w) {
      int32_t vr = fvr[rk * d + w];
      if (vr < 0) continue;
      for (int a = 0; a < d; ++a) v += B[w * d + a] * xb[(int64_t)vr * d + a];
    }
    x[coup_idx<R>(s, L, (int32_t)rk, t)] += v;
  }
}

// ---- GMG kernels ----
template <class R>
__global__ void k_jacobi(int64_t n, const int32_t* rp, const int32_t* ci, const R* va, const R* dinv, const R* b,
                         const R* x, R* xn, int first, const int* stop) {
  if (stop && *stop) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (first) {
      xn[i] = dinv[i] * b[i];
      continue;
    }
    R ax = 0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) ax += va[e] * x[ci[e]];
    xn[i] = x[i] + dinv[i] * (b[i] - ax);
  }
}
template <class R>
__global__ void k_residual_csr(int64_t n, const int32_t* rp, const int32_t* ci, const R* va, const R* b, const R* x,
                               R* r, const int* stop) {
  if (stop && *stop) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    R ax = 0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) ax += va[e] * x[ci[e]];
    r[i] = b[i] - ax;
  }
}
template <class R>
__global__ void k_spmv_csr(int64_t n, const int32_t* rp, const int32_t* ci, const R* va, const R* x, R* y, int add,
                           const int* stop) {
  if (stop && *stop) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    R v = 0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) v += va[e] * x[ci[e]];
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
    return;
  }
  const R* va = (const R*)G.val;
  const R* di = (const R*)G.dl1inv;
  R* x = P.px[l];
  R* xt = P.ptmp[l];
  for (int sw = 0; sw < P.gmg_smooth; ++sw) {
    k_jacobi<R><<<grid(G.n), bs, 0, st>>>(G.n, G.rowptr, G.col, va, di, P.pb[l], x, xt, sw == 0, stop);
    R* tmp = x; x = xt; xt = tmp;
  }
  k_residual_csr<R><<<grid(G.n), bs, 0, st>>>(G.n, G.rowptr, G.col, va, P.pb[l], x, P.pr[l], stop);
  const GmgLevel& Gc = P.lev[l - 1];
  k_spmv_csr<R><<<grid(Gc.n), bs, 0, st>>>(Gc.n, G.rrow, G.rcol, (const R*)G.rval, P.pr[l], P.pb[l - 1], 0, stop);
  vcycle(P, l - 1, stop, st);
  k_spmv_csr<R><<<grid(G.n), bs, 0, st>>>(G.n, G.prow, G.pcol, (const R*)G.pval, P.px[l - 1], x, 1, stop);
  for (int sw = 0; sw < P.gmg_smooth; ++sw) {
    k_jacobi<R><<<grid(G.n), bs, 0, st>>>(G.n, G.rowptr, G.col, va, di, P.pb[l], x, xt, 0, stop);
    R* tmp = x; x = xt; xt = tmp;
  }
  if (x != P.px[l]) cudaMemcpyAsync(P.px[l], x, sizeof(R) * G.n, cudaMemcpyDeviceToDevice, st);
}

template <class R>
static cudaError_t facet_step(const ElemSizes& s, const DevMesh& m, const Layout& L, PrecData<R>& P, const R* b,
                              const R* tb, R* x, R* rr, const int32_t* list, int64_t n, bool update,
                              const int* stop, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int wpb = 4;
  size_t sm = (size_t)wpb * (s.n_c + 2 * s.mF) * sizeof(R);
  int64_t blocks = (n + wpb - 1) / wpb;
  if (blocks > (int64_t)sm_count() * 16) blocks = (int64_t)sm_count() * 16;
  if (update)
    k_facet_step<R, true><<<(unsigned)blocks, wpb * 32, sm, st>>>(s, m, L, P.Ad, P.Dinv, b, tb, x, rr, list, n, stop);
  else
    k_facet_step<R, false><<<(unsigned)blocks, wpb * 32, sm, st>>>(s, m, L, P.Ad, P.Dinv, b, tb, x, rr, list, n, stop);
  return cudaGetLastError();
}

// Ahat^{-1}: rin (external layout, velocity part) -> out (velocity part), precision R
template <class R>
cudaError_t launch_ahat_inv(const ElemSizes& s, const DevMesh& m, const Layout& L, PrecData<R>& P, const R* rin,
                            R* out, const int* stop, cudaStream_t st) {
  const int bs = 256;
  const unsigned g = (unsigned)(sm_count() * 8);
  // tb = G^T r_o (coupling), x = 0
  cudaMemsetAsync(P.t, 0, sizeof(R) * L.ndof, st);
  cudaMemsetAsync(out, 0, sizeof(R) * L.off_p, st);
  k_bubble_elim<R><<<g, bs, 0, st>>>(s, m, L, P.G, rin, P.t, stop);
  const int64_t* co = P.colour_off;
  const bool mult = P.multiplicative != 0;
  if (mult) {
    for (int sw = 0; sw < P.smooth; ++sw)
      for (int c = 0; c < P.ncol; ++c)
        facet_step<R>(s, m, L, P, rin, P.t, out, nullptr, P.colour_list + co[c], co[c + 1] - co[c], true, stop, st);
  }
  // residual over all facets
  facet_step<R>(s, m, L, P, rin, P.t, out, P.rr, nullptr, L.nint, false, stop, st);
  // coarse correction: E^d C^{-1} E^d^T rr
  const int top = P.nlev - 1;
  k_embed_T<R><<<g, bs, 0, st>>>(s, L, P.Eb, P.vf_ptr, P.vf_idx, P.nP1, P.rr, P.pb[top], stop);
  vcycle<R>(P, top, stop, st);
  k_embed<R><<<g, bs, 0, st>>>(s, L, P.Eb, P.fvr, L.nint, P.px[top], out, stop);
  if (mult) {
    for (int sw = 0; sw < P.smooth; ++sw)
      for (int c = P.ncol - 1; c >= 0; --c)
        facet_step<R>(s, m, L, P, rin, P.t, out, nullptr, P.colour_list + co[c], co[c + 1] - co[c], true, stop, st);
  }
  k_bubble_back<R><<<g, bs, 0, st>>>(s, m, L, P.G, P.Aoi, rin, out, stop);
  return cudaGetLastError();
}

// B a  and  M_p^{-1}:  zp = (nu / |det J|) (r_p - B a),   B = -Bhat diag(sign)
template <class R>
__global__ void k_schur_p(ElemSizes s, DevTables t, DevMesh m, Layout L, double nu, const R* rR, const R* a, R* z,
                          const int* stop) {
  if (stop && *stop) return;
  const int d = s.d, nu_ = s.n_u, np_ = s.n_p;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < m.ne * np_;
       id += (int64_t)gridDim.x * blockDim.x) {
    int64_t T = id / np_;
    int j = (int)(id % np_);
    const int32_t* er = m.elem_rank + T * (d + 1);
    double v = 0;
    for (int i = 0; i < nu_; ++i) {
      int64_t g = local_to_global(s, L, er, T, i);
      if (g < 0) continue;
      double sg = (i < (d + 1) * s.nF) ? (double)m.signs[T * (d + 1) + i / s.nF] : 1.0;
      v += t.Bp[j * nu_ + i] * sg * (double)a[g];
    }
    const int64_t gp = L.off_p + T * np_ + j;
    z[gp] = (R)(nu / m.adet[T] * ((double)rR[gp] + v));
  }
}
// tt = r - B^T z_p on the velocity part (facet dofs: two contributions, computed into zero first)
template <class R>
__global__ void k_bt(ElemSizes s, DevTables t, DevMesh m, Layout L, const R* z, R* acc, const int* stop) {
  if (stop && *stop) return;
  const int d = s.d, nu_ = s.n_u, np_ = s.n_p;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < m.ne * nu_;
       id += (int64_t)gridDim.x * blockDim.x) {
    int64_t T = id / nu_;
    int i = (int)(id % nu_);
    const int32_t* er = m.elem_rank + T * (d + 1);
    int64_t g = local_to_global(s, L, er, T, i);
    if (g < 0) continue;
    double sg = (i < (d + 1) * s.nF) ? (double)m.signs[T * (d + 1) + i / s.nF] : 1.0;
    double v = 0;
    for (int j = 0; j < np_; ++j) v += t.Bp[j * nu_ + i] * (double)z[L.off_p + T * np_ + j];
    // (B^T z)_i = -sign_i * sum_j Bhat[j][i] z_j
    R bt = (R)(-sg * v);
    if (i >= (d + 1) * s.nF) acc[g] = bt;
    else atomicAdd(&acc[g], bt);
  }
}
template <class R>
__global__ void k_sub(int64_t n, const R* a, const R* b, R* c, const int* stop) {
  if (stop && *stop) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c[i] = a[i] - b[i];
}

template <class R>
cudaError_t launch_precond(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, double nu,
                           PrecData<R>& P, const double* r, double* z, const int* stop, cudaStream_t st) {
  const int bs = 256;
  const unsigned g = (unsigned)(sm_count() * 8);
  // rR = r in precision R  (P.b)
  if (sizeof(R) == 4) k_to_R_f<<<g, bs, 0, st>>>(L.ndof, r, (float*)P.b);
  else k_to_R_d<<<g, bs, 0, st>>>(L.ndof, r, (double*)P.b);
  // a = Ahat^{-1} r_u  -> P.zz
  launch_ahat_inv<R>(s, m, L, P, P.b, P.zz, stop, st);
  // zp = Sp^{-1}(r_p - B a) -> stored in P.x (p part)
  k_schur_p<R><<<g, bs, 0, st>>>(s, t, m, L, nu, P.b, P.zz, P.x, stop);
  // acc = B^T zp (velocity part) into P.rr (zeroed), then tt = r_u - acc -> P.zz
  cudaMemsetAsync(P.rr, 0, sizeof(R) * L.off_p, st);
  k_bt<R><<<g, bs, 0, st>>>(s, t, m, L, P.x, P.rr, stop);
  k_sub<R><<<g, bs, 0, st>>>(L.off_p, P.b, P.rr, P.zz, stop);
  // z_u = Ahat^{-1} tt -> P.x (velocity part; p part already there)
  launch_ahat_inv<R>(s, m, L, P, P.zz, P.x, stop, st);
  k_from_R<R><<<g, bs, 0, st>>>(L.ndof, P.x, z, stop);
  return cudaGetLastError();
}

// ============================================================================ Krylov helpers
__global__ void k_dot(const double* a, const double* b, int64_t n, double* part, double* out, const int* stop,
                      unsigned int* counter) {
  if (stop && *stop) return;
  __shared__ double red[32];
  __shared__ bool last;
  double v = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v += a[i] * b[i];
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
  k_dot<<<blocks, 256, 0, st>>>(a, b, n, scratch, out, stop, (unsigned int*)(scratch + 1024));
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
  k_mean_sub<<<blocks, 256, 0, st>>>(m, L, n_p, x, scratch + 2070, stop);
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
  return cudaGetLastError();
}
cudaError_t launch_minres_update(MinresScalars* S, int64_t n, const double* z, double* w, double* w_old,
                                 double* x, cudaStream_t st) {
  k_update<<<sm_count() * 8, 256, 0, st>>>(n, z, w, w_old, x, S);
  k_minres_commit<<<1, 1, 0, st>>>(S);
  return cudaGetLastError();
}
cudaError_t launch_minres_scale(MinresScalars* S, int64_t n, const double* zin, double* z, cudaStream_t st) {
  k_scale<<<sm_count() * 8, 256, 0, st>>>(n, zin, z, S);
  return cudaGetLastError();
}
__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  k_axpby<<<sm_count() * 8, 256, 0, st>>>(n, a, x, b, y);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- explicit instantiations
template cudaError_t launch_condense<float>(const ElemSizes&, const DevTables&, const DevMesh&, double, double*,
                                            float*, float*, float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_condense<double>(const ElemSizes&, const DevTables&, const DevMesh&, double, double*,
                                             double*, double*, double*, double*, int64_t, cudaStream_t);
template cudaError_t launch_facet_blocks<float>(const ElemSizes&, const DevMesh&, const float*, float*, cudaStream_t);
template cudaError_t launch_facet_blocks<double>(const ElemSizes&, const DevMesh&, const double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_precond<float>(const ElemSizes&, const DevTables&, const DevMesh&, const Layout&, double,
                                           PrecData<float>&, const double*, double*, const int*, cudaStream_t);
template cudaError_t launch_precond<double>(const ElemSizes&, const DevTables&, const DevMesh&, const Layout&, double,
                                            PrecData<double>&, const double*, double*, const int*, cudaStream_t);
template cudaError_t launch_ahat_inv<float>(const ElemSizes&, const DevMesh&, const Layout&, PrecData<float>&,
                                            const float*, float*, const int*, cudaStream_t);
template cudaError_t launch_ahat_inv<double>(const ElemSizes&, const DevMesh&, const Layout&, PrecData<double>&,
                                             const double*, double*, const int*, cudaStream_t);

}  // namespace mcs
