// Device kernels of libmcs and their host launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "element.cuh"

namespace mcs {

// Optional per-class kernel timing with CUDA events on the launching stream.  The API entry
// points install the handle's profiler for the duration of a call; launchers bracket their
// main kernel with prof_begin / prof_end (no-ops when no profiler is installed).
enum ProfClass { PROF_CONDENSE = 0, PROF_FACET_BLOCKS, PROF_APPLY, PROF_FACET_GS, PROF_FACET_RES, PROF_PROLOGUE,
                 PROF_EPILOGUE, PROF_GMG, PROF_FACET_PUSH, PROF_NCLASS };
struct Profiler;
extern thread_local Profiler* g_prof;
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, double bytes, double flops, cudaStream_t st);

// Launch accounting.  Every kernel launch of the library adds one to a process-wide counter;
// while a thread captures a CUDA graph its launches only record nodes and add nothing, and each
// launch of a captured graph adds the number of kernel nodes it runs.
extern thread_local bool g_capturing;
void note_launch();
void note_launches(uint64_t n);
uint64_t launch_count();

// Dof layout of the condensed system [u_d | u_o | uhat | p] (dof contract).
struct Layout {
  int64_t ne, nint;
  int64_t n_dd, n_oo, n_hat, n_pres, ndof;
  int64_t off_o, off_h, off_p;
  // 0: the external layout [u_d | u_o | uhat | p].  > 0: the preconditioner's internal layout, in
  // which the m_F coupling dofs of interior facet r (its u_d modes, then its uhat modes) sit
  // together at r*fstride .. r*fstride + m_F - 1 (fstride = m_F rounded up to 16 bytes), followed
  // by the bubbles and the pressure; one facet's values are one 16-byte-aligned segment.
  int64_t fstride = 0;
};

// Static mesh / table data resident on the device.
struct DevMesh {
  int d;
  int64_t ne, nint;
  const double* coords;      // [nv][d]
  const int32_t* elems;      // [ne][d+1]
  const int32_t* elem_rank;  // [ne][d+1]
  const int8_t* signs;       // [ne][d+1]
  const double* adet;        // [ne] |det J|
  const int32_t* fel;        // [nint][2] the two elements of each interior facet
  const int32_t* floc;       // [nint][2] local facet index in each element
  const int32_t* fsr;        // [nint][2][d+1] interior ranks of the facets of each side element
  // facet records in colour order (64 bytes each): [0] interior rank r, [1..2] the two elements,
  // [3..4] local facet indices, [5..] interior ranks of the facets of element 0 (d+1), then of
  // element 1 (d+1); [13] bit side*(d+1) + f set when element [1 + side] is side 1 of the facet
  // [5 + side*(d+1) + f]; unused entries -1
  const int4* frec;
  const int32_t* fpos;       // [nint] position of interior facet r in colour order (its record index)
  const int8_t* fout;        // [nint] 1 for an outflow facet (phantom uhat slots); NULL without outflow
};


// Compile-time element sizes for the (d, k) combinations with specialised kernels; the
// members mirror ElemSizes so kernels can take either (runtime sizes as the fallback).
__host__ __device__ constexpr int ct_npoly(int n, int k) {
  return k < 0 ? 0 : (n == 1 ? k + 1 : (n == 2 ? (k + 1) * (k + 2) / 2 : (k + 1) * (k + 2) * (k + 3) / 6));
}
template <int D, int K>
struct Ct {
  static constexpr int d = D, k = K;
  static constexpr int nk = ct_npoly(D, K), nF = ct_npoly(D - 1, K), nFm1 = ct_npoly(D - 1, K - 1);
  static constexpr int n_u = D * nk, n_bub = n_u - (D + 1) * nF, nhF = (D - 1) * nFm1, n_hat = (D + 1) * nhF;
  static constexpr int n_A = n_u + n_hat, n_p = ct_npoly(D, K - 1), mF = nF + nhF, n_c = (D + 1) * mF;
};

// Calls f(sizes) with compile-time sizes when a specialisation exists, else with s.
template <class F>
inline void dispatch_sizes(const ElemSizes& s, F&& f) {
  if (s.d == 2 && s.k == 2) f(Ct<2, 2>{});
  else if (s.d == 2 && s.k == 3) f(Ct<2, 3>{});
  else if (s.d == 2 && s.k == 4) f(Ct<2, 4>{});
  else if (s.d == 3 && s.k == 2) f(Ct<3, 2>{});
  else if (s.d == 3 && s.k == 3) f(Ct<3, 3>{});
  else f(s);
}

// Per-element device arrays are padded to multiples of 4 entries so that every slab and
// element block starts on a 16-byte boundary (vector loads into shared memory).
__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }
template <class S> __host__ __device__ inline int slab_pad(const S& s) { return pad4(s.n_c * s.mF); }
template <class S> __host__ __device__ inline int g_stride(const S& s) { return pad4(s.n_bub * s.n_c); }
template <class S> __host__ __device__ inline int a_stride(const S& s) { return pad4(s.n_bub * s.n_bub); }
template <class S> __host__ __device__ inline int dinv_stride(const S& s) { return pad4(s.mF * s.mF); }
// facet stride of the preconditioner layout: m_F rounded up to a multiple of 16 bytes (one 16-byte copy
// granule; 3D k = 2 in FP32: 12 values, 48 bytes)
template <class S> __host__ __device__ inline int facet_stride(const S& s, int elem_bytes) {
  const int v = 16 / elem_bytes;
  return (s.mF + v - 1) / v * v;
}
template <class S>
inline Layout precond_layout(const Layout& L, const S& s, int elem_bytes) {
  Layout P = L;
  P.fstride = facet_stride(s, elem_bytes);
  P.n_dd = L.nint * P.fstride;
  P.n_hat = 0;
  P.off_o = P.n_dd;
  P.off_h = P.off_o + L.n_oo;
  P.off_p = P.off_h;
  P.ndof = P.off_p + L.n_pres;
  return P;
}

// Facet stream: everything the facet-block smoother reads per interior facet, stored in colour
// order (record index i = fpos[r]) as one contiguous, 16-byte-aligned block of fs_stride entries:
//   [slab of side 0 | slab of side 1 | D_F^{-1}]
// where the slab of side s holds the m_F rows of A^d_T of that side's element T (the element
// fel[2r + s]) belonging to the facet, column-major over T's n_c coupling dofs:
//   slab[c*mF + t] = A^d_T[f*mF + t][c]   (f = the facet's local index in T),
// and D_F^{-1} is row-major [m_F][m_F] (stride dinv_stride).  A colour sweep therefore reads one
// contiguous range of the stream.
template <class S> __host__ __device__ inline int fs_stride(const S& s) { return 2 * slab_pad(s) + dinv_stride(s); }

struct DevTables {
  const double* B0;
  const double* Rf;
  const double* Bh;
  const double* Ccon;
  const double* Adiv;
  const double* nhat;
  const double* Wmom;      // k = 1: [d+1][d][nk]
  const double* Bp;        // [n_p][n_u]
  const float* Bp_hi;      // Bp split into float pairs (Bp = hi + lo to ~2^-48)
  const float* Bp_lo;
  const double* Mu;        // [d][d][n_u][n_u]
  const double* phi_load;  // [nq][n_u][d]
  const double* xq_load;   // [nq][d]
  const double* wq_load;   // [nq]
  int nq_load;
};

// ---------------------------------------------------------------- condensation
// Forms A_T (packed lower FP64), A^d_T, G_T, A_oo^{-1} (precision R) for every element.
// The operator K: A_T either in FP64 (full symmetric, AT) or as packed-lower float pairs
// (Ahi + Alo = A_T to ~2^-48; double-float arithmetic in the apply).
struct KOp {
  double* AT;
  float* Ahi;
  float* Alo;
  int eb = -1;   // elements per block of the staged K apply (-1: the shared-memory formula; autotuner)
};
template <class S> __host__ __device__ inline int packed_pad(const S& s) { return pad4(s.n_A * (s.n_A + 1) / 2); }

template <class R>
cudaError_t launch_condense(const ElemSizes& s, const DevTables& t, const DevMesh& m, double nu, KOp K,
                            R* Fs, R* G, R* Aoi, double* scratch, int64_t scratch_doubles, cudaStream_t st);
// One problem of a batched condensation: its sizes, tables, mesh and outputs; its elements take the
// global indices first .. first + m.ne - 1 of the launch.
template <class R>
struct CondenseItem {
  ElemSizes s;
  DevTables t;
  DevMesh m;
  double nu;
  KOp K;
  R* Fs;
  R* G;
  R* Aoi;
  int64_t first;
};
// Condensation of several problems (items in device memory, a host copy for the sizes) in one
// persistent launch; scratch: global workspace of scratch_doubles.
template <class R>
cudaError_t launch_condense_batch(const CondenseItem<R>* items_dev, const CondenseItem<R>* items_host, int nitems,
                                  double* scratch, int64_t scratch_doubles, cudaStream_t st);
int64_t condense_slot_bytes(const ElemSizes& s);

// Facet blocks D_F of A^d (sum of the two elements' slabs), inverted into the facet stream.
template <class R>
cudaError_t launch_facet_blocks(const ElemSizes& s, const DevMesh& m, R* Fs, cudaStream_t st);

// ---------------------------------------------------------------- operators (FP64)
// y = K x
cudaError_t launch_apply_K(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L,
                           KOp K, const double* x, double* y, const int* stop, cudaStream_t st);
// r = F - K x with the element products and the sum of a facet dof's two contributions carried in
// double-double and rounded once (the residual of a refinement cycle).  Y: workspace of 4 ndof doubles.
cudaError_t launch_residual_dd(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, KOp K,
                               const double* F, const double* x, double* Y, double* r, cudaStream_t st);
// F = M_u c (velocity mass) on the u part; zero elsewhere
cudaError_t launch_mass_u(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L,
                          const double* c, double* F, cudaStream_t st);
// F_i = (f, phi_i) with f given at the load quadrature points [ne][nq][d]
cudaError_t launch_load(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L,
                        const double* fq, double* F, cudaStream_t st);
// physical load quadrature points [ne][nq][d]
// sigma_h, omega_h of every element at nq reference points (psi: Dubiner values [nq][nk], device)
// into sig / om [ne][nq][d][d] (om may be NULL); scratch: global workspace when one element's does not
// fit in shared memory.
int64_t recover_slot_doubles(const ElemSizes& s);
cudaError_t launch_recover(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, double nu,
                           const double* x, int nq, const double* psi, double* sig, double* om, double* scratch,
                           int64_t scratch_doubles, cudaStream_t st);
cudaError_t launch_load_points(const ElemSizes& s, const DevTables& t, const DevMesh& m, double* xq,
                               cudaStream_t st);

// ---------------------------------------------------------------- preconditioner pieces (precision R)
// Sparse matrices of the multigrid in ELL form, column-major: entry k of row i at k*n + i, so the
// threads of consecutive rows read consecutive addresses; padding entries have value 0 and column 0.
struct Ell {
  int64_t n = 0;
  int k = 0;
  const int32_t* col = nullptr;  // [k][n]
  const void* val = nullptr;     // R [k][n]
};
struct GmgLevel {
  int64_t n;                 // dofs
  Ell A;                     // Abar on this level
  const void* dl1inv;        // R, 1 / sum_j |A_ij|
  Ell P;                     // prolongation to this level from the coarser one (fine rows)
  Ell Rt;                    // restriction (coarse rows)
};

template <class R>
struct PrecData {
  R* Fs;                    // facet stream [nint][fs_stride] in colour order (slabs of A^d, D_F^{-1})
  const R* G;
  const R* Aoi;
  const R* Eb;              // [nint][d][mF][d]: E^d_F entry (mode t, facet vertex w, component a) at (w*mF + t)*d + a
  const int32_t* fvr;       // [nint][d] P1 rank of each facet vertex (-1 on the boundary)
  const int32_t* vf_ptr;    // P1 vertex -> (facet rank, facet-vertex index) list, CSR over P1 vertices
  const int32_t* vf_idx;    // pairs (facet rank, col)
  int64_t nP1;
  const int32_t* colour_list;  // interior ranks sorted by colour
  const int64_t* colour_off;   // host array [ncol+1]
  int ncol;
  int smooth;        // facet-block Gauss-Seidel sweeps before / after the coarse correction
  int gmg_smooth;    // l1-Jacobi sweeps per level before / after the coarse-grid correction
  int multiplicative;
  int nlev;
  GmgLevel lev[12];
  const double* coarse_inv;    // [n0][n0] FP64
  // work vectors (R), all length ndof unless noted
  R *b, *x, *t, *rr, *zz;
  // forward sweeps with a maintained residual (push_warps > 0: warps per block of k_facet_push_warp;
  // 0: row products and a residual pass): the partial residuals of each facet's two elements, [n_dd] each
  int push_warps = 0;
  R *q0 = nullptr, *q1 = nullptr;
  int* err;  // device flag: set when a bounded wait on an asynchronous copy gave up
  int fb = -1, fthreads = -1;   // batched facet step: facets per batch and threads (-1: formulas; autotuner)
  // diagnostics (environment MCS_DEBUG_CHECKS=1 at set-up): the facet step checks every address
  // against its buffer and records the first bad one in dbg[0..3] instead of accessing it, and
  // the host synchronises after every preconditioner launch and names a kernel that failed
  int* dbg = nullptr;
  bool debug = false;
  R *pb[12], *px[12], *pr[12], *ptmp[12];  // GMG vectors per level
  double* coarse_tmp;  // [n0]
};

// Autotuner: times the candidate launch shapes of the batched facet step (the 2D blocks; 3D uses the
// warp-per-facet kernel, which has none) over the first colour and of the staged K apply on the handle's
// own data, and stores the fastest in P.fb / P.fthreads and K.eb.  Uses the preconditioner work vectors
// and two Krylov vectors as scratch (contents do not matter).  times: the measured ms per candidate
// (host, for the record).  Synchronous on st.
template <class R>
cudaError_t autotune_launches(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, PrecData<R>& P,
                              KOp& K, double* v1, double* v2, cudaStream_t st, char* report, int report_len);

// Warps per block of the maintained-residual forward sweep for these sizes in precision R (0: the
// sweep keeps the row-product form with a residual pass; facet blocks under 4 KB or 2 m_F > 32).
template <class R>
int facet_push_warps(const ElemSizes& s);

template <class R>
cudaError_t launch_precond(const ElemSizes& s, const DevTables& t, const DevMesh& m, const Layout& L, double nu,
                           PrecData<R>& P, const double* r, double* z, const int* stop, cudaStream_t st);

// ---------------------------------------------------------------- Krylov helpers (FP64)
// out[0] = a.b, deterministic: fixed grid, block partials summed in index order by the last block.
// scratch: >= 2100 doubles (partials, counters) per stream.
cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* scratch, double* out, const int* stop,
                       cudaStream_t st);
// out[0] = |a - b|^2, same fixed reduction order as launch_dot (scratch as there)
cudaError_t launch_diff_sq(const double* a, const double* b, int64_t n, double* scratch, double* out,
                           cudaStream_t st);
// remove the mean of p_h: p_{T,0} -= (sum adet_T p_{T,0}) / (sum adet_T)
cudaError_t launch_mean_zero(const DevMesh& m, const Layout& L, int n_p, double* x, double* scratch,
                             double total_adet, const int* stop, cudaStream_t st);

// MinRes state on the device
// Inputs (set by the host before each cycle): rtol (relative to g_first), floor_rtol (least
// relative reduction asked of one cycle), g_first (< 0: this is the first cycle), maxit.
struct MinresScalars {
  double gamma, gamma_old, eta, c, c_old, s, s_old, delta, res0, rtol, floor_rtol, g_first, rtol_cycle;
  double a1, a2, a3, coef_x;   // w_new = (z - a3 w_old - a2 w)/a1, x += coef_x w_new
  double dot1, dot2;           // dot results
  int it, maxit, stop, status;
};
cudaError_t launch_minres_init(MinresScalars* S, cudaStream_t st);
cudaError_t launch_minres_scalars(MinresScalars* S, cudaStream_t st);
// v_old <- Kz - (delta/gamma) v - (gamma/gamma_old) v_old  (after z <- z/gamma inside)
cudaError_t launch_minres_lanczos(MinresScalars* S, int64_t n, double* z, const double* Kz, const double* v,
                                  double* v_old, cudaStream_t st);
int64_t condense_scratch_doubles(const ElemSizes& s, int nsm);
cudaError_t launch_minres_update(MinresScalars* S, int64_t n, const double* z, double* w, double* w_old,
                                 double* x, cudaStream_t st);
cudaError_t launch_minres_scale(MinresScalars* S, int64_t n, const double* zin, double* z, cudaStream_t st);
cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);

}  // namespace mcs
