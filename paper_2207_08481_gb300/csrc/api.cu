// C-ABI of libmcs: handle management, set-up, condensation and the Krylov driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <exception>
#include <limits>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "handle.h"

using namespace mcs;

namespace {

thread_local std::string g_err = "no error";

template <class F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const McsError& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return MCS_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return MCS_ERR_INVALID_ARG;
  } catch (...) {
    g_err = "unknown error";
    return MCS_ERR_INVALID_ARG;
  }
}

// Installs the handle's profiler (if enabled) for the duration of an API call.
struct ProfScope {
  Profiler* prev;
  explicit ProfScope(Profiler* p) : prev(g_prof) { g_prof = p; }
  ~ProfScope() { g_prof = prev; }
};

ElemSizes elem_sizes(const Sizes& s) {
  ElemSizes e;
  e.d = s.d; e.k = s.k; e.nk = s.nk; e.nF = s.nF; e.nFm1 = s.nFm1; e.n_u = s.n_u; e.n_A = s.n_A;
  e.n_hat = s.n_hat; e.nhF = s.nhF; e.n_p = s.n_p; e.n_s0 = s.n_s0; e.n_raw = s.n_raw; e.n_con = s.n_con;
  e.n_w = s.n_w; e.n_wskew = s.n_wskew; e.n_cc = s.n_cc; e.n_bub = s.n_bub; e.n_c = s.n_c; e.mF = s.mF;
  e.ntF = s.ntF; e.lowest = s.lowest; e.lo_stab = 0;
  return e;
}

}  // namespace

namespace {

void validate_options(const mcs_options& o) {
  if (o.precision != MCS_FP64 && o.precision != MCS_MIXED) throw McsError(MCS_ERR_INVALID_ARG, "precision");
  if (o.smooth_steps < 0 || o.smooth_steps > 16) throw McsError(MCS_ERR_INVALID_ARG, "smooth_steps");
  if (o.gmg_smooth < 1 || o.gmg_smooth > 16) throw McsError(MCS_ERR_INVALID_ARG, "gmg_smooth");
  if (!(o.rtol > 0) || o.maxit < 1) throw McsError(MCS_ERR_INVALID_ARG, "rtol/maxit");
  if (o.residual_dd < -1 || o.residual_dd > 1) throw McsError(MCS_ERR_INVALID_ARG, "residual_dd");
  if (o.asp < 0 || o.asp > 1) throw McsError(MCS_ERR_INVALID_ARG, "asp");
  if (o.lo_stab < 0 || o.lo_stab > 1) throw McsError(MCS_ERR_INVALID_ARG, "lo_stab");
  if (o.outflow < 0 || o.outflow > 1) throw McsError(MCS_ERR_INVALID_ARG, "outflow");
  if (!(o.etol >= 0)) throw McsError(MCS_ERR_INVALID_ARG, "etol");
  if (o.etol > 0 && !(o.inner_rtol > 0 && o.inner_rtol < 1)) throw McsError(MCS_ERR_INVALID_ARG, "inner_rtol");
  if (o.tune < 0 || o.tune > 1) throw McsError(MCS_ERR_INVALID_ARG, "tune");
  if (o.facet_push < 0 || o.facet_push > 1) throw McsError(MCS_ERR_INVALID_ARG, "facet_push");
}

template <class R>
std::vector<R> cast_vec(const std::vector<double>& v) {
  return std::vector<R>(v.begin(), v.end());
}

// dense inverse of an SPD matrix (Cholesky), host FP64
std::vector<double> spd_inverse(const Csr& A) {
  const int64_t n = A.nrows;
  std::vector<double> M(n * n, 0.0);
  for (int64_t r = 0; r < n; ++r)
    for (int64_t t = A.rowptr[r]; t < A.rowptr[r + 1]; ++t) M[r * n + A.col[t]] = A.val[t];
  // Cholesky M = L L^T
  for (int64_t j = 0; j < n; ++j) {
    double s = M[j * n + j];
    for (int64_t p = 0; p < j; ++p) s -= M[j * n + p] * M[j * n + p];
    if (!(s > 0)) throw McsError(MCS_ERR_INVALID_ARG, "coarse operator not SPD");
    double l = std::sqrt(s);
    M[j * n + j] = l;
    for (int64_t i = j + 1; i < n; ++i) {
      double v = M[i * n + j];
      for (int64_t p = 0; p < j; ++p) v -= M[i * n + p] * M[j * n + p];
      M[i * n + j] = v / l;
    }
  }
  std::vector<double> Inv(n * n, 0.0), y(n);
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = 0; i < n; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int64_t p = 0; p < i; ++p) v -= M[i * n + p] * y[p];
      y[i] = v / M[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double v = y[i];
      for (int64_t p = i + 1; p < n; ++p) v -= M[p * n + i] * Inv[p * n + c];
      Inv[i * n + c] = v / M[i * n + i];
    }
  }
  return Inv;
}

std::vector<int32_t> to_i32(const std::vector<int64_t>& v) {
  std::vector<int32_t> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    if (v[i] > 0x7fffffff) throw McsError(MCS_ERR_UNSUPPORTED, "sparse matrix too large for int32 indices");
    o[i] = (int32_t)v[i];
  }
  return o;
}

// CSR -> column-major ELL on the device (precision R)
template <class R>
Ell to_ell(mcs_handle* h, const Csr& M) {
  Ell E;
  E.n = M.nrows;
  int64_t k = 0;
  for (int64_t r = 0; r < M.nrows; ++r) k = std::max<int64_t>(k, M.rowptr[r + 1] - M.rowptr[r]);
  if (M.ncols < 1) k = 0;
  E.k = (int)k;
  std::vector<int32_t> col(std::max<int64_t>(1, k * M.nrows));
  std::vector<R> val(std::max<int64_t>(1, k * M.nrows), (R)0);
  for (int64_t r = 0; r < M.nrows; ++r) {
    int64_t q = 0;
    for (int64_t t = M.rowptr[r]; t < M.rowptr[r + 1]; ++t, ++q) {
      col[q * M.nrows + r] = M.col[t];
      val[q * M.nrows + r] = (R)M.val[t];
    }
    for (; q < k; ++q) col[q * M.nrows + r] = 0;  // padding: value 0 at a column that exists
  }
  E.col = h->upload(col);
  E.val = h->upload(val);
  return E;
}

template <class R>
void build_precision(mcs_handle* h, PrecData<R>& P, const std::vector<Csr>& A, const std::vector<Csr>& Pr,
                     const std::vector<Csr>& Rt, const std::vector<double>& coarse_inv,
                     const std::vector<double>& Eb, const std::vector<int32_t>& fvr,
                     const std::vector<int32_t>& vf_ptr, const std::vector<int32_t>& vf_idx,
                     const std::vector<int32_t>& clist) {
  const Sizes& s = h->sz;
  const int64_t ne = h->mesh.ne, nint = h->mesh.nint;
  P.Fs = h->dalloc<R>(nint * (int64_t)fs_stride(s));
  cuda_check(cudaMemset((void*)P.Fs, 0, sizeof(R) * nint * (int64_t)fs_stride(s)), "memset");  // padding
  P.G = h->dalloc<R>(ne * (int64_t)g_stride(s));
  P.Aoi = h->dalloc<R>(ne * (int64_t)a_stride(s));
  {
    // device layout [nint][d][mF][d] (facet vertex w, mode t, component a): each of the d vertices of a
    // facet reads one contiguous slice in E^d^T
    const int d = h->d, mF = s.mF, dd = d * d;
    std::vector<R> Et(Eb.size());
    for (int64_t rk = 0; rk < nint; ++rk)
      for (int t = 0; t < mF; ++t)
        for (int w = 0; w < d; ++w)
          for (int a = 0; a < d; ++a) Et[((rk * d + w) * mF + t) * d + a] = (R)Eb[(rk * mF + t) * dd + w * d + a];
    P.Eb = h->upload(Et);
  }
  P.fvr = h->upload(fvr);
  P.vf_ptr = h->upload(vf_ptr);
  P.vf_idx = h->upload(vf_idx);
  P.nP1 = h->np1 / h->d;
  P.colour_list = h->upload(clist);
  P.colour_off = h->colour_off.data();
  P.ncol = h->ncol;
  P.smooth = h->opt.smooth_steps;
  P.gmg_smooth = h->opt.gmg_smooth;
  P.multiplicative = h->opt.asp == 0 ? 1 : 0;
  P.nlev = h->nlev;
  for (int l = 0; l < h->nlev; ++l) {
    GmgLevel& G = P.lev[l];
    G.n = A[l].nrows;
    G.A = to_ell<R>(h, A[l]);
    std::vector<double> dl1(A[l].nrows, 0.0);
    for (int64_t r = 0; r < A[l].nrows; ++r) {
      double sabs = 0;
      for (int64_t t = A[l].rowptr[r]; t < A[l].rowptr[r + 1]; ++t) sabs += std::fabs(A[l].val[t]);
      dl1[r] = 1.0 / sabs;
    }
    G.dl1inv = h->upload(cast_vec<R>(dl1));
    if (l > 0) {
      G.P = to_ell<R>(h, Pr[l]);
      G.Rt = to_ell<R>(h, Rt[l]);
    }
    P.pb[l] = h->dalloc<R>(G.n);
    P.px[l] = h->dalloc<R>(G.n);
    P.pr[l] = h->dalloc<R>(G.n);
    P.ptmp[l] = h->dalloc<R>(G.n);
  }
  P.coarse_inv = h->upload(coarse_inv);
  const int64_t n = precond_layout(h->L, h->es, (int)sizeof(R)).ndof;  // facet-interleaved layout
  P.b = h->dalloc<R>(n);
  P.x = h->dalloc<R>(n);
  P.t = h->dalloc<R>(n);
  P.rr = h->dalloc<R>(n);
  P.zz = h->dalloc<R>(n);
  P.push_warps = (h->opt.facet_push == 1 && P.multiplicative) ? facet_push_warps<R>(h->es) : 0;
  if (P.push_warps > 0) {
    const int64_t ndd = nint * (int64_t)facet_stride(h->es, (int)sizeof(R));
    P.q0 = h->dalloc<R>(ndd);
    P.q1 = h->dalloc<R>(ndd);
  }
  P.coarse_tmp = nullptr;
  P.err = h->dalloc<int>(1);
  cuda_check(cudaMemset(P.err, 0, sizeof(int)), "memset");
  const char* dbg = std::getenv("MCS_DEBUG_CHECKS");
  if (dbg && dbg[0] == '1') {
    P.debug = true;
    h->use_graphs = false;  // the diagnostics synchronise after launches
    P.dbg = h->dalloc<int>(8);
    cuda_check(cudaMemset(P.dbg, 0, 8 * sizeof(int)), "memset");
  }
}

void finish_setup(mcs_handle* h, std::vector<HostMesh>& levels) {
  const int d = h->d;
  HostMesh& m = h->mesh;
  h->ref = build_reference(d, h->k);
  h->sz = h->ref.s;
  h->es = elem_sizes(h->sz);
  h->es.lo_stab = h->sz.lowest ? h->opt.lo_stab : 0;
  const Sizes& s = h->sz;
  // layout
  Layout& L = h->L;
  L.ne = m.ne;
  L.nint = m.nint;
  L.n_dd = m.nint * s.nF;
  L.n_oo = m.ne * s.n_bub;
  L.n_hat = m.nint * s.nhF;
  L.n_pres = m.ne * s.n_p;
  L.off_o = L.n_dd;
  L.off_h = L.n_dd + L.n_oo;
  L.off_p = L.off_h + L.n_hat;
  L.ndof = L.off_p + L.n_pres;
  // |det J|
  std::vector<double> adet(m.ne);
  h->total_adet = 0;
  for (int64_t T = 0; T < m.ne; ++T) {
    const int32_t* e = &m.elems[T * (d + 1)];
    double J[9];
    for (int a = 0; a < d; ++a)
      for (int i = 0; i < d; ++i) J[a * d + i] = m.coords[e[i + 1] * d + a] - m.coords[e[0] * d + a];
    double det = (d == 2) ? J[0] * J[3] - J[1] * J[2]
                          : J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                                J[2] * (J[3] * J[7] - J[4] * J[6]);
    adet[T] = std::fabs(det);
    h->total_adet += adet[T];
    if (adet[T] == 0.0) throw McsError(MCS_ERR_INVALID_ARG, "degenerate element");
  }
  // interior facet -> elements / local index
  std::vector<int32_t> fel(m.nint * 2), floc(m.nint * 2);
  for (int64_t r = 0; r < m.nint; ++r) {
    int32_t F = m.int_facets[r];
    fel[r * 2] = m.facet_elems[F * 2];
    fel[r * 2 + 1] = m.facet_elems[F * 2 + 1];
    floc[r * 2] = m.int_local[r * 2];
    floc[r * 2 + 1] = std::max(0, m.int_local[r * 2 + 1]);   // outflow facet: no second element, zero slab
  }
  DevMesh& dm = h->dm;
  dm.d = d;
  dm.ne = m.ne;
  dm.nint = m.nint;
  dm.coords = h->upload(m.coords);
  dm.elems = h->upload(m.elems);
  dm.elem_rank = h->upload(m.elem_rank);
  dm.signs = h->upload(m.signs);
  dm.adet = h->upload(adet);
  dm.fel = h->upload(fel);
  dm.floc = h->upload(floc);
  std::vector<int32_t> fsr(m.nint * 2 * (d + 1));
  for (int64_t r = 0; r < m.nint; ++r)
    for (int side = 0; side < 2; ++side)
      for (int f = 0; f <= d; ++f)
        fsr[(r * 2 + side) * (d + 1) + f] = fel[r * 2 + side] < 0 ? -1 : m.elem_rank[fel[r * 2 + side] * (d + 1) + f];
  dm.fsr = h->upload(fsr);
  h->outflow = !m.outflow.empty();
  dm.fout = nullptr;
  if (h->outflow) {
    std::vector<int8_t> fout(m.nint, 0);
    for (int64_t r = 0; r < m.nint; ++r) fout[r] = m.outflow[m.int_facets[r]];
    dm.fout = h->upload(fout);
  }
  // tables
  DevTables& dt = h->dt;
  const RefTables& R = h->ref;
  dt.B0 = h->upload(R.B0);
  dt.Rf = h->upload(R.Rf);
  dt.Bh = h->upload(R.Bh);
  dt.Ccon = h->upload(R.Ccon);
  dt.Adiv = h->upload(R.Adiv);
  dt.nhat = h->upload(R.nhat);
  dt.Wmom = h->upload(R.Wmom);
  dt.Bp = h->upload(R.Bp);
  {
    std::vector<float> hi(R.Bp.size()), lo(R.Bp.size());
    for (size_t i = 0; i < R.Bp.size(); ++i) {
      hi[i] = (float)R.Bp[i];
      lo[i] = (float)(R.Bp[i] - (double)hi[i]);
    }
    dt.Bp_hi = h->upload(hi);
    dt.Bp_lo = h->upload(lo);
  }
  dt.Mu = h->upload(R.Mu);
  dt.phi_load = h->upload(R.phi_load);
  dt.xq_load = h->upload(R.xq_load);
  dt.wq_load = h->upload(R.wq_load);
  dt.nq_load = R.nq_load;
  // colouring
  h->colour = colour_facets(m, &h->ncol);
  std::vector<int32_t> clist;
  h->colour_off.assign(h->ncol + 1, 0);
  for (int c = 0; c < h->ncol; ++c) {
    h->colour_off[c] = (int64_t)clist.size();
    for (int64_t r = 0; r < m.nint; ++r)
      if (h->colour[r] == c) clist.push_back((int32_t)r);
  }
  h->colour_off[h->ncol] = (int64_t)clist.size();
  h->fpos.assign(m.nint, -1);
  for (size_t li = 0; li < clist.size(); ++li) h->fpos[clist[li]] = (int32_t)li;
  dm.fpos = h->upload(h->fpos);
  {
    // facet records in colour order
    std::vector<int32_t> rec(clist.size() * 16, -1);
    for (size_t li = 0; li < clist.size(); ++li) {
      const int32_t r = clist[li];
      int32_t* o = &rec[li * 16];
      o[0] = r;
      o[1] = fel[r * 2];
      o[2] = fel[r * 2 + 1];
      o[3] = floc[r * 2];
      o[4] = floc[r * 2 + 1];
      for (int side = 0; side < 2; ++side)
        for (int f = 0; f <= d; ++f) o[5 + side * (d + 1) + f] = fsr[(r * 2 + side) * (d + 1) + f];
      // [13]: bit side*(d+1) + f set when element o[1 + side] is side 1 of the facet o[5 + side*(d+1) + f]
      int32_t bits = 0;
      for (int side = 0; side < 2; ++side)
        for (int f = 0; f <= d; ++f) {
          const int32_t H = o[5 + side * (d + 1) + f], T = o[1 + side];
          if (H < 0 || T < 0) continue;
          if (fel[H * 2] == T) continue;
          if (fel[H * 2 + 1] != T) throw McsError(MCS_ERR_INVALID_ARG, "inconsistent facet-element incidence");
          bits |= 1 << (side * (d + 1) + f);
        }
      o[13] = bits;
    }
    dm.frec = reinterpret_cast<const int4*>(h->upload(rec));
  }
  // conforming space and multigrid
  std::vector<P1Space> sp;
  std::vector<Csr> A, Pr, Rt;
  for (size_t l = 0; l < levels.size(); ++l) {
    sp.push_back(p1_space(levels[l]));
    A.push_back(abar_matrix(levels[l], sp[l], h->nu, h->k));
  }
  Pr.resize(levels.size());
  Rt.resize(levels.size());
  for (size_t l = 1; l < levels.size(); ++l) {
    Pr[l] = prolongation(d, h->level_N[l - 1], sp[l - 1], sp[l]);
    Rt[l] = transpose(Pr[l]);
  }
  h->np1 = sp.back().n * d;
  if (A[0].nrows > 6000) throw McsError(MCS_ERR_UNSUPPORTED, "coarsest multigrid level too large for a dense solve");
  std::vector<double> cinv = spd_inverse(A[0]);
  // E^d structures
  std::vector<double> Eb = embedding_blocks(m, R);
  const P1Space& p1 = sp.back();
  std::vector<int32_t> fvr(m.nint * d);
  std::vector<std::vector<std::pair<int32_t, int32_t>>> inc(p1.n);
  for (int64_t r = 0; r < m.nint; ++r) {
    int32_t F = m.int_facets[r];
    for (int w = 0; w < d; ++w) {
      int32_t vr = p1.vrank[m.facets[F * d + w]];
      fvr[r * d + w] = vr;
      if (vr >= 0) inc[vr].push_back({(int32_t)r, w});
    }
  }
  std::vector<int32_t> vf_ptr(p1.n + 1, 0), vf_idx;
  for (int64_t v = 0; v < p1.n; ++v) {
    for (auto& pr : inc[v]) {
      vf_idx.push_back(pr.first);
      vf_idx.push_back(pr.second);
    }
    vf_ptr[v + 1] = (int32_t)(vf_idx.size() / 2);
  }
  if (h->opt.precision == MCS_MIXED)
    build_precision<float>(h, h->pf, A, Pr, Rt, cinv, Eb, fvr, vf_ptr, vf_idx, clist);
  else
    build_precision<double>(h, h->pd, A, Pr, Rt, cinv, Eb, fvr, vf_ptr, vf_idx, clist);
  // condensed operator and Krylov work
  if (h->opt.precision == MCS_MIXED) {
    h->K.Ahi = h->dalloc<float>(m.ne * (int64_t)packed_pad(s));
    h->K.Alo = h->dalloc<float>(m.ne * (int64_t)packed_pad(s));
  } else {
    h->K.AT = h->dalloc<double>(m.ne * (int64_t)s.n_A * s.n_A);
  }
  for (int i = 0; i < 12; ++i) h->kv[i] = h->dalloc<double>(L.ndof);
  h->ydd = h->dalloc<double>(4 * L.ndof);
  // an outflow facet has one element, so one of its two row-sum slots is never written: keep it 0
  cuda_check(cudaMemset(h->ydd, 0, sizeof(double) * 4 * L.ndof), "memset");
  cuda_check(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  h->scratch = h->dalloc<double>(4096);
  cuda_check(cudaMemset(h->scratch, 0, sizeof(double) * 4096), "memset");
  h->S = h->dalloc<MinresScalars>(1);
  cuda_check(cudaMallocHost(&h->S_host, sizeof(MinresScalars)), "cudaMallocHost");
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  h->cond_scratch_doubles = condense_scratch_doubles(h->es, nsm);
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (condense_slot_bytes(h->es) > maxsm || recover_slot_doubles(h->es) * 8 > maxsm)
    h->cond_scratch = h->dalloc<double>(h->cond_scratch_doubles);
  // wait for this set-up's own work only (legacy-stream memsets, the handle's stream): work of
  // other handles on other streams keeps running
  cuda_check(cudaStreamSynchronize(0), "setup");
  cuda_check(cudaStreamSynchronize(h->stream), "setup");
}

mcs_handle* new_handle(int dim, int k, double nu, const mcs_options* opt, void* stream) {
  if (dim < 2 || dim > 3) throw McsError(MCS_ERR_UNSUPPORTED, "dim must be 2 or 3");
  // k = 1 is the lowest-order variant of Sec. 7, which the paper states for d = 3 (vector rotations).
  if (k < 1 || k > 6) throw McsError(MCS_ERR_UNSUPPORTED, "k must be in 1..6");
  if (k == 1 && dim != 3) throw McsError(MCS_ERR_UNSUPPORTED, "k = 1 (lowest-order variant) needs dim = 3");
  if (!(nu > 0)) throw McsError(MCS_ERR_INVALID_ARG, "nu must be positive");
  auto h = std::make_unique<mcs_handle>();
  h->d = dim;
  h->k = k;
  h->nu = nu;
  if (opt) h->opt = *opt;
  else mcs_default_options(&h->opt);
  validate_options(h->opt);
  if (h->opt.tune_cache) {   // the caller's string need not outlive the call
    h->tune_cache = h->opt.tune_cache;
    h->opt.tune_cache = h->tune_cache.c_str();
  }
  if (h->opt.outflow && k == 1) throw McsError(MCS_ERR_UNSUPPORTED, "outflow with k = 1");
  h->stream = (cudaStream_t)stream;
  cuda_check(cudaGetDevice(&h->device), "cudaGetDevice");
  return h.release();
}

}  // namespace

void mcs::set_last_error(const char* msg) { g_err = msg ? msg : "unknown error"; }

namespace {
// The tuned launch shapes of a handle: from the cache file when it has a line for this (dim, k, precision,
// element count), else by timing the candidates (autotune_launches), then appended to the cache.
template <class R>
void tune_handle(mcs_handle* h, PrecData<R>& P) {
  char key[160];
  std::snprintf(key, sizeof(key), "mcs-tune dim=%d k=%d precision=%d ne=%lld lo_stab=%d", h->d, h->k,
                h->opt.precision, (long long)h->mesh.ne, h->es.lo_stab);
  if (h->opt.tune_cache) {
    if (FILE* f = std::fopen(h->opt.tune_cache, "r")) {
      char line[512];
      while (std::fgets(line, sizeof(line), f)) {
        if (std::strncmp(line, key, std::strlen(key)) != 0 || line[std::strlen(key)] != ' ') continue;
        int fb = -1, th = -1, eb = -1;
        if (std::sscanf(line + std::strlen(key), " fb=%d threads=%d eb=%d", &fb, &th, &eb) == 3) {
          P.fb = fb;
          P.fthreads = th;
          h->K.eb = eb;
          std::fclose(f);
          h->tuned = true;
          return;
        }
      }
      std::fclose(f);
    }
  }
  char report[4096] = {0};
  cuda_check(autotune_launches<R>(h->es, h->dt, h->dm, h->L, P, h->K, h->kv[0], h->kv[1], h->stream, report,
                                  (int)sizeof(report)),
             "autotune");
  h->tuned = true;
  if (h->opt.tune_cache) {
    if (FILE* f = std::fopen(h->opt.tune_cache, "a")) {
      std::fprintf(f, "%s fb=%d threads=%d eb=%d  # %s\n", key, P.fb, P.fthreads, h->K.eb, report);
      std::fclose(f);
    }
  }
}
}  // namespace

namespace {
template <class R>
void condense_batch(mcs_handle* const* hs, int count) {
  mcs_handle* h0 = hs[0];
  cudaStream_t st = h0->stream;
  std::vector<CondenseItem<R>> items(count);
  int64_t total = 0, slot_bytes = 0;
  for (int i = 0; i < count; ++i) {
    mcs_handle* h = hs[i];
    PrecData<R>& P = *reinterpret_cast<PrecData<R>*>(sizeof(R) == 4 ? (void*)&h->pf : (void*)&h->pd);
    CondenseItem<R>& it = items[i];
    it.s = h->es;
    it.t = h->dt;
    it.m = h->dm;
    it.nu = h->nu;
    it.K = h->K;
    it.Fs = P.Fs;
    it.G = const_cast<R*>(P.G);
    it.Aoi = const_cast<R*>(P.Aoi);
    it.first = total;
    total += h->mesh.ne;
    slot_bytes = std::max<int64_t>(slot_bytes, condense_slot_bytes(h->es));
  }
  // order against the other handles' streams
  std::vector<cudaEvent_t> evs;
  auto event_on = [&](cudaStream_t s) {
    cudaEvent_t e;
    cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    evs.push_back(e);
    cuda_check(cudaEventRecord(e, s), "cudaEventRecord");
    return e;
  };
  for (int i = 1; i < count; ++i)
    if (hs[i]->stream != st) cuda_check(cudaStreamWaitEvent(st, event_on(hs[i]->stream), 0), "wait");
  int nsm = 0;
  cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h0->device), "attribute");
  // up to 4 blocks per SM, fewer where their workspaces would exceed 2 GiB (3D k = 6: 6 MB each)
  int64_t blocks = std::min<int64_t>((int64_t)nsm * 4, std::max<int64_t>(total, 1));
  while (blocks > nsm && blocks * slot_bytes > (int64_t(2) << 30)) blocks -= nsm;
  const int64_t scratch_doubles = blocks * (slot_bytes / 8);
  void* items_dev = nullptr;
  double* scratch = nullptr;
  cuda_check(cudaMallocAsync(&items_dev, sizeof(CondenseItem<R>) * count, st), "cudaMallocAsync");
  cudaError_t e = cudaMallocAsync((void**)&scratch, sizeof(double) * scratch_doubles, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(items_dev, st);
    throw McsError(MCS_ERR_OOM, "batched condensation workspace");
  }
  cuda_check(cudaMemcpyAsync(items_dev, items.data(), sizeof(CondenseItem<R>) * count, cudaMemcpyHostToDevice, st),
             "copy items");
  e = launch_condense_batch<R>((const CondenseItem<R>*)items_dev, items.data(), count, scratch, scratch_doubles, st);
  cudaFreeAsync(scratch, st);
  cudaFreeAsync(items_dev, st);
  cuda_check(e, "condense batch");
  // the items were copied from pageable memory before the call returned; facet blocks per problem
  for (int i = 0; i < count; ++i) {
    PrecData<R>& P = *reinterpret_cast<PrecData<R>*>(sizeof(R) == 4 ? (void*)&hs[i]->pf : (void*)&hs[i]->pd);
    cuda_check(launch_facet_blocks<R>(hs[i]->es, hs[i]->dm, P.Fs, st), "facet blocks");
    hs[i]->condensed = true;
  }
  for (int i = 1; i < count; ++i)
    if (hs[i]->stream != st) cuda_check(cudaStreamWaitEvent(hs[i]->stream, event_on(st), 0), "wait");
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
}
}  // namespace

extern "C" {

int mcs_version(void) { return 200; }



const char* mcs_last_error(void) { return g_err.c_str(); }

int mcs_default_options(mcs_options* o) {
  if (!o) return MCS_ERR_INVALID_ARG;
  o->precision = MCS_MIXED;
  o->smooth_steps = 2;
  o->gmg_levels = -1;
  o->gmg_smooth = 2;
  o->rtol = 1e-8;
  o->maxit = 1000;
  o->max_refine = 8;
  o->inner_rtol = 1e-5;
  o->residual_dd = -1;
  o->asp = 0;
  o->lo_stab = 0;
  o->outflow = 0;
  o->etol = 0.0;
  o->tune = 0;
  o->tune_cache = nullptr;
  o->facet_push = 1;
  return MCS_OK;
}

int mcs_setup_structured(int dim, int N, int k, double nu, const mcs_options* opt, void* stream,
                         mcs_handle** out) {
  return guarded([&]() -> int {
    if (!out) throw McsError(MCS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (N < 1 || N > 4096) throw McsError(MCS_ERR_INVALID_ARG, "N out of range");
    std::unique_ptr<mcs_handle> h(new_handle(dim, k, nu, opt, stream));
    int levels = h->opt.gmg_levels;
    if (levels < 0) {
      const int target = (dim == 2) ? 16 : 4;
      levels = 1;
      int n = N;
      while (n > target && n % 2 == 0) {
        n /= 2;
        ++levels;
      }
    }
    if (levels < 1 || levels > 12) throw McsError(MCS_ERR_INVALID_ARG, "gmg_levels out of range");
    if (N % (1 << (levels - 1)) != 0) throw McsError(MCS_ERR_INVALID_ARG, "N not divisible by 2^(levels-1)");
    h->nlev = levels;
    std::vector<HostMesh> lv;
    for (int l = 0; l < levels; ++l) {
      int Nl = N >> (levels - 1 - l);
      h->level_N.push_back(Nl);
      lv.push_back(l + 1 == levels ? structured_mesh(dim, N) : structured_mesh(dim, Nl));
      if (h->opt.outflow) mark_outflow(lv.back());
    }
    h->mesh = lv.back();
    finish_setup(h.get(), lv);
    *out = h.release();
    return MCS_OK;
  });
}

int mcs_setup_mesh(int dim, int64_t nv, const double* coords, int64_t ne, const int32_t* elems, int k,
                   double nu, const mcs_options* opt, void* stream, mcs_handle** out) {
  return guarded([&]() -> int {
    if (!out || !coords || !elems || nv < 1 || ne < 1) throw McsError(MCS_ERR_INVALID_ARG, "bad mesh arguments");
    *out = nullptr;
    std::unique_ptr<mcs_handle> h(new_handle(dim, k, nu, opt, stream));
    if (h->opt.outflow) throw McsError(MCS_ERR_UNSUPPORTED, "outflow needs mcs_setup_structured");
    HostMesh m;
    m.d = dim;
    m.nv = nv;
    m.ne = ne;
    m.coords.assign(coords, coords + nv * dim);
    m.elems.assign(elems, elems + ne * (dim + 1));
    for (int64_t T = 0; T < ne; ++T)
      for (int v = 0; v <= dim; ++v) {
        int32_t id = m.elems[T * (dim + 1) + v];
        if (id < 0 || id >= nv) throw McsError(MCS_ERR_INVALID_ARG, "vertex id out of range");
        if (v > 0 && id <= m.elems[T * (dim + 1) + v - 1])
          throw McsError(MCS_ERR_INVALID_ARG, "element vertex ids must be ascending");
      }
    build_facets(m);
    h->nlev = 1;
    h->level_N.push_back(0);
    std::vector<HostMesh> lv{m};
    h->mesh = m;
    finish_setup(h.get(), lv);
    *out = h.release();
    return MCS_OK;
  });
}

int mcs_sizes(const mcs_handle* h, mcs_sizes_t* s) {
  return guarded([&]() -> int {
    if (!h || !s) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    const Layout& L = h->L;
    s->ndof = L.ndof; s->n_dd = L.n_dd; s->n_oo = L.n_oo; s->n_hat = L.n_hat; s->n_pres = L.n_pres;
    s->off_o = L.off_o; s->off_h = L.off_h; s->off_p = L.off_p;
    s->ne = h->mesh.ne; s->nint = h->mesh.nint; s->nfacets = h->mesh.nf; s->nvertices = h->mesh.nv;
    s->np1 = h->np1;
    s->dim = h->d; s->k = h->k; s->nF = h->sz.nF; s->n_bub = h->sz.n_bub; s->nhF = h->sz.nhF;
    s->n_p = h->sz.n_p; s->n_A = h->sz.n_A; s->n_c = h->sz.n_c; s->mF = h->sz.mF;
    s->ncolours = h->ncol; s->gmg_levels = h->nlev;
    s->nq_load = h->ref.nq_load;
    s->bytes_resident = h->bytes;
    s->facet_batch = h->opt.precision == MCS_MIXED ? h->pf.fb : h->pd.fb;
    s->facet_threads = h->opt.precision == MCS_MIXED ? h->pf.fthreads : h->pd.fthreads;
    s->apply_batch = h->K.eb;
    s->push_warps = h->opt.precision == MCS_MIXED ? h->pf.push_warps : h->pd.push_warps;
    return MCS_OK;
  });
}

int mcs_export_mesh(const mcs_handle* h, int32_t* facets, int32_t* elem_facets, int8_t* signs, int32_t* colour) {
  return guarded([&]() -> int {
    if (!h) throw McsError(MCS_ERR_INVALID_ARG, "NULL handle");
    const HostMesh& m = h->mesh;
    if (facets) std::copy(m.facets.begin(), m.facets.end(), facets);
    if (elem_facets) std::copy(m.elem_facets.begin(), m.elem_facets.end(), elem_facets);
    if (signs) std::copy(m.signs.begin(), m.signs.end(), signs);
    if (colour) std::copy(h->colour.begin(), h->colour.end(), colour);
    return MCS_OK;
  });
}

int mcs_export_dofmap(const mcs_handle* h, int64_t* out) {
  return guarded([&]() -> int {
    if (!h || !out) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    const Sizes& s = h->sz;
    const Layout& L = h->L;
    const int d = h->d;
    const int nloc = s.n_A + s.n_p;
    for (int64_t T = 0; T < h->mesh.ne; ++T) {
      int64_t* o = out + T * nloc;
      const int32_t* er = &h->mesh.elem_rank[T * (d + 1)];
      for (int i = 0; i < s.n_A; ++i) {
        const int nfd = (d + 1) * s.nF;
        int64_t g;
        if (i < nfd) {
          int f = i / s.nF;
          g = er[f] < 0 ? -1 : (int64_t)er[f] * s.nF + (i - f * s.nF);
        } else if (i < s.n_u) {
          g = L.off_o + T * s.n_bub + (i - nfd);
        } else {
          int q = i - s.n_u, f = q / s.nhF;
          g = er[f] < 0 ? -1 : L.off_h + (int64_t)er[f] * s.nhF + (q - f * s.nhF);
        }
        o[i] = g;
      }
      for (int j = 0; j < s.n_p; ++j) o[s.n_A + j] = L.off_p + T * s.n_p + j;
    }
    return MCS_OK;
  });
}

int mcs_export_pattern(const mcs_handle* h, int64_t* rowptr, int32_t* col) {
  return guarded([&]() -> int {
    if (!h || !rowptr) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    const Sizes& s = h->sz;
    const int nloc = s.n_A + s.n_p;
    std::vector<int64_t> dm(h->mesh.ne * nloc);
    mcs_export_dofmap(h, dm.data());
    const int64_t n = h->L.ndof;
    // rows coupled through elements: velocity-velocity (A), velocity-pressure (B^T, B);
    // p-p block is zero
    std::vector<std::vector<int32_t>> rows(n);
    for (int64_t T = 0; T < h->mesh.ne; ++T) {
      const int64_t* o = &dm[T * nloc];
      for (int i = 0; i < nloc; ++i) {
        if (o[i] < 0) continue;
        for (int j = 0; j < nloc; ++j) {
          if (o[j] < 0) continue;
          bool ip = i >= s.n_A, jp = j >= s.n_A;
          if (ip && jp) continue;
          if ((ip && j >= s.n_u) || (jp && i >= s.n_u)) continue;  // p couples to u only
          rows[o[i]].push_back((int32_t)o[j]);
        }
      }
    }
    rowptr[0] = 0;
    for (int64_t r = 0; r < n; ++r) {
      auto& v = rows[r];
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
      rowptr[r + 1] = rowptr[r] + (int64_t)v.size();
      if (col) std::copy(v.begin(), v.end(), col + rowptr[r]);
    }
    return MCS_OK;
  });
}

int mcs_condense_batch(mcs_handle* const* handles, int count) {
  return guarded([&]() -> int {
    if (!handles || count < 1) throw McsError(MCS_ERR_INVALID_ARG, "NULL handles or count < 1");
    for (int i = 0; i < count; ++i) {
      if (!handles[i]) throw McsError(MCS_ERR_INVALID_ARG, "NULL handle");
      if (handles[i]->opt.precision != handles[0]->opt.precision)
        throw McsError(MCS_ERR_INVALID_ARG, "handles of different precisions");
      if (handles[i]->device != handles[0]->device) throw McsError(MCS_ERR_INVALID_ARG, "handles on different devices");
    }
    if (handles[0]->opt.precision == MCS_MIXED) condense_batch<float>(handles, count);
    else condense_batch<double>(handles, count);
    return MCS_OK;
  });
}

int mcs_condense(mcs_handle* h) {
  return guarded([&]() -> int {
    if (!h) throw McsError(MCS_ERR_INVALID_ARG, "NULL handle");
    ProfScope ps(h->prof.get());
    if (h->opt.precision == MCS_MIXED) {
      cuda_check(launch_condense<float>(h->es, h->dt, h->dm, h->nu, h->K, h->pf.Fs, (float*)h->pf.G,
                                        (float*)h->pf.Aoi, h->cond_scratch, h->cond_scratch_doubles, h->stream),
                 "condense");
      cuda_check(launch_facet_blocks<float>(h->es, h->dm, h->pf.Fs, h->stream), "facet blocks");
    } else {
      cuda_check(launch_condense<double>(h->es, h->dt, h->dm, h->nu, h->K, h->pd.Fs, (double*)h->pd.G,
                                         (double*)h->pd.Aoi, h->cond_scratch, h->cond_scratch_doubles, h->stream),
                 "condense");
      cuda_check(launch_facet_blocks<double>(h->es, h->dm, h->pd.Fs, h->stream), "facet blocks");
    }
    h->condensed = true;
    if (h->opt.tune && !h->tuned) {
      if (h->opt.precision == MCS_MIXED) tune_handle<float>(h, h->pf);
      else tune_handle<double>(h, h->pd);
    }
    return MCS_OK;
  });
}

int mcs_copy_element_matrices(const mcs_handle* h, int64_t T0, int64_t count, double* out) {
  return guarded([&]() -> int {
    if (!h || !out || T0 < 0 || count < 0 || T0 + count > h->mesh.ne) throw McsError(MCS_ERR_INVALID_ARG, "range");
    const int nA = h->sz.n_A;
    const int64_t np = (int64_t)nA * (nA + 1) / 2, full = (int64_t)nA * nA;
    cuda_check(cudaStreamSynchronize(h->stream), "sync");
    if (h->K.AT) {
      std::vector<double> tmp(full * count);
      cuda_check(cudaMemcpy(tmp.data(), h->K.AT + T0 * full, sizeof(double) * full * count, cudaMemcpyDeviceToHost),
                 "copy");
      for (int64_t T = 0; T < count; ++T)
        for (int i = 0; i < nA; ++i)
          for (int j = 0; j <= i; ++j)
            out[T * np + (int64_t)i * (i + 1) / 2 + j] = tmp[T * full + (int64_t)i * nA + j];
    } else {
      const int64_t pp = packed_pad(h->sz);
      std::vector<float> hi(pp * count), lo(pp * count);
      cuda_check(cudaMemcpy(hi.data(), h->K.Ahi + T0 * pp, sizeof(float) * pp * count, cudaMemcpyDeviceToHost), "copy");
      cuda_check(cudaMemcpy(lo.data(), h->K.Alo + T0 * pp, sizeof(float) * pp * count, cudaMemcpyDeviceToHost), "copy");
      for (int64_t T = 0; T < count; ++T)
        for (int64_t q = 0; q < np; ++q) out[T * np + q] = (double)hi[T * pp + q] + (double)lo[T * pp + q];
    }
    return MCS_OK;
  });
}

int mcs_copy_schur(const mcs_handle* h, int64_t T0, int64_t count, double* Ad_host, double* G_host) {
  return guarded([&]() -> int {
    if (!h || T0 < 0 || count < 0 || T0 + count > h->mesh.ne) throw McsError(MCS_ERR_INVALID_ARG, "range");
    const Sizes& s = h->sz;
    cuda_check(cudaStreamSynchronize(h->stream), "sync");
    auto fetch = [&](const void* src, int64_t per, double* dst) {
      if (h->opt.precision == MCS_MIXED) {
        std::vector<float> tmp(per * count);
        cuda_check(cudaMemcpy(tmp.data(), (const float*)src + T0 * per, sizeof(float) * per * count,
                              cudaMemcpyDeviceToHost), "copy");
        for (int64_t i = 0; i < per * count; ++i) dst[i] = tmp[i];
      } else {
        cuda_check(cudaMemcpy(dst, (const double*)src + T0 * per, sizeof(double) * per * count,
                              cudaMemcpyDeviceToHost), "copy");
      }
    };
    const void* Fs = h->opt.precision == MCS_MIXED ? (const void*)h->pf.Fs : (const void*)h->pd.Fs;
    const void* G = h->opt.precision == MCS_MIXED ? (const void*)h->pf.G : (const void*)h->pd.G;
    if (Ad_host) {
      // rows of interior facets from the facet stream; rows of boundary facets are not stored (NaN)
      const int64_t fss = fs_stride(s), nc2 = (int64_t)s.n_c * s.n_c, nint = h->mesh.nint;
      std::vector<double> stream(fss * nint);
      if (h->opt.precision == MCS_MIXED) {
        std::vector<float> tmp(fss * nint);
        cuda_check(cudaMemcpy(tmp.data(), Fs, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost), "copy");
        for (size_t i = 0; i < tmp.size(); ++i) stream[i] = tmp[i];
      } else {
        cuda_check(cudaMemcpy(stream.data(), Fs, sizeof(double) * stream.size(), cudaMemcpyDeviceToHost), "copy");
      }
      const int mF = s.mF, dp1 = s.d + 1, slab = slab_pad(s);
      for (int64_t e = 0; e < count; ++e) {
        const int64_t T = T0 + e;
        for (int f = 0; f < dp1; ++f) {
          const int32_t rk = h->mesh.elem_rank[T * dp1 + f];
          const double* blk = nullptr;
          if (rk >= 0) {
            const int32_t F = h->mesh.int_facets[rk];
            const int side = h->mesh.facet_elems[(int64_t)F * 2] == (int32_t)T ? 0 : 1;
            blk = stream.data() + (int64_t)h->fpos[rk] * fss + side * slab;
          }
          for (int t = 0; t < mF; ++t)
            for (int c = 0; c < s.n_c; ++c)
              Ad_host[e * nc2 + (int64_t)(f * mF + t) * s.n_c + c] = blk ? blk[c * mF + t] : std::nan("");
        }
      }
    }
    if (G_host) {
      const int64_t per = g_stride(s), ng = (int64_t)s.n_bub * s.n_c;
      std::vector<double> tmp(per * count);
      fetch(G, per, tmp.data());
      for (int64_t T = 0; T < count; ++T)
        for (int64_t q = 0; q < ng; ++q) G_host[T * ng + q] = tmp[T * per + q];
    }
    return MCS_OK;
  });
}

int mcs_load_points(mcs_handle* h, double* xq) {
  return guarded([&]() -> int {
    if (!h || !xq) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    cuda_check(launch_load_points(h->es, h->dt, h->dm, xq, h->stream), "load points");
    return MCS_OK;
  });
}

int mcs_load_vector(mcs_handle* h, const double* fq, double* F) {
  return guarded([&]() -> int {
    if (!h || !fq || !F) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    cuda_check(launch_load(h->es, h->dt, h->dm, h->L, fq, F, h->stream), "load vector");
    return MCS_OK;
  });
}

int mcs_mass_velocity(mcs_handle* h, const double* c, double* F) {
  return guarded([&]() -> int {
    if (!h || !c || !F) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    cuda_check(launch_mass_u(h->es, h->dt, h->dm, h->L, c, F, h->stream), "mass");
    return MCS_OK;
  });
}

int mcs_apply(mcs_handle* h, const double* x, double* y) {
  return guarded([&]() -> int {
    if (!h || !x || !y) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    ProfScope ps(h->prof.get());
    if (!h->condensed) throw McsError(MCS_ERR_INVALID_ARG, "mcs_condense has not been called");
    cuda_check(launch_apply_K(h->es, h->dt, h->dm, h->L, h->K, x, y, nullptr, h->stream), "apply");
    return MCS_OK;
  });
}

int mcs_residual(mcs_handle* h, const double* F, const double* x, double* r) {
  return guarded([&]() -> int {
    if (!h || !F || !x || !r) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    if (!h->condensed) throw McsError(MCS_ERR_INVALID_ARG, "mcs_condense has not been called");
    if (r == x) throw McsError(MCS_ERR_INVALID_ARG, "r must not alias x");
    cuda_check(launch_residual_dd(h->es, h->dt, h->dm, h->L, h->K, F, x, h->ydd, r, h->stream), "residual");
    return MCS_OK;
  });
}

static void precond_any(mcs_handle* h, const double* r, double* z, const int* stop, cudaStream_t st = nullptr) {
  if (!st) st = h->stream;
  cudaError_t e = (h->opt.precision == MCS_MIXED)
                      ? launch_precond<float>(h->es, h->dt, h->dm, h->L, h->nu, h->pf, r, z, stop, st)
                      : launch_precond<double>(h->es, h->dt, h->dm, h->L, h->nu, h->pd, r, z, stop, st);
  cuda_check(e, "precond");
}

int mcs_precond(mcs_handle* h, const double* r, double* z) {
  return guarded([&]() -> int {
    if (!h || !r || !z) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    ProfScope ps(h->prof.get());
    if (!h->condensed) throw McsError(MCS_ERR_INVALID_ARG, "mcs_condense has not been called");
    precond_any(h, r, z, nullptr);
    return MCS_OK;
  });
}

namespace {

// One preconditioned MinRes iteration (all scalars stay on the device; kernels return early once
// the state says stop).  The vector roles rotate: after two iterations they are back in place.
void minres_iteration(mcs_handle* h, cudaStream_t st, double*& v_old, double*& v, double*& z, double*& zn,
                      double*& w_old, double*& w, double* Kz, double* x_acc) {
  const int64_t n = h->L.ndof;
  MinresScalars* S = h->S;
  const int* stop = &S->stop;
  cuda_check(launch_minres_scale(S, n, z, z, st), "scale");
  cuda_check(launch_apply_K(h->es, h->dt, h->dm, h->L, h->K, z, Kz, stop, st), "apply");
  cuda_check(launch_dot(Kz, z, n, h->scratch, &S->delta, stop, st), "dot");
  cuda_check(launch_minres_lanczos(S, n, z, Kz, v, v_old, st), "lanczos");
  precond_any(h, v_old, zn, stop, st);
  if (!h->outflow)   // pure Dirichlet: p is fixed by its mean (reading R6); with Gamma_Ntilde it is unique
    cuda_check(launch_mean_zero(h->dm, h->L, h->sz.n_p, zn, h->scratch, h->total_adet, stop, st), "mean");
  cuda_check(launch_dot(zn, v_old, n, h->scratch, &S->dot1, stop, st), "dot");
  cuda_check(launch_minres_scalars(S, st), "scalars");
  cuda_check(launch_minres_update(S, n, z, w, w_old, x_acc, st), "update");
  std::swap(v_old, v);
  std::swap(w_old, w);
  std::swap(z, zn);
}

// Captures two iterations (one full rotation of the vector roles) as a CUDA graph on the
// handle's capture stream; the graph is later launched on the handle's stream.
void capture_iterations(mcs_handle* h, double* x_acc) {
  double *v_old = h->kv[0], *v = h->kv[1], *z = h->kv[2], *zn = h->kv[3];
  double *w_old = h->kv[4], *w = h->kv[5], *Kz = h->kv[6];
  cudaStream_t cs = h->cap_stream;
  cuda_check(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  cudaGraph_t g = nullptr;
  g_capturing = true;
  try {
    minres_iteration(h, cs, v_old, v, z, zn, w_old, w, Kz, x_acc);
    minres_iteration(h, cs, v_old, v, z, zn, w_old, w, Kz, x_acc);
  } catch (...) {
    g_capturing = false;
    cudaStreamEndCapture(cs, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  g_capturing = false;
  cuda_check(cudaStreamEndCapture(cs, &g), "cudaStreamEndCapture");
  size_t nn = 0;
  cudaError_t ce = cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (ce == cudaSuccess && nn) ce = cudaGraphGetNodes(g, nodes.data(), &nn);
  uint64_t nk = 0;
  for (size_t i = 0; ce == cudaSuccess && i < nn; ++i) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
  }
  if (ce != cudaSuccess) {
    cudaGraphDestroy(g);
    cuda_check(ce, "cudaGraphGetNodes");
  }
  h->graph_kernels = nk;
  cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
  cudaGraphDestroy(g);
  cuda_check(e, "cudaGraphInstantiate");
}

// One MinRes cycle on K d = rhs from d = 0, accumulating d into x_acc.
// g_first: preconditioned norm of the first cycle's residual (< 0 before the first cycle).
// Early end of a cycle on the error bound (etol > 0): with x_start the iterate at the cycle's start, the
// cycle stops at a check once bound * (|eta| / res0) * rho <= etol, rho = max(|d_u|/|x_u|, |d_p|/|x_p|)
// for the correction d = x_acc - x_start so far (bound = the safety factor times the lag).
struct CycleBound {
  const double* x_start = nullptr;   // nullptr: no early end
  double bound = 0, etol = 0;
};

void minres_cycle(mcs_handle* h, const double* rhs, double* x_acc, double rtol, double floor_rtol, int maxit,
                  double g_first, const CycleBound& cb = CycleBound()) {
  const int64_t n = h->L.ndof;
  cudaStream_t st = h->stream;
  double *v_old = h->kv[0], *v = h->kv[1], *z = h->kv[2], *zn = h->kv[3];
  double *w_old = h->kv[4], *w = h->kv[5], *Kz = h->kv[6];
  MinresScalars* S = h->S;
  MinresScalars init{};
  init.rtol = rtol;
  init.floor_rtol = floor_rtol;
  init.g_first = g_first;
  init.maxit = maxit;
  cuda_check(cudaMemcpyAsync(S, &init, sizeof(MinresScalars), cudaMemcpyHostToDevice, st), "init S");
  cuda_check(cudaMemcpyAsync(v, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
  cuda_check(cudaMemsetAsync(v_old, 0, sizeof(double) * n, st), "memset");
  cuda_check(cudaMemsetAsync(w, 0, sizeof(double) * n, st), "memset");
  cuda_check(cudaMemsetAsync(w_old, 0, sizeof(double) * n, st), "memset");
  precond_any(h, v, z, nullptr);
  if (!h->outflow)
    cuda_check(launch_mean_zero(h->dm, h->L, h->sz.n_p, z, h->scratch, h->total_adet, nullptr, st), "mean");
  cuda_check(launch_dot(z, v, n, h->scratch, &S->dot1, nullptr, st), "dot");
  cuda_check(launch_minres_init(S, st), "init");
  const int* stop = &S->stop;
  const bool graphs = h->use_graphs && !h->prof;
  if (graphs && !h->gexec) capture_iterations(h, x_acc);
  // iterations between reads of the convergence state; 4 in a cycle that may end on the error bound,
  // whose check is cheap against the iterations a coarser check would run past it
  const int check_every = cb.x_start ? 4 : 8;
  const int64_t nu_blk = h->L.off_p, np_blk = n - h->L.off_p;
  double* res = h->scratch + 3010;   // [|d_u|^2, |d_p|^2, |x_u|^2, |x_p|^2] of the early-end check
  while (true) {
    cuda_check(cudaMemcpyAsync(h->S_host, S, sizeof(MinresScalars), cudaMemcpyDeviceToHost, st), "read S");
    cuda_check(cudaStreamSynchronize(st), "sync");
    if (h->S_host->stop) break;
    if (cb.x_start && h->S_host->it > 0 && h->S_host->res0 > 0) {
      cuda_check(launch_diff_sq(x_acc, cb.x_start, nu_blk, h->scratch, res, st), "diff");
      cuda_check(launch_diff_sq(x_acc + nu_blk, cb.x_start + nu_blk, np_blk, h->scratch, res + 1, st), "diff");
      cuda_check(launch_dot(x_acc, x_acc, nu_blk, h->scratch, res + 2, nullptr, st), "dot");
      cuda_check(launch_dot(x_acc + nu_blk, x_acc + nu_blk, np_blk, h->scratch, res + 3, nullptr, st), "dot");
      double hv[4];
      cuda_check(cudaMemcpyAsync(hv, res, sizeof(hv), cudaMemcpyDeviceToHost, st), "copy");
      cuda_check(cudaStreamSynchronize(st), "sync");
      const double rho = std::min(1.0, std::max(hv[2] > 0 ? std::sqrt(hv[0] / hv[2]) : 0.0,
                                                hv[3] > 0 ? std::sqrt(hv[1] / hv[3]) : 0.0));
      if (cb.bound * (std::fabs(h->S_host->eta) / h->S_host->res0) * rho <= cb.etol) break;
    }
    if (graphs) {
      for (int q = 0; q < check_every / 2; ++q) {
        cuda_check(cudaGraphLaunch(h->gexec, st), "cudaGraphLaunch");
        note_launches(h->graph_kernels);
      }
    } else {
      for (int q = 0; q < check_every; ++q) minres_iteration(h, st, v_old, v, z, zn, w_old, w, Kz, x_acc);
    }
  }
}

}  // namespace

int mcs_solve(mcs_handle* h, const double* F, double* x, mcs_solve_info* info) {
  return guarded([&]() -> int {
    if (!h || !F || !x) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    ProfScope ps(h->prof.get());
    if (!h->condensed) throw McsError(MCS_ERR_INVALID_ARG, "mcs_condense has not been called");
    const int64_t n = h->L.ndof;
    cudaStream_t st = h->stream;
    double* r = h->kv[7];
    double* xi = h->kv[10];  // the iterate (fixed address for the captured iterations)
    cuda_check(cudaMemcpyAsync(xi, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy x");
    const bool mixed = h->opt.precision == MCS_MIXED;
    const double etol = h->opt.etol;
    // FP64 form: cycles to rtol, restarted from the recomputed residual (at most 3).  Mixed
    // form, and both forms with an error target: iterative refinement, each cycle asked for at
    // least inner_rtol reduction.
    const int max_cycles = (mixed || etol > 0) ? std::max(2, h->opt.max_refine + 1)
                                               : std::min(3, std::max(2, h->opt.max_refine + 1));
    const double floor_rtol = (mixed || etol > 0) ? h->opt.inner_rtol : 0.0;
    // an error target needs the exact residual: with nu << 1 the velocity part of F - K x is a small
    // difference of O(1) terms whose FP64 rounding floors the attainable velocity error
    const bool dd = h->opt.residual_dd == 1 ||
                    (h->opt.residual_dd == -1 && (h->opt.rtol < 1e-10 || h->opt.etol > 0));
    auto residual = [&](const double* xv) {  // r = F - K xv
      if (dd) {
        cuda_check(launch_residual_dd(h->es, h->dt, h->dm, h->L, h->K, F, xv, h->ydd, r, st), "residual");
      } else {
        cuda_check(launch_apply_K(h->es, h->dt, h->dm, h->L, h->K, xv, r, nullptr, st), "apply");
        cuda_check(launch_axpby(n, 1.0, F, -1.0, r, st), "axpby");
      }
    };
    int total_it = 0, cycles = 0, status = MCS_ERR_NOT_CONVERGED;
    double g_first = -1.0, g_now = 0.0;
    // Error target (etol > 0): cycle c's correction d_c estimates the error entering it (relative size
    // rho_c, the larger of the u and p blocks).  The error leaving it is taken as lag * R_c * rho_c, R_c
    // the cycle's achieved residual reduction and lag = max(1, (rho_c / rho_{c-1}) / R_{c-1}) how much
    // less the previous cycle reduced the error than the residual (from the third correction on), and
    // bounded by est_c = kSafety lag R_c rho_c.  The first cycle runs to rtol (mixed: inner_rtol); every
    // later one runs until its own correction so far shows the bound met (checked every 4 iterations),
    // or to the least reduction r_min.
    constexpr double kSafety = 3.0;
    const double r_min = mixed ? h->opt.inner_rtol : 1e-12;   // least reduction asked of one cycle
    double est = std::numeric_limits<double>::infinity();
    double rho_prev = -1.0, red_prev = -1.0, lag_now = 1.0;
    int ncorr = 0;   // corrections measured so far
    double r_next = mixed ? std::max(h->opt.rtol, h->opt.inner_rtol) : h->opt.rtol;
    double* xprev = h->kv[11];
    double* res = h->scratch + 3002;   // [|d_u|^2, |d_p|^2, |x_u|^2, |x_p|^2]
    const int64_t nu_blk = h->L.off_p, np_blk = n - h->L.off_p;
    while (cycles < max_cycles) {
      residual(xi);
      if (etol > 0) cuda_check(cudaMemcpyAsync(xprev, xi, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
      // the residual test may end the solve only once the error bound meets etol
      const bool err_ok = etol > 0 && est <= etol;
      const double rtol_now = (etol > 0 && !err_ok) ? 0.0 : h->opt.rtol;
      // after the first correction a cycle runs to the least reduction and ends early once its own
      // correction shows the error bound met (the check every 4 iterations)
      const bool adaptive = etol > 0 && !err_ok && ncorr >= 1;
      const double floor_now = etol > 0 ? ((err_ok || adaptive) ? r_min : r_next) : floor_rtol;
      CycleBound cbound;
      if (adaptive) {
        cbound.x_start = xprev;
        cbound.bound = kSafety * lag_now;
        cbound.etol = etol;
      }
      minres_cycle(h, r, xi, rtol_now, floor_now, std::max(1, h->opt.maxit - total_it), g_first, cbound);
      const MinresScalars& Sh = *h->S_host;
      g_first = Sh.g_first;
      g_now = Sh.res0;
      total_it += Sh.it;
      ++cycles;
      if (Sh.status == MCS_ERR_BREAKDOWN) {
        status = MCS_ERR_BREAKDOWN;
        break;
      }
      if (Sh.it == 0 && (g_now <= h->opt.rtol * g_first || g_now == 0.0)) {
        status = MCS_OK;  // the recomputed residual meets the tolerance
        break;
      }
      if (etol > 0) {
        const double achieved = Sh.res0 > 0 ? std::fabs(Sh.eta) / Sh.res0 : 0.0;
        // d = xi - xprev, the cycle's correction; block norms of d and of the iterate
        if (!h->outflow)
          cuda_check(launch_mean_zero(h->dm, h->L, h->sz.n_p, xi, h->scratch, h->total_adet, nullptr, st), "mean");
        cuda_check(launch_axpby(n, 1.0, xi, -1.0, xprev, st), "axpby");
        cuda_check(launch_dot(xprev, xprev, nu_blk, h->scratch, res, nullptr, st), "dot");
        cuda_check(launch_dot(xprev + nu_blk, xprev + nu_blk, np_blk, h->scratch, res + 1, nullptr, st), "dot");
        cuda_check(launch_dot(xi, xi, nu_blk, h->scratch, res + 2, nullptr, st), "dot");
        cuda_check(launch_dot(xi + nu_blk, xi + nu_blk, np_blk, h->scratch, res + 3, nullptr, st), "dot");
        double hv[4];
        cuda_check(cudaMemcpyAsync(hv, res, sizeof(hv), cudaMemcpyDeviceToHost, st), "copy");
        cuda_check(cudaStreamSynchronize(st), "sync");
        const double ru = hv[2] > 0 ? std::sqrt(hv[0] / hv[2]) : 0.0;
        const double rp = hv[3] > 0 ? std::sqrt(hv[1] / hv[3]) : 0.0;
        const double rho = std::min(1.0, std::max(ru, rp));
        if (ncorr >= 2 && rho_prev > 0 && red_prev > 0) lag_now = std::max(1.0, (rho / rho_prev) / red_prev);
        const double e_now = lag_now * achieved * rho;   // nominal error leaving this cycle
        est = kSafety * e_now;
        r_next = e_now > 0 ? std::min(0.1, std::max(r_min, etol / (kSafety * lag_now * e_now))) : 0.1;
        rho_prev = rho;
        red_prev = achieved;
        ++ncorr;
      }
      if (total_it >= h->opt.maxit) break;
    }
    if (!h->outflow)
      cuda_check(launch_mean_zero(h->dm, h->L, h->sz.n_p, xi, h->scratch, h->total_adet, nullptr, st), "mean");
    cuda_check(cudaMemcpyAsync(x, xi, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy x");
    if (info) {
      residual(x);
      double* res = h->scratch + 3000;
      cuda_check(launch_dot(r, r, n, h->scratch, res, nullptr, st), "dot");
      cuda_check(launch_dot(F, F, n, h->scratch, res + 1, nullptr, st), "dot");
      double hv[2];
      cuda_check(cudaMemcpyAsync(hv, res, sizeof(hv), cudaMemcpyDeviceToHost, st), "copy");
      cuda_check(cudaStreamSynchronize(st), "sync");
      info->iterations = total_it;
      info->refinements = cycles;
      info->status = status;
      info->rel_res_true = hv[1] > 0 ? std::sqrt(hv[0] / hv[1]) : 0.0;
      info->rel_res_precond = g_first > 0 ? g_now / g_first : 0.0;
      info->err_est = etol > 0 ? est : 0.0;
    }
    {
      // a bounded wait inside the preconditioner that gave up marks the solve as timed out
      int* errp = h->opt.precision == MCS_MIXED ? h->pf.err : h->pd.err;
      int herr = 0;
      cuda_check(cudaMemcpyAsync(&herr, errp, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
      cuda_check(cudaStreamSynchronize(st), "sync");
      if (herr) {
        cuda_check(cudaMemsetAsync(errp, 0, sizeof(int), st), "memset");
        status = MCS_ERR_TIMEOUT;
        if (info) info->status = status;
      }
    }
    if (status != MCS_OK)
      g_err = status == MCS_ERR_BREAKDOWN ? "Krylov breakdown"
              : status == MCS_ERR_TIMEOUT ? "an asynchronous copy in the preconditioner did not complete"
                                          : "not converged";
    return status;
  });
}

int mcs_solve_host(mcs_handle* h, const double* F_host, double* x_host, mcs_solve_info* info) {
  return guarded([&]() -> int {
    if (!h || !F_host || !x_host) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    const int64_t n = h->L.ndof;
    double* F = h->kv[8];
    double* x = h->kv[9];
    cuda_check(cudaMemcpyAsync(F, F_host, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream), "h2d");
    cuda_check(cudaMemcpyAsync(x, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream), "h2d");
    int rc = mcs_solve(h, F, x, info);
    cuda_check(cudaMemcpyAsync(x_host, x, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream), "d2h");
    cuda_check(cudaStreamSynchronize(h->stream), "sync");
    return rc;
  });
}

int mcs_profile(mcs_handle* h, int enable) {
  return guarded([&]() -> int {
    if (!h) throw McsError(MCS_ERR_INVALID_ARG, "NULL handle");
    if (enable) {
      if (!h->prof) h->prof.reset(new Profiler());
      h->prof->reset();
    } else {
      h->prof.reset();
    }
    return MCS_OK;
  });
}

int mcs_recover_stress(mcs_handle* h, const double* x, int nq, const double* xhat_host, double* sigma,
                       double* omega) {
  return guarded([&]() -> int {
    if (!h || !x || !xhat_host || !sigma || nq < 1) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument or nq < 1");
    if (h->sz.lowest && omega)
      throw McsError(MCS_ERR_UNSUPPORTED, "k = 1: the rotation is a global unknown (flux dofs in x); pass omega = NULL");
    const int d = h->d, nk = h->sz.nk;
    std::vector<double> psi((size_t)nq * nk);
    for (int q = 0; q < nq; ++q) dubiner_eval(d, h->k, xhat_host + (size_t)q * d, psi.data() + (size_t)q * nk, nullptr);
    cudaStream_t st = h->stream;
    double* psi_dev = nullptr;
    cuda_check(cudaMallocAsync((void**)&psi_dev, sizeof(double) * psi.size(), st), "cudaMallocAsync");
    cudaError_t e = cudaMemcpyAsync(psi_dev, psi.data(), sizeof(double) * psi.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = launch_recover(h->es, h->dt, h->dm, h->L, h->nu, x, nq, psi_dev, sigma, omega, h->cond_scratch,
                         h->cond_scratch_doubles, st);
    cudaFreeAsync(psi_dev, st);
    cuda_check(e, "stress recovery");
    return MCS_OK;
  });
}

int mcs_launch_count(uint64_t* count) {
  return guarded([&]() -> int {
    if (!count) throw McsError(MCS_ERR_INVALID_ARG, "count is NULL");
    *count = launch_count();
    return MCS_OK;
  });
}

int mcs_profile_read(mcs_handle* h, mcs_kernel_stat* out, int max_n) {
  return guarded([&]() -> int {
    if (!h || !out || max_n < 0) throw McsError(MCS_ERR_INVALID_ARG, "NULL argument");
    if (!h->prof) return 0;
    h->prof->collect();
    static const char* names[PROF_NCLASS] = {"condense", "facet_blocks", "apply_K", "facet_gs_step",
                                             "facet_residual", "elem_prologue", "elem_epilogue", "gmg_vcycle",
                                             "facet_push"};
    int n = 0;
    for (int c = 0; c < PROF_NCLASS && n < max_n; ++c) {
      mcs_kernel_stat& o = out[n++];
      std::memset(&o, 0, sizeof(o));
      std::strncpy(o.name, names[c], sizeof(o.name) - 1);
      o.launches = h->prof->launches[c];
      o.total_ms = h->prof->ms[c];
      o.bytes = h->prof->bytes[c];
      o.flops = h->prof->flops[c];
    }
    return n;
  });
}

int mcs_destroy(mcs_handle* h) {
  return guarded([&]() -> int {
    if (!h) return MCS_OK;
    cudaStreamSynchronize(h->stream);
    delete h;
    return MCS_OK;
  });
}

}  // extern "C"
