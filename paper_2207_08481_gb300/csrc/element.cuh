// Element-level static condensation of the MCS method (host/device code).
//
// For one simplex T with vertex coordinates X (ascending global ids) this forms
//
//   A_T = A^div_T - B_sigma,T M_T^{-1} B_sigma,T^T          (arXiv 2207.08481 Sec. 4.2)
//
// where M_T is the local saddle-point block over Sigma_h(T) x W_h(T) of
// eq. (bigfemSPmat).  Sigma_h(T) is represented in the raw trace-free basis
// J^{-T}(psi_i E_s)J^T; its nt conditions (eq. fes_Sigma) and the rotation
// constraints (B_omega sigma = 0) are eliminated together by Lagrange
// multipliers:  with M_raw = (|det J|/nu) (I (x) g), g_st = tr(E_s^T G^{-1} E_t G),
// G = J^T J, and all constraints C,
//
//   -(M^{-1})_{sigma sigma} = M_raw^{-1} - M_raw^{-1} C^T (C M_raw^{-1} C^T)^{-1} C M_raw^{-1},
//
// so A_T = A^div + Bt Bt^T - Z^T Z with Bt = B_raw (I (x) L) sqrt(nu/|det J|),
// Ct = C (I (x) L), g^{-1} = L L^T, Sc = Ct Ct^T = Lc Lc^T, Z = Lc^{-1} Ct Bt^T.
//
// The geometric dependence of B_sigma (raw basis, u by the |det J| Piola map):
//   B_u[i,j]  = B0[i,j] - sum_{f,a} w_{f,a} Rf[f,a][i,j],  w_{f,a} = (G^{-1} n_f)_a / (n_f^T G^{-1} n_f)
//   B_uh[i,j] = |det J| Bh[i,j]
//   B_omega   = |det J| (h (x) I_{P^{k-1}}),  h_rs = K_r : (J^{-T} E_s J^T)
//   A^div     = nu / (d |det J|) Adiv_ref.
//
// All routines are written for `nl` cooperating lanes (a warp on the device, a
// single lane on the host); `sync()` separates phases.
#pragma once
#include <cmath>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace mcs {

struct ElemSizes {
  int d, k, nk, nF, nFm1, n_u, n_A, n_hat, nhF, n_p, n_s0, n_raw, n_con, n_w, n_wskew, n_cc;
  int n_bub, n_c, mF;
  int ntF, lowest;   // tangential Vhat_h dofs per facet; 1 for the lowest-order variant (k = 1)
  int lo_stab;       // k = 1: coefficient of (div omega, div eta)_T is nu (0) or nu h_T^2 (1)
};

// Local index i of A_T is the rotation flux dof of a facet (lowest-order variant only).
__host__ __device__ inline bool is_rot_dof(const ElemSizes& s, int i) {
  return s.lowest && i >= s.n_u && (i - s.n_u) % s.nhF == s.ntF;
}

struct ElemTables {
  const double* B0;    // [n_u][n_raw]
  const double* Rf;    // [d+1][d][nF][n_raw]
  const double* Bh;    // [n_hat][n_raw]
  const double* Ccon;  // [n_con][n_raw]
  const double* Adiv;  // [n_u][n_u]
  const double* nhat;  // [d+1][d]
  const double* Wmom;  // k = 1: [d+1][d][nk]
};

// workspace layout (doubles), per element
struct ElemWork {
  double* geo;   // 128 scalars: L (8x8), h (3x8), w (4x3), adet
  double* Bt;    // [n_A][n_raw]
  double* Ct;    // [n_cc][n_raw]
  double* V;     // [n_cc][n_A]
  double* Sc;    // [n_cc][n_cc]
  double* A;     // [n_A][n_A]
};

// Row stride of Bt and Ct in the workspace: odd, so that threads reading different rows of
// 8-byte words hit different shared-memory banks.
__host__ __device__ inline int raw_stride(const ElemSizes& s) { return s.n_raw | 1; }

__host__ __device__ inline int elem_work_doubles(const ElemSizes& s) {
  return 128 + s.n_A * raw_stride(s) + s.n_cc * raw_stride(s) + s.n_cc * s.n_A + s.n_cc * s.n_cc + s.n_A * s.n_A;
}

__host__ __device__ inline ElemWork elem_work_carve(const ElemSizes& s, double* base) {
  ElemWork w;
  w.geo = base;
  w.Bt = base + 128;
  w.Ct = w.Bt + s.n_A * raw_stride(s);
  w.V = w.Ct + s.n_cc * raw_stride(s);
  w.Sc = w.V + s.n_cc * s.n_A;
  w.A = w.Sc + s.n_cc * s.n_cc;
  return w;
}

// trace-free unit E_s entry (a, b) (same order as the host tables)
__host__ __device__ inline double tf_unit(int d, int s, int a, int b) {
  int noff = d * (d - 1);
  if (s < noff) {
    int cnt = 0;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        if (i != j) {
          if (cnt == s) return (a == i && b == j) ? 1.0 : 0.0;
          ++cnt;
        }
    return 0.0;
  }
  int t = s - noff;
  if (a != b) return 0.0;
  if (a == t) return 1.0;
  if (a == t + 1) return -1.0;
  return 0.0;
}

// skew unit K_r = e_b e_a^T - e_a e_b^T for the r-th pair a < b: entry (i, j)
__host__ __device__ inline double skew_unit(int d, int r, int i, int j) {
  int cnt = 0;
  for (int a = 0; a < d; ++a)
    for (int b = a + 1; b < d; ++b) {
      if (cnt == r) {
        if (i == b && j == a) return 1.0;
        if (i == a && j == b) return -1.0;
        return 0.0;
      }
      ++cnt;
    }
  return 0.0;
}

__host__ __device__ inline void small_inverse(int n, double* A, double* Inv) {
  // Gauss-Jordan with partial pivoting on an n x n (n <= 8) matrix; A is destroyed.
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Inv[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        double t = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = t;
        t = Inv[c * n + j]; Inv[c * n + j] = Inv[p * n + j]; Inv[p * n + j] = t;
      }
    double iv = 1.0 / A[c * n + c];
    for (int j = 0; j < n; ++j) { A[c * n + j] *= iv; Inv[c * n + j] *= iv; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      for (int j = 0; j < n; ++j) { A[r * n + j] -= f * A[c * n + j]; Inv[r * n + j] -= f * Inv[c * n + j]; }
    }
  }
}

// Nonzeros of the trace-free unit E_s (same order as tf_unit): rows a[], columns b[], values c[];
// returns their number (1 for an off-diagonal unit e_i e_j^T, 2 for e_t e_t^T - e_{t+1} e_{t+1}^T).
__host__ __device__ inline int tf_nonzeros(int d, int s, int* a, int* b, double* c) {
  const int noff = d * (d - 1);
  if (s < noff) {
    const int i = s / (d - 1), jj = s - i * (d - 1);
    a[0] = i;
    b[0] = jj < i ? jj : jj + 1;
    c[0] = 1.0;
    return 1;
  }
  const int t = s - noff;
  a[0] = b[0] = t;
  c[0] = 1.0;
  a[1] = b[1] = t + 1;
  c[1] = -1.0;
  return 2;
}

// The pair (a, b), a < b, of the r-th skew unit K_r = e_b e_a^T - e_a e_b^T (order (0,1), (0,2), (1,2)).
__host__ __device__ inline void skew_pair(int d, int r, int& a, int& b) {
  int cnt = 0;
  for (int i = 0; i < d; ++i)
    for (int j = i + 1; j < d; ++j) {
      if (cnt == r) { a = i; b = j; }
      ++cnt;
    }
}

// Geometric factors of one element, computed by nl cooperating lanes.
// geo: [0..63] L (n_s0 x n_s0, lower, g^{-1} = L L^T), [64..87] h (n_wskew x n_s0),
//      [88..99] w (d+1 x d), [100] |det J|, [101] det J
// tmp: 164 doubles of scratch (J, J^{-1}, G, G^{-1}, g, g^{-1}).
// With g_st = tr(E_s^T G^{-1} E_t G) written out over the nonzeros of the units and
// h_rs = K_r : (J^{-T} E_s J^T) = sum over E_s's nonzeros (a, b, c) of c (Ji[a][q] J[p][b] - Ji[a][p] J[q][b])
// for the pair (p, q) of K_r (Ji[a][i] = (J^{-1})_{ai}, J[j][b] = J_{jb}).
template <class Sync>
__host__ __device__ inline void elem_geometry(const ElemSizes& s, const double* X, const double* nhat, double* geo,
                                              double* tmp, int lane, int nl, Sync sync) {
  const int d = s.d, ns0 = s.n_s0;
  double* J = tmp;
  double* Ji = tmp + 9;
  double* G = tmp + 18;
  double* Gi = tmp + 27;
  double* gm = tmp + 36;
  double* ginv = tmp + 100;
  if (lane == 0) {
    for (int a = 0; a < d; ++a)
      for (int i = 0; i < d; ++i) J[a * d + i] = X[(i + 1) * d + a] - X[a];  // column i = x_{i+1} - x_0
    double det;
    if (d == 2) {
      det = J[0] * J[3] - J[1] * J[2];
      Ji[0] = J[3] / det; Ji[1] = -J[1] / det; Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
    } else {
      det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
      Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
      Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
      Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
      Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
      Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
      Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
      Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
      Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
      Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    }
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double g = 0, gi = 0;
        for (int c = 0; c < d; ++c) {
          g += J[c * d + a] * J[c * d + b];
          gi += Ji[a * d + c] * Ji[b * d + c];
        }
        G[a * d + b] = g;
        Gi[a * d + b] = gi;
      }
    geo[100] = fabs(det);
    geo[101] = det;
  }
  sync();
  // g (n_s0^2 entries), h (n_wskew * n_s0) and the facet weights w (d + 1) over the lanes
  const int ng = ns0 * ns0, nh = s.n_wskew * ns0;
  for (int q = lane; q < ng + nh + d + 1; q += nl) {
    if (q < ng) {
      const int s1 = q / ns0, t = q - s1 * ns0;
      int a1[2], b1[2], a2[2], b2[2];
      double c1[2], c2[2];
      const int n1 = tf_nonzeros(d, s1, a1, b1, c1), n2 = tf_nonzeros(d, t, a2, b2, c2);
      double v = 0;
      for (int u = 0; u < n1; ++u)
        for (int w2 = 0; w2 < n2; ++w2) v += c1[u] * c2[w2] * Gi[a1[u] * d + a2[w2]] * G[b2[w2] * d + b1[u]];
      gm[q] = v;
    } else if (q < ng + nh) {
      const int r = (q - ng) / ns0, s1 = (q - ng) - r * ns0;
      int p, qq;
      skew_pair(d, r, p, qq);
      int a1[2], b1[2];
      double c1[2];
      const int n1 = tf_nonzeros(d, s1, a1, b1, c1);
      double v = 0;
      for (int u = 0; u < n1; ++u)
        v += c1[u] * (Ji[a1[u] * d + qq] * J[p * d + b1[u]] - Ji[a1[u] * d + p] * J[qq * d + b1[u]]);
      geo[64 + r * ns0 + s1] = v;
    } else {
      const int f = q - ng - nh;
      double gn[3] = {0, 0, 0}, nn = 0;
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) gn[a] += Gi[a * d + b] * nhat[f * d + b];
      for (int a = 0; a < d; ++a) nn += gn[a] * nhat[f * d + a];
      for (int a = 0; a < d; ++a) geo[88 + f * d + a] = gn[a] / nn;
    }
  }
  sync();
  if (lane == 0) {
    small_inverse(ns0, gm, ginv);
    // symmetrise and Cholesky g^{-1} = L L^T
    double* L = geo;
    for (int i = 0; i < 64; ++i) L[i] = 0.0;
    for (int j = 0; j < ns0; ++j) {
      double sdiag = ginv[j * ns0 + j];
      for (int p = 0; p < j; ++p) sdiag -= L[j * ns0 + p] * L[j * ns0 + p];
      const double ljj = sqrt(sdiag);
      L[j * ns0 + j] = ljj;
      for (int i = j + 1; i < ns0; ++i) {
        double v = 0.5 * (ginv[i * ns0 + j] + ginv[j * ns0 + i]);
        for (int p = 0; p < j; ++p) v -= L[i * ns0 + p] * L[j * ns0 + p];
        L[i * ns0 + j] = v / ljj;
      }
    }
  }
  sync();
}

// Row i and column j (j <= i) of packed lower-triangle position q = i(i+1)/2 + j.
__host__ __device__ inline void packed_ij(int q, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > q) --r;
  while ((r + 1) * (r + 2) / 2 <= q) ++r;
  i = r;
  j = q - r * (r + 1) / 2;
}

// Lane-parallel Cholesky of the n x n SPD matrix A (row-major, lower triangle used), applied at
// the same time to the m right-hand-side columns of V (row-major [n][m]):  on return the lower
// triangle of A holds the factor Lc (A = Lc Lc^T) and V holds Lc^{-1} V.  Right-looking
// elimination on the augmented matrix [A | V] without pivoting: for pivot j every entry (i, c),
// j < c <= i, of A and every V[i][.], i > j, takes its update from column j and row j, which no
// lane writes during that step, so one barrier per pivot suffices.  The scaling by the square
// roots of the pivots follows in two passes.
template <class Sync>
__host__ __device__ inline void chol_solve_inplace(int n, double* A, int m, double* V, int lane, int nl, Sync sync) {
  for (int j = 0; j + 1 < n; ++j) {
    const double inv = 1.0 / A[j * n + j];
    const int r = n - j - 1;   // rows below the pivot
    const int wa = r, wt = r + m;
    for (int t = lane; t < r * wt; t += nl) {
      const int i = j + 1 + t / wt, c = t - (t / wt) * wt;
      const double f = A[i * n + j] * inv;
      if (c < wa) {
        const int cc = j + 1 + c;
        if (cc <= i) A[i * n + cc] -= f * A[cc * n + j];
      } else {
        const int cv = c - wa;
        V[i * m + cv] -= f * V[j * m + cv];
      }
    }
    sync();
  }
  // A = L D L^T with unit L (stored as L D); Lc = L D^{1/2}, Lc^{-1} V = D^{-1/2} (L^{-1} V)
  for (int t = lane; t < n * (n + m); t += nl) {
    const int i = t / (n + m), c = t - i * (n + m);
    const double di = A[i * n + i];
    if (c < n) {
      if (c < i) A[i * n + c] /= sqrt(A[c * n + c]);
    } else {
      V[i * m + (c - n)] /= sqrt(di);
    }
  }
  sync();
  for (int i = lane; i < n; i += nl) A[i * n + i] = sqrt(A[i * n + i]);
  sync();
}

// Lowest-order variant (Sec. 7): raw row of the rotation flux function phi_f = (x - x_f) / (d |T|)
// of local facet f, int (psi_i J^{-T} E_s J^T) : kappa(phi_f).  With x - x_f = J (xhat - xhat_f) and
// kappa(v) = (v_3 K_0 - v_2 K_1 + v_1 K_2) / 2 it is
//   sum_c Wmom[f][c][i] (J_2c h_0s - J_1c h_1s + J_0c h_2s)      (|det J| / (d |T|) = 2, d = 3).
__host__ __device__ inline void rotation_row(const ElemSizes& s, const ElemTables& t, const double* X, const double* h,
                                      int f, double* row) {
  const int ns0 = s.n_s0;
  double Jc[9];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) Jc[a * 3 + c] = X[(c + 1) * 3 + a] - X[a];
  for (int e = 0; e < ns0; ++e) {
    double kc[3];
    for (int c = 0; c < 3; ++c) kc[c] = Jc[6 + c] * h[e] - Jc[3 + c] * h[ns0 + e] + Jc[c] * h[2 * ns0 + e];
    for (int i = 0; i < s.nk; ++i) {
      const double* wm = t.Wmom + (f * 3) * s.nk + i;
      row[i * ns0 + e] = wm[0] * kc[0] + wm[s.nk] * kc[1] + wm[2 * s.nk] * kc[2];
    }
  }
}

// Full condensation of one element: A_T (n_A x n_A, row-major) with the orientation
// signs of the facet-BDM dofs (and, for k = 1, of the rotation flux dofs) applied.
// Lowest-order variant (k = 1, Sec. 7): the rotation is not eliminated; its flux dofs are rows
// of Bt (coupling through kappa(omega)), the constraints are the nt conditions alone, and
// A_T gains nu (div omega, div eta)_T on the rotation rows.
// LO is the compile-time form of s.lowest (condense_element below dispatches at run time), so that
// the k >= 2 instantiation carries none of the lowest-order code.
template <bool LO, class Sync>
__host__ __device__ inline void condense_element_t(const ElemSizes& s, const ElemTables& t, const double* X,
                                                   const int* sgn, double nu, ElemWork w, int lane, int nl,
                                                   Sync sync) {
  const int nraw = s.n_raw, ns0 = s.n_s0, nA = s.n_A, nu_ = s.n_u, ncc = s.n_cc, d = s.d, rs = raw_stride(s);
  elem_geometry(s, X, t.nhat, w.geo, w.A, lane, nl, sync);   // w.A is free until the product pass
  if (lane == 0) w.geo[102] = nu;
  const double* L = w.geo;
  const double* h = w.geo + 64;
  const double* wf = w.geo + 88;
  const double adet = w.geo[100];
  const double cB = sqrt(nu / adet);
  // ---- rows of Bt and Ct, one work item per (row, polynomial block i): the n_s0 raw entries of
  // block i are formed and transformed by L, times cB for Bt (the whitening (I (x) L)) ----
  const int nkb = s.nk, nrows = nA + ncc;
  for (int q = lane; q < nrows * nkb; q += nl) {
    const int r = q / nkb, i = q - r * nkb;
    double tmp[8];
    double scale = 1.0;
    bool zero = false;
    if (r < nA) {
      scale = cB;
      if (r < nu_) {
        for (int p = 0; p < ns0; ++p) tmp[p] = t.B0[r * nraw + i * ns0 + p];
        if (r < (d + 1) * s.nF) {
          const int f = r / s.nF, jF = r % s.nF;
          for (int a2 = 0; a2 < d; ++a2) {
            const double wa = wf[f * d + a2];
            const double* R = t.Rf + ((f * d + a2) * s.nF + jF) * nraw + i * ns0;
            for (int p = 0; p < ns0; ++p) tmp[p] -= wa * R[p];
          }
        }
      } else if (LO && is_rot_dof(s, r)) {
        continue;   // lowest-order rotation rows: filled below
      } else {
        const double* Bh = t.Bh + (r - nu_) * nraw + i * ns0;
        for (int p = 0; p < ns0; ++p) tmp[p] = adet * Bh[p];
      }
    } else if (r - nA < s.n_con) {
      const double* C = t.Ccon + (r - nA) * nraw + i * ns0;
      for (int p = 0; p < ns0; ++p) tmp[p] = C[p];
    } else {
      const int rr = r - nA - s.n_con, kr = rr / s.n_p, ip = rr - kr * s.n_p;
      zero = i != ip;
      for (int p = 0; p < ns0; ++p) tmp[p] = zero ? 0.0 : h[kr * ns0 + p];
    }
    double* row = (r < nA ? w.Bt + r * rs : w.Ct + (r - nA) * rs) + i * ns0;
    for (int q2 = 0; q2 < ns0; ++q2) {
      double v = 0;
      if (!zero)
        for (int p = q2; p < ns0; ++p) v += tmp[p] * L[p * ns0 + q2];
      row[q2] = scale * v;
    }
  }
  if (LO)
    for (int f = lane; f <= d; f += nl) {
      double* row = w.Bt + (nu_ + f * s.nhF + s.ntF) * rs;
      rotation_row(s, t, X, h, f, row);
      for (int i = 0; i < s.nk; ++i) {
        double tmp[8];
        for (int q = 0; q < ns0; ++q) tmp[q] = row[i * ns0 + q];
        for (int q = 0; q < ns0; ++q) {
          double v = 0;
          for (int p = q; p < ns0; ++p) v += tmp[p] * L[p * ns0 + q];
          row[i * ns0 + q] = cB * v;
        }
      }
    }
  sync();
  // ---- one pass over A = Adiv + Bt Bt^T (lower), V = Ct Bt^T, Sc = Ct Ct^T (lower) ----
  const double cdiv = nu / (d * adet);
  // k = 1 (d = 3): div phi_f = 1/|T|, |T| = |det J| / 6; coefficient nu or nu h_T^2 (h_T: longest edge)
  double cstab = nu * 6.0 / adet;
  if (LO && s.lo_stab) {
    double h2 = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        double e2 = 0.0;
        for (int c = 0; c < 3; ++c) e2 += (X[b * 3 + c] - X[a * 3 + c]) * (X[b * 3 + c] - X[a * 3 + c]);
        h2 = e2 > h2 ? e2 : h2;
      }
    cstab *= h2;
  }
  const int PA = nA * (nA + 1) / 2, PV = ncc * nA, PS = ncc * (ncc + 1) / 2;
  for (int q = lane; q < PA + PV + PS; q += nl) {
    const double *a, *b;
    double* out;
    double add = 0.0;
    if (q < PA) {
      int i, j;
      packed_ij(q, i, j);
      a = w.Bt + i * rs;
      b = w.Bt + j * rs;
      out = w.A + i * nA + j;
      if (i < nu_) add = cdiv * t.Adiv[i * nu_ + j];
      else if (LO && is_rot_dof(s, i) && is_rot_dof(s, j)) add = cstab;   // nu (div phi_f, div phi_g)_T
    } else if (q < PA + PV) {
      const int qq = q - PA, i = qq / nA, j = qq - i * nA;
      a = w.Ct + i * rs;
      b = w.Bt + j * rs;
      out = w.V + i * nA + j;
    } else {
      int i, j;
      packed_ij(q - PA - PV, i, j);
      a = w.Ct + i * rs;
      b = w.Ct + j * rs;
      out = w.Sc + i * ncc + j;
    }
    double v0 = 0.0, v1 = 0.0;
    int k2 = 0;
    for (; k2 + 1 < nraw; k2 += 2) {
      v0 += a[k2] * b[k2];
      v1 += a[k2 + 1] * b[k2 + 1];
    }
    if (k2 < nraw) v0 += a[k2] * b[k2];
    *out = v0 + v1 + add;
  }
  sync();
  // ---- Sc = Lc Lc^T and Z = Lc^{-1} V in one elimination ----
  chol_solve_inplace(ncc, w.Sc, nA, w.V, lane, nl, sync);
  // ---- A -= Z^T Z (packed lower), signs, symmetric fill ----
  const int nfd = (d + 1) * s.nF;
  for (int q = lane; q < PA; q += nl) {
    int i, j;
    packed_ij(q, i, j);
    double v = w.A[i * nA + j];
    for (int p = 0; p < ncc; ++p) v -= w.V[p * nA + i] * w.V[p * nA + j];
    const double si = (i < nfd) ? (double)sgn[i / s.nF] : ((LO && is_rot_dof(s, i)) ? (double)sgn[(i - nu_) / s.nhF] : 1.0);
    const double sj = (j < nfd) ? (double)sgn[j / s.nF] : ((LO && is_rot_dof(s, j)) ? (double)sgn[(j - nu_) / s.nhF] : 1.0);
    v *= si * sj;
    w.A[i * nA + j] = v;
    w.A[j * nA + i] = v;
  }
  sync();
}

template <class Sync>
__host__ __device__ inline void condense_element(const ElemSizes& s, const ElemTables& t, const double* X,
                                                 const int* sgn, double nu, ElemWork w, int lane, int nl,
                                                 Sync sync) {
  if (s.lowest) condense_element_t<true>(s, t, X, sgn, nu, w, lane, nl, sync);
  else condense_element_t<false>(s, t, X, sgn, nu, w, lane, nl, sync);
}

// Local stress recovery (eq. projection): after condense_element for the same element, the
// stress of the element-local problem for the velocity coefficients a (local basis, n_A values,
// orientation signs removed) is sigma = (I - Ct^T (Ct Ct^T)^{-1} Ct) Bt^T a in the whitened raw
// basis, i.e. M^{-1} B_sigma^T a on the nt- and rotation-constrained space.  It is mapped back to the
// raw basis (sigma_raw = cB (I (x) L) sigma~) and evaluated at nq reference points with the Dubiner
// values psi [nq][nk]:  sigma(x) = J^{-T} (sum_{i,s} sigma_raw[i,s] psi_i(x^) E_s) J^T.
// work: n_cc + n_raw + n_raw doubles; out: [nq][d][d].  X: vertex coordinates [(d+1)][d].
// The rotation omega is the multiplier of the weak-symmetry rows of Ct: in the raw basis
// M sigma = B^T a - C^T y / cB, and the raw rotation rows are (1/|det J|) (Phi : K_r psi), so
// omega = sum_{r, i<n_p} w_{r,i} psi_i K_r with w = -y_rot / (cB |det J|) (skew units K_r unmapped);
// out_w [nq][d][d] (may be NULL).
template <class Sync>
__host__ __device__ inline void recover_element(const ElemSizes& s, ElemWork w, const double* X, const double* a,
                                                int nq, const double* psi, double* work, double* out,
                                                double* out_w, int lane, int nl, Sync sync) {
  const int nA = s.n_A, ncc = s.n_cc, nraw = s.n_raw, ns0 = s.n_s0, d = s.d, rs = raw_stride(s);
  double* y = work;              // [ncc]
  double* st = y + ncc;          // [nraw] whitened
  double* sr = st + nraw;        // [nraw] raw
  // g = Z a (Z = Lc^{-1} Ct Bt^T is in w.V), then y = Lc^{-T} g
  for (int c = lane; c < ncc; c += nl) {
    double v = 0;
    for (int i = 0; i < nA; ++i) v += w.V[c * nA + i] * a[i];
    y[c] = v;
  }
  sync();
  if (lane == 0)
    for (int i = ncc - 1; i >= 0; --i) {
      double v = y[i];
      for (int p = i + 1; p < ncc; ++p) v -= w.Sc[p * ncc + i] * y[p];
      y[i] = v / w.Sc[i * ncc + i];
    }
  sync();
  for (int j = lane; j < nraw; j += nl) {
    double v = 0;
    for (int i = 0; i < nA; ++i) v += w.Bt[i * rs + j] * a[i];
    for (int c = 0; c < ncc; ++c) v -= w.Ct[c * rs + j] * y[c];
    st[j] = v;
  }
  sync();
  const double* L = w.geo;
  const double cB = sqrt(w.geo[102] / w.geo[100]);
  for (int j = lane; j < nraw; j += nl) {
    const int i = j / ns0, p = j - i * ns0;
    double v = 0;
    for (int q = 0; q <= p; ++q) v += L[p * ns0 + q] * st[i * ns0 + q];
    sr[j] = cB * v;
  }
  sync();
  double J[9], Ji[9];
  for (int aa = 0; aa < d; ++aa)
    for (int i = 0; i < d; ++i) J[aa * d + i] = X[(i + 1) * d + aa] - X[aa];
  if (d == 2) {
    const double det = J[0] * J[3] - J[1] * J[2];
    Ji[0] = J[3] / det; Ji[1] = -J[1] / det; Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
  } else {
    const double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                       J[2] * (J[3] * J[7] - J[4] * J[6]);
    Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
    Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
    Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
    Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
    Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
  }
  for (int q = lane; q < nq; q += nl) {
    double E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // sum_{i,s} sigma_raw psi_i E_s (reference tensor)
    for (int i = 0; i < s.nk; ++i) {
      const double pv = psi[q * s.nk + i];
      for (int p = 0; p < ns0; ++p) {
        const double c = sr[i * ns0 + p] * pv;
        for (int aa = 0; aa < d; ++aa)
          for (int bb = 0; bb < d; ++bb) E[aa * d + bb] += c * tf_unit(d, p, aa, bb);
      }
    }
    // J^{-T} E J^T: entry (i, j) = sum_{a,b} Ji[a][i] E[a][b] J[j][b]
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        double v = 0;
        for (int aa = 0; aa < d; ++aa)
          for (int bb = 0; bb < d; ++bb) v += Ji[aa * d + i] * E[aa * d + bb] * J[j * d + bb];
        out[(q * d + i) * d + j] = v;
      }
    if (out_w && !s.lowest) {
      const double sc = -1.0 / (cB * w.geo[100]);
      double Wm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int r = 0; r < s.n_wskew; ++r)
        for (int ip = 0; ip < s.n_p; ++ip) {
          const double c = sc * y[s.n_con + r * s.n_p + ip] * psi[q * s.nk + ip];
          for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) Wm[i * d + j] += c * skew_unit(d, r, i, j);
        }
      for (int i = 0; i < d * d; ++i) out_w[q * d * d + i] = Wm[i];
    }
  }
  sync();
}

// coupling index (facet-major: facet f, t < nF facet-BDM mode, t >= nF uhat mode) -> local A index
__host__ __device__ inline int coupling_to_local(const ElemSizes& s, int c) {
  int f = c / s.mF, t = c % s.mF;
  return (t < s.nF) ? f * s.nF + t : s.n_u + f * s.nhF + (t - s.nF);
}

// Bubble ("double Schur") condensation of A (n_A x n_A, full, in/out scratch):
//   Aoo^{-1} (n_o x n_o), G = Aoo^{-1} Aoc (n_o x n_c), Ad = Acc - Aoc^T G (n_c x n_c),
// coupling dofs in facet-major order.  work needs n_o*n_o + n_o*n_c doubles.
template <class Sync>
__host__ __device__ inline void bubble_condense(const ElemSizes& s, const double* A, double* work, double* Ad,
                                                double* G, double* Aoo_inv, int lane, int nl, Sync sync) {
  const int no = s.n_bub, nc = s.n_c, nA = s.n_A, ob = (s.d + 1) * s.nF;
  double* Lo = work;           // Cholesky of Aoo
  double* Tm = work + no * no; // Lo^{-1} Aoc
  for (int t = lane; t < no * no; t += nl) {
    int i = t / no, j = t % no;
    Lo[t] = A[(ob + i) * nA + ob + j];
  }
  for (int t = lane; t < no * nc; t += nl) {
    int i = t / nc, c = t % nc;
    Tm[t] = A[(ob + i) * nA + coupling_to_local(s, c)];
  }
  sync();
  chol_solve_inplace(no, Lo, nc, Tm, lane, nl, sync);   // Aoo = Lo Lo^T, Tm = Lo^{-1} Aoc
  // Ad = Acc - Y^T Y
  for (int t = lane; t < nc * nc; t += nl) {
    int i = t / nc, j = t % nc;
    double v = A[coupling_to_local(s, i) * nA + coupling_to_local(s, j)];
    for (int p = 0; p < no; ++p) v -= Tm[p * nc + i] * Tm[p * nc + j];
    Ad[t] = v;
  }
  // G = Lo^{-T} Y (back substitution, columns per lane)
  for (int c = lane; c < nc; c += nl)
    for (int i = no - 1; i >= 0; --i) {
      double v = Tm[i * nc + c];
      for (int p = i + 1; p < no; ++p) v -= Lo[p * no + i] * G[p * nc + c];
      G[i * nc + c] = v / Lo[i * no + i];
    }
  // Aoo^{-1} = Lo^{-T} Lo^{-1}: column j solves, the forward result kept in the output column itself
  // (the backward pass reads y_i before it overwrites it)
  for (int j = lane; j < no; j += nl) {
    for (int i = 0; i < no; ++i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int p = 0; p < i; ++p) v -= Lo[i * no + p] * Aoo_inv[p * no + j];
      Aoo_inv[i * no + j] = v / Lo[i * no + i];
    }
    for (int i = no - 1; i >= 0; --i) {
      double v = Aoo_inv[i * no + j];
      for (int p = i + 1; p < no; ++p) v -= Lo[p * no + i] * Aoo_inv[p * no + j];
      Aoo_inv[i * no + j] = v / Lo[i * no + i];
    }
  }
  sync();
}

}  // namespace mcs
