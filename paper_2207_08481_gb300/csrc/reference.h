// Reference-element tables of the MCS discretization (host side of libmcs).
//
// Everything here is computed once per (d, k) on the host, in FP64, from the
// space definitions of arXiv 2207.08481 Sec. 3 (eqs. fes_V .. fes_Vbar) and the
// dof contract documented in include/mcs.h.  The element kernels combine these
// tables with per-element geometric factors:
//
//   * V_h = BDM^k, mapped by the |det J| Piola transform u = J uhat / |det J|;
//   * Sigma_h(T) = J^{-T} Sigma(T_hat) J^T (covariant-contravariant map, which
//     preserves trace-freeness and the degree of the nt trace); its elements
//     are written in a raw trace-free basis psi_i E_s and the nt conditions are
//     kept as linear constraints, eliminated with the rotation constraints by
//     Lagrange multipliers inside the condensation;
//   * W_h(T) = P^{k-1}(T, skew), Vhat_h on facets q_j e_m (edge vectors e_m),
//     Q_h = P^{k-1}(T);
//   * lowest-order variant (k = 1, Sec. 7, d = 3): W_h in H(div), P^0(T, R^3) + x P^0(T),
//     one flux dof per facet stored behind that facet's two tangential Vhat_h dofs and kept
//     after condensation; the constraint set is then the nt conditions alone.
#pragma once
#include <cstdint>
#include <vector>

namespace mcs {

int n_poly(int n, int k);  // dim P^k(R^n)

struct Sizes {
  int d, k;
  int nk;        // dim P^k(T)
  int nF;        // dim P^k(F)      (BDM facet modes)
  int nFm1;      // dim P^{k-1}(F)
  int n_full;    // d * nk = n_u
  int n_bub;     // interior (bubble) BDM functions
  int ntF;       // (d-1) * nFm1 tangential facet dofs per facet
  int nhF;       // Vhat_h dofs per facet: ntF, plus the rotation flux for the lowest-order variant
  int lowest;    // 1 for the lowest-order variant (k = 1, Sec. 7; d = 3)
  int n_hat;     // (d+1) * nhF
  int n_u, n_A;  // n_A = n_u + n_hat
  int n_p;       // dim P^{k-1}(T)
  int n_s0;      // d*d - 1 trace-free units
  int n_raw;     // n_s0 * nk raw stress functions
  int n_con;     // nt constraints
  int n_w;       // element-local rotation functions (d(d-1)/2 * n_p; 0 for k = 1)
  int n_cc;      // n_con + n_w
  int n_c;       // coupling dofs per element: (d+1)*(nF + nhF)
  int mF;        // nF + nhF dofs per facet
  int n_wskew;   // d(d-1)/2
};
Sizes make_sizes(int d, int k);

struct RefTables {
  Sizes s;
  // ---- condensation tables (row-major) ----
  std::vector<double> B0;     // [n_u][n_raw]  -int R:Dphi + int_dT (R n).phi
  std::vector<double> Rf;     // [d+1][d][nF][n_raw]  int_Ff (R n)_a (phi_i . n), facet-f rows only
  std::vector<double> Bh;     // [n_hat][n_raw]  -int_Ff q e_m^T R n
  std::vector<double> Ccon;   // [n_con][n_raw]  nt constraints (top-degree facet moments)
  std::vector<double> Adiv;   // [n_u][n_u]      int div phi_i div phi_j
  std::vector<double> Bp;     // [n_p][n_u]      int div phi_j psi_i
  std::vector<double> Mu;     // [d][d][n_u][n_u] int phi_{i,a} phi_{j,b}
  std::vector<double> nhat;   // [d+1][d] unit outward reference normals
  std::vector<double> Wmom;   // k = 1: [d+1][d][nk]  int psi_i (xhat_c - xhat_f,c), xhat_f = vertex f
  // ---- load vector (f given at quadrature points) ----
  int nq_load;
  std::vector<double> xq_load;   // [nq][d] reference points
  std::vector<double> wq_load;   // [nq]
  std::vector<double> phi_load;  // [nq][n_u][d] reference basis values
  // ---- embedding E^d: int over the facet parameter simplex of lambda_w q_j ----
  std::vector<double> Ilam;      // [d][nF]
  double facet_ref_measure;      // |T_{d-1}| = 1/(d-1)!
  // ---- BDM reference dual basis (for tests / diagnostics) ----
  std::vector<double> CU;        // [n_full][n_full] ambient (a*nk+i) x dual function
};

RefTables build_reference(int d, int k);

// Reference quadrature (collapsed Gauss-Legendre with the Duffy Jacobian in the
// weights); q points per direction integrate total degree 2q-3 (n=3),
// 2q-2 (n=2), 2q-1 (n=1) exactly.
void duffy_rule(int n, int q, std::vector<double>& pts, std::vector<double>& w);
// Collapsed Gauss-Jacobi rule on T_n (n = 2, 3) with q points per direction (the load rule).
void collapsed_gauss_rule(int n, int q, std::vector<double>& pts, std::vector<double>& w);
// Orthonormal (Dubiner) basis of P^k(T_n) at one point: val[nb], grad[nb][n].
void dubiner_eval(int n, int k, const double* x, double* val, double* grad);

}  // namespace mcs
