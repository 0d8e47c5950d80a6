// Reference-element tables of the MCS discretization (see reference.h).
#include "reference.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <stdexcept>
#include <utility>

namespace mcs {

int n_poly(int n, int k) {
  if (k < 0) return 0;
  long r = 1;
  for (int i = 1; i <= n; ++i) r = r * (k + i) / i;
  return (int)r;
}

Sizes make_sizes(int d, int k) {
  Sizes s{};
  s.d = d;
  s.k = k;
  s.nk = n_poly(d, k);
  s.nF = n_poly(d - 1, k);
  s.nFm1 = n_poly(d - 1, k - 1);
  s.n_full = d * s.nk;
  s.n_bub = s.n_full - (d + 1) * s.nF;
  s.lowest = (k == 1) ? 1 : 0;
  s.ntF = (d - 1) * s.nFm1;
  s.nhF = s.ntF + s.lowest;
  s.n_hat = (d + 1) * s.nhF;
  s.n_u = s.n_full;
  s.n_A = s.n_u + s.n_hat;
  s.n_p = n_poly(d, k - 1);
  s.n_s0 = d * d - 1;
  s.n_raw = s.n_s0 * s.nk;
  s.n_con = (d + 1) * (d - 1) * (s.nF - s.nFm1);
  s.n_wskew = d * (d - 1) / 2;
  s.n_w = s.lowest ? 0 : s.n_wskew * s.n_p;
  s.n_cc = s.n_con + s.n_w;
  s.mF = s.nF + s.nhF;
  s.n_c = (d + 1) * s.mF;
  return s;
}

// ------------------------------------------------------------ quadrature
static void gauss_legendre01(int q, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on P_q from Chebyshev-like starting points, mapped to [0, 1].
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; ++i) {
    double t = std::cos(pi * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int n = 2; n <= q; ++n) {
        double p2 = ((2 * n - 1) * t * p1 - (n - 1) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      double pq = (q == 0) ? 1.0 : (q == 1 ? t : p1);
      double pqm1 = (q == 1) ? 1.0 : p0;
      dp = q * (t * pq - pqm1) / (t * t - 1.0);
      double dt = pq / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    // recompute derivative at converged node
    double p0 = 1.0, p1 = t;
    for (int n = 2; n <= q; ++n) {
      double p2 = ((2 * n - 1) * t * p1 - (n - 1) * p0) / n;
      p0 = p1;
      p1 = p2;
    }
    double pq = (q == 1) ? t : p1, pqm1 = (q == 1) ? 1.0 : p0;
    dp = q * (t * pq - pqm1) / (t * t - 1.0);
    x[i] = 0.5 * (1.0 - t);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2) P'^2) halved for [0,1]
  }
}

// Gauss-Jacobi rule with q nodes on [-1, 1] for the weight (1 - x)^alpha: Newton's method on
// P_q^{(alpha,0)} (three-term recurrence), each root deflated by the ones already found;
// weights 2^{alpha+1} / ((1 - x^2) P_q'(x)^2).
static void jacobi_p(int q, double alpha, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = 0.5 * ((alpha + 2.0) * x + alpha);
  if (q == 0) { p = 1.0; dp = 0.0; return; }
  for (int n = 2; n <= q; ++n) {
    const double c = 2.0 * n + alpha;
    const double a1 = 2.0 * n * (n + alpha) * (c - 2.0);
    const double a2 = (c - 1.0) * (c * (c - 2.0) * x + alpha * alpha);
    const double a3 = 2.0 * (n + alpha - 1.0) * (n - 1.0) * c;
    const double p2 = (a2 * p1 - a3 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  // (2q + alpha)(1 - x^2) P_q' = q (alpha - (2q + alpha) x) P_q + 2 (q + alpha) q P_{q-1}
  const double c = 2.0 * q + alpha;
  dp = (q * (alpha - c * x) * p1 + 2.0 * (q + alpha) * q * p0) / (c * (1.0 - x * x));
}

static void gauss_jacobi(int q, double alpha, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; ++i) {
    double t = -std::cos(pi * (i + 0.75) / (q + 0.5));   // ascending starting points
    for (int it = 0; it < 200; ++it) {
      double p, dp;
      jacobi_p(q, alpha, t, p, dp);
      double sdef = 0.0;                                 // deflation by the roots found
      for (int j = 0; j < i; ++j) sdef += 1.0 / (t - x[j]);
      const double dt = p / (dp - sdef * p);
      t -= dt;
      if (std::fabs(dt) < 1e-15) break;
    }
    double p, dp;
    jacobi_p(q, alpha, t, p, dp);
    x[i] = t;
    w[i] = std::pow(2.0, alpha + 1.0) / ((1.0 - t * t) * dp * dp);
  }
  // ascending nodes
  for (int i = 1; i < q; ++i)
    for (int j = i; j > 0 && x[j] < x[j - 1]; --j) {
      std::swap(x[j], x[j - 1]);
      std::swap(w[j], w[j - 1]);
    }
}

// Collapsed Gauss rule on the reference simplex T_n with q points per direction (the load rule of the
// dof contract): Gauss-Jacobi nodes a (alpha 0), b (alpha 1), c (alpha 2) on [-1, 1] mapped by
// z = (1 + c)/2, y = (1 + b)(1 - c)/4, x = (1 + a)(1 - b)(1 - c)/8 (2D: y = (1 + b)/2,
// x = (1 + a)(1 - b)/4), weights w_a w_b w_c / 64 (2D: / 8).
void collapsed_gauss_rule(int n, int q, std::vector<double>& pts, std::vector<double>& w) {
  std::vector<double> a, wa, b, wb, c, wc;
  gauss_jacobi(q, 0.0, a, wa);
  gauss_jacobi(q, 1.0, b, wb);
  gauss_jacobi(q, 2.0, c, wc);
  pts.clear();
  w.clear();
  if (n == 2) {
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        pts.push_back((1 + a[i]) * (1 - b[j]) / 4);
        pts.push_back((1 + b[j]) / 2);
        w.push_back(wa[i] * wb[j] / 8);
      }
    return;
  }
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j)
      for (int l = 0; l < q; ++l) {
        pts.push_back((1 + a[i]) * (1 - b[j]) * (1 - c[l]) / 8);
        pts.push_back((1 + b[j]) * (1 - c[l]) / 4);
        pts.push_back((1 + c[l]) / 2);
        w.push_back(wa[i] * wb[j] * wc[l] / 64);
      }
}

void duffy_rule(int n, int q, std::vector<double>& pts, std::vector<double>& w) {
  std::vector<double> g, gw;
  gauss_legendre01(q, g, gw);
  pts.clear();
  w.clear();
  if (n == 0) {
    w.push_back(1.0);
    return;
  }
  if (n == 1) {
    for (int i = 0; i < q; ++i) {
      pts.push_back(g[i]);
      w.push_back(gw[i]);
    }
    return;
  }
  if (n == 2) {
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        double a = g[i], b = g[j];
        pts.push_back(a * (1 - b));
        pts.push_back(b);
        w.push_back(gw[i] * gw[j] * (1 - b));
      }
    return;
  }
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j)
      for (int l = 0; l < q; ++l) {
        double a = g[i], b = g[j], c = g[l];
        pts.push_back(a * (1 - b) * (1 - c));
        pts.push_back(b * (1 - c));
        pts.push_back(c);
        w.push_back(gw[i] * gw[j] * gw[l] * (1 - b) * (1 - c) * (1 - c));
      }
}

// ------------------------------------------------------------ Dubiner basis
// Homogeneous Jacobi H_m^{(alpha)}(x, s) = s^m P_m^{(alpha,0)}(2x/s - 1) with d/dx, d/ds.
static void hjac(int m, int alpha, double x, double s, double& v, double& vx, double& vs) {
  double h0 = 1, h0x = 0, h0s = 0;
  if (m == 0) {
    v = 1;
    vx = 0;
    vs = 0;
    return;
  }
  double h1 = (alpha + 2) * x - s, h1x = alpha + 2, h1s = -1;
  const double a = alpha;
  for (int n = 2; n <= m; ++n) {
    double an = 2.0 * n * (n + a) * (2 * n + a - 2);
    double bn = (2 * n + a - 1) * (2 * n + a) * (2 * n + a - 2);
    double cn = (2 * n + a - 1) * a * a;
    double dn = 2.0 * (n + a - 1) * (n - 1) * (2 * n + a);
    double lin = bn * (2 * x - s) + cn * s;
    double h2 = (lin * h1 - dn * s * s * h0) / an;
    double h2x = (2 * bn * h1 + lin * h1x - dn * s * s * h0x) / an;
    double h2s = ((cn - bn) * h1 + lin * h1s - 2 * dn * s * h0 - dn * s * s * h0s) / an;
    h0 = h1; h0x = h1x; h0s = h1s;
    h1 = h2; h1x = h2x; h1s = h2s;
  }
  v = h1;
  vx = h1x;
  vs = h1s;
}

struct Idx3 { int p, q, r; };

static std::vector<Idx3> dubiner_indices(int n, int k) {
  std::vector<Idx3> out;
  for (int m = 0; m <= k; ++m) {
    if (n == 1) out.push_back({m, 0, 0});
    else if (n == 2)
      for (int q = 0; q <= m; ++q) out.push_back({m - q, q, 0});
    else
      for (int r = 0; r <= m; ++r)
        for (int q = 0; q <= m - r; ++q) out.push_back({m - q - r, q, r});
  }
  return out;
}

static void raw_dubiner(int n, const Idx3& id, const double* x, double& v, double* g) {
  if (n == 1) {
    double A, Ax, As;
    hjac(id.p, 0, x[0], 1.0, A, Ax, As);
    v = A;
    g[0] = Ax;
    return;
  }
  if (n == 2) {
    double A, Ax, As, B, Bx, Bs;
    hjac(id.p, 0, x[0], 1.0 - x[1], A, Ax, As);
    hjac(id.q, 2 * id.p + 1, x[1], 1.0, B, Bx, Bs);
    v = A * B;
    g[0] = Ax * B;
    g[1] = -As * B + A * Bx;
    return;
  }
  double A, Ax, As, B, Bx, Bs, C, Cx, Cs;
  hjac(id.p, 0, x[0], 1.0 - x[1] - x[2], A, Ax, As);
  hjac(id.q, 2 * id.p + 1, x[1], 1.0 - x[2], B, Bx, Bs);
  hjac(id.r, 2 * id.p + 2 * id.q + 2, x[2], 1.0, C, Cx, Cs);
  v = A * B * C;
  g[0] = Ax * B * C;
  g[1] = -As * B * C + A * Bx * C;
  g[2] = -As * B * C - A * Bs * C + A * B * Cx;
}

static const std::vector<double>& dubiner_norms(int n, int k) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, std::vector<double>> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(n, k);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  std::vector<double> pts, w;
  duffy_rule(n, k + 3, pts, w);
  auto ids = dubiner_indices(n, k);
  std::vector<double> nrm(ids.size());
  double g[3];
  for (size_t b = 0; b < ids.size(); ++b) {
    double acc = 0;
    for (size_t q = 0; q < w.size(); ++q) {
      double v;
      raw_dubiner(n, ids[b], &pts[q * n], v, g);
      acc += w[q] * v * v;
    }
    nrm[b] = 1.0 / std::sqrt(acc);
  }
  return cache.emplace(key, std::move(nrm)).first->second;
}

void dubiner_eval(int n, int k, const double* x, double* val, double* grad) {
  auto ids = dubiner_indices(n, k);
  const auto& nrm = dubiner_norms(n, k);
  double g[3];
  for (size_t b = 0; b < ids.size(); ++b) {
    double v;
    raw_dubiner(n, ids[b], x, v, g);
    val[b] = nrm[b] * v;
    if (grad)
      for (int a = 0; a < n; ++a) grad[b * n + a] = nrm[b] * g[a];
  }
}

// ------------------------------------------------------------ dense helpers
static void invert(int n, std::vector<double>& A) {
  // Gauss-Jordan with partial pivoting, in place (row-major).
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (std::fabs(A[piv * n + c]) < 1e-300) throw std::runtime_error("singular reference matrix");
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[c * n + j], A[piv * n + j]);
        std::swap(I[c * n + j], I[piv * n + j]);
      }
    double inv = 1.0 / A[c * n + c];
    for (int j = 0; j < n; ++j) {
      A[c * n + j] *= inv;
      I[c * n + j] *= inv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[r * n + j] -= f * A[c * n + j];
        I[r * n + j] -= f * I[c * n + j];
      }
    }
  }
  A.swap(I);
}

// ------------------------------------------------------------ the element spaces
namespace {

struct RefGeom {
  int d;
  std::vector<std::vector<double>> V;        // reference vertices
  std::vector<std::vector<int>> fv;          // facet f: sorted local vertices (all but f)
  std::vector<std::vector<double>> n;        // unit outward normals
  std::vector<double> meas;                  // facet measures
};

RefGeom ref_geom(int d) {
  RefGeom g;
  g.d = d;
  g.V.assign(d + 1, std::vector<double>(d, 0.0));
  for (int i = 0; i < d; ++i) g.V[i + 1][i] = 1.0;
  g.fv.resize(d + 1);
  g.n.assign(d + 1, std::vector<double>(d, 0.0));
  g.meas.resize(d + 1);
  for (int f = 0; f <= d; ++f) {
    for (int v = 0; v <= d; ++v)
      if (v != f) g.fv[f].push_back(v);
    if (f == 0)
      for (int a = 0; a < d; ++a) g.n[f][a] = 1.0 / std::sqrt((double)d);
    else
      g.n[f][f - 1] = -1.0;
    // measure: sqrt(det(E E^T)) / (d-1)!
    std::vector<std::vector<double>> E(d - 1, std::vector<double>(d));
    for (int m = 1; m < d; ++m)
      for (int a = 0; a < d; ++a) E[m - 1][a] = g.V[g.fv[f][m]][a] - g.V[g.fv[f][0]][a];
    double G;
    if (d == 2) G = E[0][0] * E[0][0] + E[0][1] * E[0][1];
    else {
      double g00 = 0, g01 = 0, g11 = 0;
      for (int a = 0; a < 3; ++a) {
        g00 += E[0][a] * E[0][a];
        g01 += E[0][a] * E[1][a];
        g11 += E[1][a] * E[1][a];
      }
      G = g00 * g11 - g01 * g01;
    }
    g.meas[f] = std::sqrt(G) / (d == 3 ? 2.0 : 1.0);
  }
  return g;
}

// interior test functions g_m(xhat) before orthonormalisation: the first-kind Nedelec list of the dof
// contract (build_reference makes it L2(T_hat)-orthonormal)
void interior_tests(int d, int k, const double* x, std::vector<double>& out /* [nb][d] */) {
  out.clear();
  int nkm2 = n_poly(d, k - 2);
  std::vector<double> psi(std::max(nkm2, 1));
  if (k >= 2) dubiner_eval(d, k - 2, x, psi.data(), nullptr);
  for (int a = 0; a < nkm2; ++a)
    for (int c = 0; c < d; ++c)
      for (int e = 0; e < d; ++e) out.push_back(e == c ? psi[a] : 0.0);
  int m = k - 2;
  if (d == 2) {
    for (int a = m; a >= 0; --a) {
      double mono = std::pow(x[0], a) * std::pow(x[1], m - a);
      out.push_back(-x[1] * mono);
      out.push_back(x[0] * mono);
    }
  } else {
    for (int a0 = m; a0 >= 0; --a0)
      for (int a1 = m - a0; a1 >= 0; --a1) {
        int a2 = m - a0 - a1;
        double mono = std::pow(x[0], a0) * std::pow(x[1], a1) * std::pow(x[2], a2);
        for (int c = 0; c < 3; ++c) {
          if (c == 2 && a2 >= 1) continue;
          double q[3] = {0, 0, 0};
          q[c] = mono;
          out.push_back(x[1] * q[2] - x[2] * q[1]);
          out.push_back(x[2] * q[0] - x[0] * q[2]);
          out.push_back(x[0] * q[1] - x[1] * q[0]);
        }
      }
  }
}

}  // namespace

RefTables build_reference(int d, int k) {
  if (d < 2 || d > 3 || k < 1 || k > 8 || (k == 1 && d != 3)) throw std::runtime_error("unsupported (d, k)");
  RefTables T;
  Sizes s = make_sizes(d, k);
  T.s = s;
  RefGeom rg = ref_geom(d);
  const int nk = s.nk, nF = s.nF, nu = s.n_u, nraw = s.n_raw, ns0 = s.n_s0;

  // trace-free units E_s (off-diagonal row-major, then e_a e_a^T - e_{a+1} e_{a+1}^T)
  std::vector<double> TF;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b)
      if (a != b) {
        std::vector<double> E(d * d, 0.0);
        E[a * d + b] = 1;
        TF.insert(TF.end(), E.begin(), E.end());
      }
  for (int a = 0; a + 1 < d; ++a) {
    std::vector<double> E(d * d, 0.0);
    E[a * d + a] = 1;
    E[(a + 1) * d + a + 1] = -1;
    TF.insert(TF.end(), E.begin(), E.end());
  }

  // quadrature rules
  std::vector<double> xv, wv, sf, wf;
  duffy_rule(d, k + 2, xv, wv);
  duffy_rule(d - 1, k + 2, sf, wf);
  const int nq = (int)wv.size(), nqf = (int)wf.size();
  const double refF = (d == 3) ? 0.5 : 1.0;  // |T_{d-1}|
  T.facet_ref_measure = refF;

  // ---- BDM dual basis on the reference element ----
  auto amb = [&](const double* x, std::vector<double>& val, std::vector<double>& grad) {
    // ambient Phi_{a*nk+i} = psi_i e_a : val[c][d], grad[c][d][d] (d Phi_a / d x_b)
    std::vector<double> psi(nk), gp(nk * d);
    dubiner_eval(d, k, x, psi.data(), gp.data());
    val.assign(s.n_full * d, 0.0);
    grad.assign(s.n_full * d * d, 0.0);
    for (int a = 0; a < d; ++a)
      for (int i = 0; i < nk; ++i) {
        int c = a * nk + i;
        val[c * d + a] = psi[i];
        for (int b = 0; b < d; ++b) grad[(c * d + a) * d + b] = gp[i * d + b];
      }
  };
  auto facet_point = [&](int f, const double* sp, double* x) {
    const auto& w = rg.fv[f];
    for (int a = 0; a < d; ++a) {
      x[a] = rg.V[w[0]][a];
      for (int m = 1; m < d; ++m) x[a] += sp[m - 1] * (rg.V[w[m]][a] - rg.V[w[0]][a]);
    }
  };
  std::vector<double> qF(nqf * nF);  // facet orthonormal basis at facet points
  for (int q = 0; q < nqf; ++q) dubiner_eval(d - 1, k, &sf[q * (d - 1)], &qF[q * nF], nullptr);

  std::vector<double> C(s.n_full * s.n_full, 0.0);
  std::vector<double> val, grad, x(d);
  for (int f = 0; f <= d; ++f)
    for (int q = 0; q < nqf; ++q) {
      facet_point(f, &sf[q * (d - 1)], x.data());
      amb(x.data(), val, grad);
      double ws = wf[q] * rg.meas[f] / refF;
      for (int c = 0; c < s.n_full; ++c) {
        double fl = 0;
        for (int a = 0; a < d; ++a) fl += val[c * d + a] * rg.n[f][a];
        for (int j = 0; j < nF; ++j) C[(f * nF + j) * s.n_full + c] += ws * fl * qF[q * nF + j];
      }
    }
  // interior moment functions: the contract's list made L2(T_hat)-orthonormal in list order, i.e.
  // g = Lg^{-1} g_list with Lg Lg^T the Gram matrix of the list on T_hat (the rule is exact for it)
  const int nb = s.n_bub;
  std::vector<double> Lgi(std::max(1, nb * nb), 0.0);
  std::vector<double> gt;
  if (nb > 0) {
    std::vector<double> Gm(nb * nb, 0.0);
    for (int q = 0; q < nq; ++q) {
      interior_tests(d, k, &xv[q * d], gt);
      for (int m = 0; m < nb; ++m)
        for (int n2 = 0; n2 < nb; ++n2) {
          double v = 0;
          for (int a = 0; a < d; ++a) v += gt[m * d + a] * gt[n2 * d + a];
          Gm[m * nb + n2] += wv[q] * v;
        }
    }
    // Cholesky Gm = Lg Lg^T, then Lgi = Lg^{-1} (lower) by forward substitution of the unit columns
    std::vector<double> Lg(nb * nb, 0.0);
    for (int j = 0; j < nb; ++j) {
      double dj = Gm[j * nb + j];
      for (int p = 0; p < j; ++p) dj -= Lg[j * nb + p] * Lg[j * nb + p];
      if (!(dj > 0)) throw std::runtime_error("interior moment functions are dependent");
      Lg[j * nb + j] = std::sqrt(dj);
      for (int i = j + 1; i < nb; ++i) {
        double v = Gm[i * nb + j];
        for (int p = 0; p < j; ++p) v -= Lg[i * nb + p] * Lg[j * nb + p];
        Lg[i * nb + j] = v / Lg[j * nb + j];
      }
    }
    for (int c = 0; c < nb; ++c)
      for (int i = c; i < nb; ++i) {
        double v = (i == c) ? 1.0 : 0.0;
        for (int p = c; p < i; ++p) v -= Lg[i * nb + p] * Lgi[p * nb + c];
        Lgi[i * nb + c] = v / Lg[i * nb + i];
      }
  }
  std::vector<double> go(std::max(1, nb * d));
  for (int q = 0; q < nq; ++q) {
    amb(&xv[q * d], val, grad);
    interior_tests(d, k, &xv[q * d], gt);
    for (int m = 0; m < nb; ++m)
      for (int a = 0; a < d; ++a) {
        double v = 0;
        for (int n2 = 0; n2 <= m; ++n2) v += Lgi[m * nb + n2] * gt[n2 * d + a];
        go[m * d + a] = v;
      }
    for (int m = 0; m < nb; ++m)
      for (int c = 0; c < s.n_full; ++c) {
        double v = 0;
        for (int a = 0; a < d; ++a) v += val[c * d + a] * go[m * d + a];
        C[((d + 1) * nF + m) * s.n_full + c] += wv[q] * v;
      }
  }
  invert(s.n_full, C);  // columns of C^{-1} = dual functions
  T.CU = C;

  auto basis = [&](const double* x, std::vector<double>& bv, std::vector<double>& bg) {
    // reference basis phi_r at x: bv[r][d], bg[r][d][d]
    amb(x, val, grad);
    bv.assign(nu * d, 0.0);
    bg.assign(nu * d * d, 0.0);
    for (int c = 0; c < s.n_full; ++c)
      for (int r = 0; r < nu; ++r) {
        double cr = C[c * s.n_full + r];
        if (cr == 0.0) continue;
        for (int a = 0; a < d; ++a) {
          bv[r * d + a] += cr * val[c * d + a];
          for (int b = 0; b < d; ++b) bg[(r * d + a) * d + b] += cr * grad[(c * d + a) * d + b];
        }
      }
  };
  auto raw = [&](const double* x, std::vector<double>& rv, std::vector<double>& rdiv) {
    // raw stress R_{i*ns0+s} = psi_i E_s : rv[j][d][d]; div (row-wise) rdiv[j][d]
    std::vector<double> psi(nk), gp(nk * d);
    dubiner_eval(d, k, x, psi.data(), gp.data());
    rv.assign(nraw * d * d, 0.0);
    rdiv.assign(nraw * d, 0.0);
    for (int i = 0; i < nk; ++i)
      for (int e = 0; e < ns0; ++e) {
        int j = i * ns0 + e;
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) {
            double E = TF[e * d * d + a * d + b];
            rv[(j * d + a) * d + b] = psi[i] * E;
            rdiv[j * d + a] += E * gp[i * d + b];
          }
      }
  };

  // ---- volume tables ----
  T.B0.assign(nu * nraw, 0.0);
  T.Adiv.assign(nu * nu, 0.0);
  T.Bp.assign(s.n_p * nu, 0.0);
  T.Mu.assign(d * d * nu * nu, 0.0);
  std::vector<double> bv, bg, rv, rdiv, psi(nk);
  for (int q = 0; q < nq; ++q) {
    const double* xq = &xv[q * d];
    basis(xq, bv, bg);
    raw(xq, rv, rdiv);
    dubiner_eval(d, k, xq, psi.data(), nullptr);
    std::vector<double> dv(nu, 0.0);
    for (int r = 0; r < nu; ++r)
      for (int a = 0; a < d; ++a) dv[r] += bg[(r * d + a) * d + a];
    for (int r = 0; r < nu; ++r) {
      for (int j = 0; j < nraw; ++j) {
        double v = 0;
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) v += rv[(j * d + a) * d + b] * bg[(r * d + a) * d + b];
        T.B0[r * nraw + j] -= wv[q] * v;
      }
      for (int c = 0; c < nu; ++c) T.Adiv[r * nu + c] += wv[q] * dv[r] * dv[c];
      for (int i = 0; i < s.n_p; ++i) T.Bp[i * nu + r] += wv[q] * dv[r] * psi[i];
      for (int c = 0; c < nu; ++c)
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b)
            T.Mu[((a * d + b) * nu + r) * nu + c] += wv[q] * bv[r * d + a] * bv[c * d + b];
    }
  }

  // ---- facet tables ----
  T.Rf.assign((d + 1) * d * nF * nraw, 0.0);
  T.Bh.assign(s.n_hat * nraw, 0.0);
  T.Ccon.assign(s.n_con * nraw, 0.0);
  T.nhat.assign((d + 1) * d, 0.0);
  int con_row = 0;
  for (int f = 0; f <= d; ++f) {
    const auto& n = rg.n[f];
    for (int a = 0; a < d; ++a) T.nhat[f * d + a] = n[a];
    const auto& w = rg.fv[f];
    std::vector<std::vector<double>> e(d - 1, std::vector<double>(d));
    for (int m = 1; m < d; ++m)
      for (int a = 0; a < d; ++a) e[m - 1][a] = rg.V[w[m]][a] - rg.V[w[0]][a];
    std::vector<int> top;
    {
      // facet modes of exact degree k are the last nF - nFm1 ones
      for (int j = s.nFm1; j < nF; ++j) top.push_back(j);
    }
    for (int q = 0; q < nqf; ++q) {
      facet_point(f, &sf[q * (d - 1)], x.data());
      basis(x.data(), bv, bg);
      raw(x.data(), rv, rdiv);
      double ws = wf[q] * rg.meas[f] / refF;
      const double* qq = &qF[q * nF];
      for (int j = 0; j < nraw; ++j) {
        double Rn[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) Rn[a] += rv[(j * d + a) * d + b] * n[b];
        // B0 boundary part: (R n) . phi_r over all functions
        for (int r = 0; r < nu; ++r) {
          double v = 0;
          for (int a = 0; a < d; ++a) v += Rn[a] * bv[r * d + a];
          T.B0[r * nraw + j] += ws * v;
        }
        // Rf: facet-f functions only
        for (int jF = 0; jF < nF; ++jF) {
          int r = f * nF + jF;
          double un = 0;
          for (int a = 0; a < d; ++a) un += bv[r * d + a] * n[a];
          for (int a = 0; a < d; ++a) T.Rf[((f * d + a) * nF + jF) * nraw + j] += ws * Rn[a] * un;
        }
        // Bh and the nt constraints
        for (int m = 0; m < d - 1; ++m) {
          double tRn = 0;
          for (int a = 0; a < d; ++a) tRn += e[m][a] * Rn[a];
          for (int jq = 0; jq < s.nFm1; ++jq) {
            int row = f * s.nhF + m * s.nFm1 + jq;
            T.Bh[row * nraw + j] -= ws * qq[jq] * tRn;
          }
          for (size_t t = 0; t < top.size(); ++t) {
            int row = con_row + m * (int)top.size() + (int)t;
            T.Ccon[row * nraw + j] += ws * qq[top[t]] * tRn;
          }
        }
      }
    }
    con_row += (d - 1) * (int)top.size();
  }

  // ---- k = 1: moments of the rotation flux functions (x - x_f) / (d |T|) against psi_i ----
  if (s.lowest) {
    T.Wmom.assign((d + 1) * d * nk, 0.0);
    for (int q = 0; q < nq; ++q) {
      dubiner_eval(d, k, &xv[q * d], psi.data(), nullptr);
      for (int f = 0; f <= d; ++f)
        for (int c = 0; c < d; ++c)
          for (int i = 0; i < nk; ++i) T.Wmom[(f * d + c) * nk + i] += wv[q] * psi[i] * (xv[q * d + c] - rg.V[f][c]);
    }
  }

  // ---- load vector quadrature ----
  {
    std::vector<double> xl, wl;
    collapsed_gauss_rule(d, k + 8, xl, wl);   // the load rule of the dof contract, k + 8 points per direction
    T.nq_load = (int)wl.size();
    T.xq_load = xl;
    T.wq_load = wl;
    T.phi_load.assign(T.nq_load * nu * d, 0.0);
    for (int q = 0; q < T.nq_load; ++q) {
      basis(&xl[q * d], bv, bg);
      for (int i = 0; i < nu * d; ++i) T.phi_load[q * nu * d + i] = bv[i];
    }
  }

  // ---- E^d facet integrals: int lambda_w q_j over the facet parameter simplex ----
  T.Ilam.assign(d * nF, 0.0);
  for (int q = 0; q < nqf; ++q) {
    const double* sp = &sf[q * (d - 1)];
    double lam[3];
    lam[0] = 1.0;
    for (int m = 1; m < d; ++m) {
      lam[m] = sp[m - 1];
      lam[0] -= sp[m - 1];
    }
    for (int wv_ = 0; wv_ < d; ++wv_)
      for (int j = 0; j < nF; ++j) T.Ilam[wv_ * nF + j] += wf[q] * lam[wv_] * qF[q * nF + j];
  }
  return T;
}

}  // namespace mcs
