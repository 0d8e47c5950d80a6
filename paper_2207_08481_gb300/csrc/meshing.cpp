// Host-side mesh, dof maps, colouring and multigrid hierarchy (see meshing.h).
#include "meshing.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>
#include <stdexcept>

namespace mcs {

void build_facets(HostMesh& m) {
  const int d = m.d;
  const int64_t ne = m.ne;
  struct Key {
    std::array<int32_t, 3> v;
    int32_t T, f;
  };
  std::vector<Key> keys((size_t)ne * (d + 1));
  for (int64_t T = 0; T < ne; ++T)
    for (int f = 0; f <= d; ++f) {
      Key& k = keys[T * (d + 1) + f];
      int c = 0;
      k.v = {0, 0, 0};
      for (int v = 0; v <= d; ++v)
        if (v != f) k.v[c++] = m.elems[T * (d + 1) + v];
      k.T = (int32_t)T;
      k.f = f;
    }
  std::sort(keys.begin(), keys.end(), [d](const Key& a, const Key& b) {
    for (int i = 0; i < d; ++i)
      if (a.v[i] != b.v[i]) return a.v[i] < b.v[i];
    return a.T < b.T;
  });
  m.elem_facets.assign(ne * (d + 1), -1);
  m.facets.clear();
  m.facet_elems.clear();
  int64_t nf = 0;
  for (size_t i = 0; i < keys.size(); ++i) {
    bool same = i > 0;
    if (same)
      for (int a = 0; a < d; ++a)
        if (keys[i].v[a] != keys[i - 1].v[a]) same = false;
    if (!same) {
      for (int a = 0; a < d; ++a) m.facets.push_back(keys[i].v[a]);
      m.facet_elems.push_back(keys[i].T);
      m.facet_elems.push_back(-1);
      ++nf;
    } else {
      if (m.facet_elems[(nf - 1) * 2 + 1] >= 0) throw std::runtime_error("facet shared by more than two elements");
      m.facet_elems[(nf - 1) * 2 + 1] = keys[i].T;
    }
    m.elem_facets[keys[i].T * (d + 1) + keys[i].f] = (int32_t)(nf - 1);
  }
  m.nf = nf;
  m.int_rank.assign(nf, -1);
  m.int_facets.clear();
  for (int64_t F = 0; F < nf; ++F)
    if (m.facet_elems[F * 2 + 1] >= 0) {
      m.int_rank[F] = (int32_t)m.int_facets.size();
      m.int_facets.push_back((int32_t)F);
    }
  m.nint = (int64_t)m.int_facets.size();
  // normals: det[e_1..e_{d-1}, n] > 0
  m.normals.assign(nf * d, 0.0);
  for (int64_t F = 0; F < nf; ++F) {
    const int32_t* w = &m.facets[F * d];
    double e[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (int mm = 1; mm < d; ++mm)
      for (int a = 0; a < d; ++a) e[mm - 1][a] = m.coords[w[mm] * d + a] - m.coords[w[0] * d + a];
    double n[3];
    if (d == 2) {
      n[0] = -e[0][1];
      n[1] = e[0][0];
    } else {
      n[0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
      n[1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
      n[2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
    }
    double len = 0;
    for (int a = 0; a < d; ++a) len += n[a] * n[a];
    len = std::sqrt(len);
    for (int a = 0; a < d; ++a) m.normals[F * d + a] = n[a] / len;
  }
  m.signs.assign(ne * (d + 1), 0);
  m.elem_rank.assign(ne * (d + 1), -1);
  for (int64_t T = 0; T < ne; ++T)
    for (int f = 0; f <= d; ++f) {
      int32_t F = m.elem_facets[T * (d + 1) + f];
      int32_t w0 = m.facets[F * d], vf = m.elems[T * (d + 1) + f];
      double dot = 0;
      for (int a = 0; a < d; ++a) dot += m.normals[F * d + a] * (m.coords[w0 * d + a] - m.coords[vf * d + a]);
      m.signs[T * (d + 1) + f] = dot > 0 ? 1 : -1;
      m.elem_rank[T * (d + 1) + f] = m.int_rank[F];
    }
  m.int_local.assign(m.nint * 2, -1);
  for (int64_t r = 0; r < m.nint; ++r) {
    int32_t F = m.int_facets[r];
    for (int side = 0; side < 2; ++side) {
      int32_t T = m.facet_elems[F * 2 + side];
      for (int f = 0; f <= d; ++f)
        if (m.elem_facets[T * (d + 1) + f] == F) m.int_local[r * 2 + side] = f;
    }
  }
}

void mark_outflow(HostMesh& m) {
  const int d = m.d;
  m.outflow.assign(m.nf, 0);
  for (int64_t F = 0; F < m.nf; ++F) {
    if (m.facet_elems[F * 2 + 1] >= 0) continue;
    bool on = true;
    for (int a = 0; a < d; ++a) on = on && m.coords[(int64_t)m.facets[F * d + a] * d] == 1.0;
    m.outflow[F] = on ? 1 : 0;
  }
  m.int_rank.assign(m.nf, -1);
  m.int_facets.clear();
  for (int64_t F = 0; F < m.nf; ++F)
    if (m.facet_elems[F * 2 + 1] >= 0 || m.outflow[F]) {
      m.int_rank[F] = (int32_t)m.int_facets.size();
      m.int_facets.push_back((int32_t)F);
    }
  m.nint = (int64_t)m.int_facets.size();
  for (int64_t T = 0; T < m.ne; ++T)
    for (int f = 0; f <= d; ++f) m.elem_rank[T * (d + 1) + f] = m.int_rank[m.elem_facets[T * (d + 1) + f]];
  m.int_local.assign(m.nint * 2, -1);
  for (int64_t r = 0; r < m.nint; ++r) {
    const int32_t F = m.int_facets[r];
    for (int side = 0; side < 2; ++side) {
      const int32_t T = m.facet_elems[F * 2 + side];
      if (T < 0) continue;
      for (int f = 0; f <= d; ++f)
        if (m.elem_facets[T * (d + 1) + f] == F) m.int_local[r * 2 + side] = f;
    }
  }
}

HostMesh structured_mesh(int d, int N) {
  if (d < 2 || d > 3 || N < 1) throw std::runtime_error("structured_mesh: bad arguments");
  HostMesh m;
  m.d = d;
  const int64_t n1 = N + 1;
  m.nv = (d == 2) ? n1 * n1 : n1 * n1 * n1;
  m.coords.resize(m.nv * d);
  for (int64_t v = 0; v < m.nv; ++v) {
    int64_t t = v;
    for (int a = 0; a < d; ++a) {
      m.coords[v * d + a] = (double)(t % n1) / N;
      t /= n1;
    }
  }
  std::vector<std::array<int, 3>> perms;
  std::array<int, 3> p = {0, 1, 2};
  do {
    perms.push_back(p);
  } while (std::next_permutation(p.begin(), p.begin() + d));
  const int64_t ncell = (d == 2) ? (int64_t)N * N : (int64_t)N * N * N;
  m.ne = ncell * (int64_t)perms.size();
  m.elems.resize(m.ne * (d + 1));
  int64_t T = 0;
  for (int64_t c = 0; c < ncell; ++c) {
    int64_t idx[3], t = c;
    for (int a = 0; a < d; ++a) {
      idx[a] = t % N;
      t /= N;
    }
    for (auto& pp : perms) {
      int64_t v[3] = {idx[0], idx[1], d == 3 ? idx[2] : 0};
      auto id = [&]() {
        int64_t r = 0, s = 1;
        for (int a = 0; a < d; ++a) {
          r += v[a] * s;
          s *= n1;
        }
        return (int32_t)r;
      };
      m.elems[T * (d + 1)] = id();
      for (int mm = 0; mm < d; ++mm) {
        v[pp[mm]] += 1;
        m.elems[T * (d + 1) + mm + 1] = id();
      }
      ++T;
    }
  }
  build_facets(m);
  return m;
}

std::vector<int32_t> colour_facets(const HostMesh& m, int* ncolours) {
  const int d = m.d;
  std::vector<int32_t> col(m.nint, -1);
  int nc = 0;
  for (int64_t r = 0; r < m.nint; ++r) {
    int32_t F = m.int_facets[r];
    uint64_t used = 0;
    std::vector<int> usedv;
    for (int side = 0; side < 2; ++side) {
      int32_t T = m.facet_elems[F * 2 + side];
      if (T < 0) continue;   // outflow facet: one element
      for (int f = 0; f <= d; ++f) {
        int32_t g = m.elem_rank[T * (d + 1) + f];
        if (g >= 0 && col[g] >= 0) {
          if (col[g] < 64) used |= (1ull << col[g]);
          else usedv.push_back(col[g]);
        }
      }
    }
    int c = 0;
    while (true) {
      bool u = (c < 64) ? ((used >> c) & 1ull) : (std::find(usedv.begin(), usedv.end(), c) != usedv.end());
      if (!u) break;
      ++c;
    }
    col[r] = c;
    nc = std::max(nc, c + 1);
  }
  *ncolours = nc;
  return col;
}

P1Space p1_space(const HostMesh& m) {
  P1Space p;
  const int d = m.d;
  p.vrank.assign(m.nv, -1);
  // a vertex is interior iff it lies on no boundary facet
  std::vector<char> bnd(m.nv, 0);
  for (int64_t F = 0; F < m.nf; ++F)
    if (m.int_rank[F] < 0)
      for (int a = 0; a < d; ++a) bnd[m.facets[F * d + a]] = 1;
  for (int64_t v = 0; v < m.nv; ++v)
    if (!bnd[v]) p.vrank[v] = (int32_t)p.n++;
  return p;
}

static Csr from_triplets(int64_t nr, int64_t nc, std::vector<std::array<int64_t, 2>>& ij, std::vector<double>& v) {
  std::vector<int64_t> order(ij.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return ij[a] < ij[b]; });
  Csr A;
  A.nrows = nr;
  A.ncols = nc;
  A.rowptr.assign(nr + 1, 0);
  int64_t last_r = -1, last_c = -1;
  for (int64_t t : order) {
    int64_t r = ij[t][0], c = ij[t][1];
    if (r == last_r && c == last_c) {
      A.val.back() += v[t];
    } else {
      A.col.push_back((int32_t)c);
      A.val.push_back(v[t]);
      A.rowptr[r + 1]++;
      last_r = r;
      last_c = c;
    }
  }
  for (int64_t r = 0; r < nr; ++r) A.rowptr[r + 1] += A.rowptr[r];
  return A;
}

Csr abar_matrix(const HostMesh& m, const P1Space& p, double nu, int k) {
  const int d = m.d;
  std::vector<std::array<int64_t, 2>> ij;
  std::vector<double> v;
  for (int64_t T = 0; T < m.ne; ++T) {
    const int32_t* e = &m.elems[T * (d + 1)];
    double J[9], Ji[9];
    for (int a = 0; a < d; ++a)
      for (int i = 0; i < d; ++i) J[a * d + i] = m.coords[e[i + 1] * d + a] - m.coords[e[0] * d + a];
    double det;
    if (d == 2) {
      det = J[0] * J[3] - J[1] * J[2];
      Ji[0] = J[3] / det; Ji[1] = -J[1] / det; Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
    } else {
      det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
      Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det; Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
      Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det; Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
      Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det; Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
      Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det; Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
      Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    }
    double vol = std::fabs(det) / (d == 2 ? 2.0 : 6.0);
    // gradients of barycentric coordinates: g_v = J^{-T} ghat_v
    double g[4][3];
    for (int vv = 0; vv <= d; ++vv)
      for (int a = 0; a < d; ++a) {
        double s = 0;
        for (int b = 0; b < d; ++b) {
          double gh = (vv == 0) ? -1.0 : (b == vv - 1 ? 1.0 : 0.0);
          s += Ji[b * d + a] * gh;
        }
        g[vv][a] = s;
      }
    for (int vi = 0; vi <= d; ++vi) {
      int32_t ri = p.vrank[e[vi]];
      if (ri < 0) continue;
      for (int vj = 0; vj <= d; ++vj) {
        int32_t rj = p.vrank[e[vj]];
        if (rj < 0) continue;
        double gg = 0;
        for (int a = 0; a < d; ++a) gg += g[vi][a] * g[vj][a];
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) {
            // eps(e_a lam_i) : eps(e_b lam_j) = (delta_ab g_i.g_j + g_i,b g_j,a) / 2
            double val = 0.5 * ((a == b ? gg : 0.0) + g[vi][b] * g[vj][a]);
            ij.push_back({(int64_t)ri * d + a, (int64_t)rj * d + b});
            v.push_back(nu * vol * val);
          }
      }
    }
  }
  // Lemma outflow: nu C k^2 / h_F int_F u_t . v_t on Gamma_Ntilde, with int_F lam_a lam_b =
  // |F| (1 + delta_ab) / (d (d + 1)) for the P1 hat functions of the facet's d vertices
  for (int64_t F = 0; F < (int64_t)m.outflow.size(); ++F) {
    if (!m.outflow[F]) continue;
    const int32_t* w = &m.facets[F * d];
    const double* n = &m.normals[F * d];
    double e[2][3] = {{0, 0, 0}, {0, 0, 0}}, hF = 0.0;
    for (int mm = 1; mm < d; ++mm)
      for (int a = 0; a < d; ++a) e[mm - 1][a] = m.coords[w[mm] * d + a] - m.coords[w[0] * d + a];
    for (int a = 0; a < d; ++a)
      for (int b = a + 1; b < d; ++b) {
        double l2 = 0;
        for (int c = 0; c < d; ++c) l2 += (m.coords[w[a] * d + c] - m.coords[w[b] * d + c]) *
                                          (m.coords[w[a] * d + c] - m.coords[w[b] * d + c]);
        hF = std::max(hF, std::sqrt(l2));
      }
    double meas;
    if (d == 2) {
      meas = std::sqrt(e[0][0] * e[0][0] + e[0][1] * e[0][1]);
    } else {
      const double cx = e[0][1] * e[1][2] - e[0][2] * e[1][1], cy = e[0][2] * e[1][0] - e[0][0] * e[1][2],
                   cz = e[0][0] * e[1][1] - e[0][1] * e[1][0];
      meas = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }
    const double c = nu * kOutflowC * k * k / hF;
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        const int32_t ra = p.vrank[w[a]], rb = p.vrank[w[b]];
        if (ra < 0 || rb < 0) continue;
        const double mab = meas * (a == b ? 2.0 : 1.0) / (d * (d + 1));
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j) {
            ij.push_back({(int64_t)ra * d + i, (int64_t)rb * d + j});
            v.push_back(c * mab * ((i == j ? 1.0 : 0.0) - n[i] * n[j]));
          }
      }
  }
  return from_triplets(p.n * d, p.n * d, ij, v);
}

Csr prolongation(int d, int Nc, const P1Space& pc, const P1Space& pf) {
  const int Nf = 2 * Nc;
  const int64_t nf1 = Nf + 1, nc1 = Nc + 1;
  std::vector<std::array<int64_t, 2>> ij;
  std::vector<double> v;
  const int64_t nvf = (d == 2) ? nf1 * nf1 : nf1 * nf1 * nf1;
  for (int64_t vid = 0; vid < nvf; ++vid) {
    int32_t rf = pf.vrank[vid];
    if (rf < 0) continue;
    int64_t I[3], t = vid;
    for (int a = 0; a < d; ++a) {
      I[a] = t % nf1;
      t /= nf1;
    }
    int64_t A[3], B[3];
    bool odd = false;
    for (int a = 0; a < d; ++a) {
      int64_t o = I[a] % 2;
      odd = odd || o;
      A[a] = (I[a] - o) / 2;
      B[a] = (I[a] + o) / 2;
    }
    int nends = odd ? 2 : 1;
    for (int e = 0; e < nends; ++e) {
      const int64_t* P = e == 0 ? A : B;
      int64_t cid = 0, s = 1;
      for (int a = 0; a < d; ++a) {
        cid += P[a] * s;
        s *= nc1;
      }
      int32_t rc = pc.vrank[cid];
      if (rc < 0) continue;
      for (int c = 0; c < d; ++c) {
        ij.push_back({(int64_t)rf * d + c, (int64_t)rc * d + c});
        v.push_back(1.0 / nends);
      }
    }
  }
  return from_triplets(pf.n * d, pc.n * d, ij, v);
}

Csr transpose(const Csr& A) {
  std::vector<std::array<int64_t, 2>> ij;
  std::vector<double> v;
  for (int64_t r = 0; r < A.nrows; ++r)
    for (int64_t t = A.rowptr[r]; t < A.rowptr[r + 1]; ++t) {
      ij.push_back({(int64_t)A.col[t], r});
      v.push_back(A.val[t]);
    }
  return from_triplets(A.ncols, A.nrows, ij, v);
}

std::vector<double> embedding_blocks(const HostMesh& m, const RefTables& T) {
  const int d = m.d;
  const Sizes& s = T.s;
  std::vector<double> out((size_t)m.nint * s.mF * d * d, 0.0);
  for (int64_t r = 0; r < m.nint; ++r) {
    int32_t F = m.int_facets[r];
    const int32_t* w = &m.facets[F * d];
    double e[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (int mm = 1; mm < d; ++mm)
      for (int a = 0; a < d; ++a) e[mm - 1][a] = m.coords[w[mm] * d + a] - m.coords[w[0] * d + a];
    // facet measure and dual tangents e^m = sum_l (G_F^{-1})_{ml} e_l
    double G[2][2] = {{0, 0}, {0, 0}};
    for (int i = 0; i < d - 1; ++i)
      for (int j = 0; j < d - 1; ++j)
        for (int a = 0; a < d; ++a) G[i][j] += e[i][a] * e[j][a];
    double meas, Gi[2][2];
    if (d == 2) {
      meas = std::sqrt(G[0][0]);
      Gi[0][0] = 1.0 / G[0][0];
    } else {
      double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
      meas = std::sqrt(det) / 2.0;
      Gi[0][0] = G[1][1] / det; Gi[1][1] = G[0][0] / det;
      Gi[0][1] = -G[0][1] / det; Gi[1][0] = -G[1][0] / det;
    }
    double ed[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < d - 1; ++i)
      for (int l = 0; l < d - 1; ++l)
        for (int a = 0; a < d; ++a) ed[i][a] += Gi[i][l] * e[l][a];
    double* B = &out[(size_t)r * s.mF * d * d];
    const double* n = &m.normals[F * d];
    for (int wv = 0; wv < d; ++wv)
      for (int a = 0; a < d; ++a) {
        int col = wv * d + a;
        for (int j = 0; j < s.nF; ++j) B[j * d * d + col] = n[a] * meas / T.facet_ref_measure * T.Ilam[wv * s.nF + j];
        const bool out = !m.outflow.empty() && m.outflow[F];   // pi_0 of Lemma outflow: no uhat rows
        for (int mm = 0; mm < d - 1 && !out; ++mm)
          for (int j = 0; j < s.nFm1; ++j)
            B[(s.nF + mm * s.nFm1 + j) * d * d + col] = ed[mm][a] * T.Ilam[wv * s.nF + j];
        if (s.lowest) {
          // k = 1 (Sec. 7): third component curl(ubar), as its flux through F along n_F.  By Stokes'
          // theorem int_F curl(lambda_w e_a).n_F is the circulation of lambda_w e_a around the facet
          // boundary w_0 -> w_1 -> w_2 (counter-clockwise about n_F = e_1 x e_2 / |e_1 x e_2|): with
          // lambda_w linear on the edges it is (x_{w+1} - x_{w-1})_a / 2, indices mod 3.
          const int wn = w[(wv + 1) % 3], wp = w[(wv + 2) % 3];
          B[(s.nF + s.ntF) * d * d + col] = 0.5 * (m.coords[wn * d + a] - m.coords[wp * d + a]);
        }
      }
  }
  return out;
}

}  // namespace mcs
