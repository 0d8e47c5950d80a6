"""CPU parity of the library's host-compiled code against the oracle (no GPU).

The element condensation (csrc/element.cuh, the same source the CUDA kernels run with a warp or a
block of lanes) is compiled here with g++ for a single lane, together with the host set-up code
(csrc/reference.cpp, csrc/meshing.cpp: reference tables, numbering with an outflow face, the
conforming operator with its penalty and the E^d blocks), and compared with the oracle element by
element.  This checks the arithmetic of the element algorithm and of the host tables on every CPU
run; the GPU tests check the same quantities through the C-ABI."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fem, mesh, precond, system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2207_08481_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "reference.h"
#include "meshing.h"
#include "element.cuh"
using namespace mcs;

static ElemSizes sizes_of(const Sizes& s, int lo_stab) {
  ElemSizes e;
  e.d = s.d; e.k = s.k; e.nk = s.nk; e.nF = s.nF; e.nFm1 = s.nFm1; e.n_u = s.n_u; e.n_A = s.n_A;
  e.n_hat = s.n_hat; e.nhF = s.nhF; e.n_p = s.n_p; e.n_s0 = s.n_s0; e.n_raw = s.n_raw; e.n_con = s.n_con;
  e.n_w = s.n_w; e.n_wskew = s.n_wskew; e.n_cc = s.n_cc; e.n_bub = s.n_bub; e.n_c = s.n_c; e.mF = s.mF;
  e.ntF = s.ntF; e.lowest = s.lowest; e.lo_stab = lo_stab;
  return e;
}

int main(int argc, char** argv) {
  const char* mode = argv[1];
  const int d = atoi(argv[2]), k = atoi(argv[3]);
  if (!strcmp(mode, "condense")) {
    // stdin: nu lo_stab, then per element (d+1)*d coordinates and d+1 signs
    double nu; int lo;
    if (scanf("%lf %d", &nu, &lo) != 2) return 1;
    RefTables R = build_reference(d, k);
    ElemSizes e = sizes_of(R.s, lo);
    ElemTables t{R.B0.data(), R.Rf.data(), R.Bh.data(), R.Ccon.data(), R.Adiv.data(), R.nhat.data(),
                 R.Wmom.data()};
    std::vector<double> ws(elem_work_doubles(e));
    double X[12];
    int sg[4];
    while (true) {
      for (int i = 0; i < (d + 1) * d; ++i)
        if (scanf("%lf", &X[i]) != 1) return 0;
      for (int i = 0; i <= d; ++i)
        if (scanf("%d", &sg[i]) != 1) return 1;
      ElemWork w = elem_work_carve(e, ws.data());
      condense_element(e, t, X, sg, nu, w, 0, 1, []() {});
      for (int i = 0; i < e.n_A * e.n_A; ++i) printf("%.17g\n", w.A[i]);
      // bubble condensation (eqs. Hcoeffs, factorSsigma): A^d (coupling order), G, A_oo^{-1}
      const int no = e.n_bub, nc = e.n_c;
      std::vector<double> bw(no * no + no * nc + 1), Ad(nc * nc), G(no * nc + 1), Ai(no * no + 1);
      bubble_condense(e, w.A, bw.data(), Ad.data(), G.data(), Ai.data(), 0, 1, []() {});
      for (int i = 0; i < nc * nc; ++i) printf("%.17g\n", Ad[i]);
      for (int i = 0; i < no * nc; ++i) printf("%.17g\n", G[i]);
    }
  }
  if (!strcmp(mode, "recover")) {
    // stdin: nu nq, nq reference points, then per element: coordinates, signs, n_A local coefficients
    double nu; int nq;
    if (scanf("%lf %d", &nu, &nq) != 2) return 1;
    RefTables R = build_reference(d, k);
    ElemSizes e = sizes_of(R.s, 0);
    ElemTables t{R.B0.data(), R.Rf.data(), R.Bh.data(), R.Ccon.data(), R.Adiv.data(), R.nhat.data(),
                 R.Wmom.data()};
    std::vector<double> xh(nq * d), psi(nq * e.nk);
    for (int i = 0; i < nq * d; ++i)
      if (scanf("%lf", &xh[i]) != 1) return 1;
    for (int q = 0; q < nq; ++q) dubiner_eval(d, k, &xh[q * d], &psi[q * e.nk], nullptr);
    std::vector<double> ws(elem_work_doubles(e)), a(e.n_A), wk(e.n_cc + 2 * e.n_raw), sig(nq * d * d),
        om(nq * d * d);
    double X[12];
    int sg[4];
    while (true) {
      for (int i = 0; i < (d + 1) * d; ++i)
        if (scanf("%lf", &X[i]) != 1) return 0;
      for (int i = 0; i <= d; ++i)
        if (scanf("%d", &sg[i]) != 1) return 1;
      for (int i = 0; i < e.n_A; ++i)
        if (scanf("%lf", &a[i]) != 1) return 1;
      ElemWork w = elem_work_carve(e, ws.data());
      condense_element(e, t, X, sg, nu, w, 0, 1, []() {});
      recover_element(e, w, X, a.data(), nq, psi.data(), wk.data(), sig.data(), e.lowest ? nullptr : om.data(), 0, 1,
                      []() {});
      for (int i = 0; i < nq * d * d; ++i) printf("%.17g\n", sig[i]);
      for (int i = 0; i < nq * d * d; ++i) printf("%.17g\n", e.lowest ? 0.0 : om[i]);
    }
  }
  if (!strcmp(mode, "loadrule")) {
    RefTables R = build_reference(d, k);
    for (int q = 0; q < R.nq_load; ++q) {
      for (int a = 0; a < d; ++a) printf("%.17g ", R.xq_load[q * d + a]);
      printf("%.17g\n", R.wq_load[q]);
    }
    return 0;
  }
  // "mesh": structured N, optional outflow face; numbering, Abar (nu = 0.7) and E^d blocks
  const int N = atoi(argv[4]), outflow = atoi(argv[5]);
  HostMesh m = structured_mesh(d, N);
  if (outflow) mark_outflow(m);
  RefTables R = build_reference(d, k);
  const Sizes& s = R.s;
  for (int64_t r = 0; r < m.nint; ++r) printf("CF %d\n", m.int_facets[r]);
  int ncol = 0;
  std::vector<int32_t> col = colour_facets(m, &ncol);
  for (int64_t r = 0; r < m.nint; ++r) printf("CL %d\n", col[r]);
  P1Space p = p1_space(m);
  for (int64_t v = 0; v < m.nv; ++v) printf("VR %d\n", p.vrank[v]);
  Csr A = abar_matrix(m, p, 0.7, k);
  for (int64_t r = 0; r < A.nrows; ++r)
    for (int64_t q = A.rowptr[r]; q < A.rowptr[r + 1]; ++q) printf("A %ld %d %.17g\n", (long)r, A.col[q], A.val[q]);
  std::vector<double> B = embedding_blocks(m, R);
  for (int64_t r = 0; r < m.nint; ++r) {
    const int F = m.int_facets[r];
    for (int tt = 0; tt < s.mF; ++tt)
      for (int w = 0; w < d; ++w)
        for (int a = 0; a < d; ++a)
          printf("E %ld %d %d %d %.17g\n", (long)r, tt, m.facets[F * d + w], a, B[((size_t)r * s.mF + tt) * d * d + w * d + a]);
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("host")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    cmd = [cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "reference.cpp"),
           os.path.join(CSRC, "meshing.cpp"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return str(exe)


def _perturbed(d, N, seed=1):
    m = mesh.structured(d, N)
    c = m.coords.copy()
    inner = np.all((c > 1e-12) & (c < 1 - 1e-12), axis=1)
    c[inner] += 0.15 / N * np.random.default_rng(seed).uniform(-1, 1, size=(inner.sum(), d))
    return mesh.structured(d, N, coords=c)


@pytest.mark.parametrize("d,k,N,lo", [(2, 2, 3, 0), (2, 3, 2, 0), (2, 4, 1, 0), (3, 2, 1, 0), (3, 1, 2, 0),
                                      (3, 1, 2, 1), (2, 5, 1, 0), (2, 6, 1, 0), (3, 5, 1, 0), (3, 6, 1, 0)])
def test_element_condensation_matches_oracle(harness, d, k, N, lo):
    """A_T of every element of a perturbed mesh (orientation signs applied), 1e-12 relative; the double
    Schur complement A^d_T and G_T = A_oo^{-1} A_od (eqs. Hcoeffs, factorSsigma) to 1e-11 / 1e-10."""
    nu = 0.7
    m = _perturbed(d, N)
    D = system.discretize(m, k, nu, lo_stab=lo)
    AT = system.condense(D)
    X = m.coords[m.elems]
    lines = [f"{nu!r} {lo}"] + [" ".join("%.17g" % v for v in X[e].ravel()) + " " + " ".join(map(str, m.signs[e]))
                                for e in range(X.shape[0])]
    out = subprocess.run([harness, "condense", str(d), str(k)], input="\n".join(lines), capture_output=True,
                         text=True, check=True).stdout
    sz = D.sz
    ne, nA = AT.shape[0], AT.shape[1]
    nc, no = (d + 1) * (sz["nF"] + sz["n_hatF"]), sz["n_bub"]
    vals = np.array(out.split(), dtype=float).reshape(ne, nA * nA + nc * nc + no * nc)
    A = vals[:, :nA * nA].reshape(AT.shape)
    err = np.abs(A - AT).max(axis=(1, 2)) / np.abs(AT).max(axis=(1, 2))
    assert err.max() < (1e-12 if k <= 4 else 1e-10), err.max()   # rounding grows with the local sizes (3D k = 6: 3.5e-11)
    # A^d and G in the library's facet-major coupling order against the oracle's [u_d | uhat] order
    Ad_o, G_o, _ = system.bubble_condense(D, AT)
    mF = sz["nF"] + sz["n_hatF"]
    perm = [f * sz["nF"] + t if t < sz["nF"] else (d + 1) * sz["nF"] + f * sz["n_hatF"] + (t - sz["nF"])
            for f in range(d + 1) for t in range(mF)]
    Ad = vals[:, nA * nA:nA * nA + nc * nc].reshape(ne, nc, nc)
    assert np.abs(Ad - Ad_o[:, perm][:, :, perm]).max() < 1e-11 * np.abs(Ad_o).max()
    if no:
        G = vals[:, nA * nA + nc * nc:].reshape(ne, no, nc)
        assert np.abs(G - G_o[:, :, perm]).max() < 1e-10 * np.abs(G_o).max()


@pytest.mark.parametrize("d,k,N,outflow", [(2, 2, 4, 0), (2, 3, 4, 1), (3, 1, 2, 0), (3, 2, 2, 1)])
def test_numbering_abar_and_embedding_match_oracle(harness, d, k, N, outflow):
    """Coupling facets (interior, plus the outflow face) and their colouring, free P1 vertices, Abar with the tangential
    penalty of Lemma outflow, and the E^d blocks (uhat rows by L2 projection, zero on the outflow face;
    the curl rows for k = 1) against the oracle's assembled operators."""
    m = mesh.structured(d, N)
    if outflow:
        m = mesh.with_outflow(m)
    D = system.discretize(m, k, 0.7)
    out = subprocess.run([harness, "mesh", str(d), str(k), str(N), str(outflow)], capture_output=True, text=True,
                         check=True).stdout.splitlines()
    udof = np.nonzero(m.udof)[0]
    assert [int(l.split()[1]) for l in out if l.startswith("CF ")] == list(udof)
    col = np.array([int(l.split()[1]) for l in out if l.startswith("CL ")])
    assert np.array_equal(col, mesh.colouring(m))            # greedy colouring of the coupling facets
    for c in range(col.max() + 1):                           # one colour: no two facets share an element
        els = m.facet_elems[udof[col == c]].ravel()
        els = els[els >= 0]
        assert len(els) == len(np.unique(els))
    rank, _ = precond.p1_map(m)
    assert np.array_equal(np.array([int(l.split()[1]) for l in out if l.startswith("VR ")]), rank)
    Ao = precond.abar(m, 0.7, k).toarray()
    Ah = np.zeros_like(Ao)
    for l in out:
        if l.startswith("A "):
            _, r, c, v = l.split()
            Ah[int(r), int(c)] += float(v)
    assert np.abs(Ah - Ao).max() < 1e-13 * np.abs(Ao).max()
    E = precond.embedding(D).tocsr()
    nF, nhF = D.sz["nF"], D.sz["n_hatF"]
    err, seen = 0.0, 0
    for l in out:
        if not l.startswith("E "):
            continue
        _, r, t, vid, a, v = l.split()
        r, t, vid, a, v = int(r), int(t), int(vid), int(a), float(v)
        if rank[vid] < 0:
            continue
        ri = m.int_rank[udof[r]]
        row = r * nF + t if t < nF else (D.off_h + ri * nhF + (t - nF) if ri >= 0 else None)
        ref = E[row, rank[vid] * d + a] if row is not None else 0.0
        err = max(err, abs(ref - v))
        seen += 1
    assert seen > 0 and err < 1e-13 * abs(E).max()


@pytest.mark.parametrize("d,k,N", [(2, 3, 2), (3, 2, 1), (3, 1, 2)])
def test_stress_recovery_matches_oracle(harness, d, k, N):
    """Local solves of eq. (projection) for a random coefficient vector: sigma_h (and omega_h for
    k >= 2) at the oracle's quadrature points, from the element code against the oracle's solves."""
    nu = 0.9
    m = _perturbed(d, N, seed=4)
    D = system.discretize(m, k, nu)
    x = np.random.default_rng(8).standard_normal(D.ndof)
    sig, om = system.recover_stress(D, x)
    X = m.coords[m.elems]
    E = fem.element_data(X, m.signs, k)
    so = np.einsum("ej,eqjab->eqab", sig, E.S)
    # local coefficients with the orientation signs removed (facet BDM dofs; rotation fluxes for k = 1)
    sz = D.sz
    am = D.a_map
    a = np.where(am >= 0, x[np.maximum(am, 0)], 0.0)
    nfd = (d + 1) * sz["nF"]
    a[:, :nfd] *= np.repeat(m.signs, sz["nF"], axis=1)
    if sz["lowest"]:
        a[:, sz["n_u"] + 2::3] *= m.signs
    J0 = (X[0, 1:, :] - X[0, :1, :]).T
    xhat = np.linalg.solve(J0, (E.xq[0] - X[0, 0]).T).T
    nq = xhat.shape[0]
    lines = [f"{nu!r} {nq}", " ".join("%.17g" % v for v in xhat.ravel())]
    lines += [" ".join("%.17g" % v for v in X[e].ravel()) + " " + " ".join(map(str, m.signs[e])) + " " +
              " ".join("%.17g" % v for v in a[e]) for e in range(X.shape[0])]
    out = subprocess.run([harness, "recover", str(d), str(k)], input="\n".join(lines), capture_output=True,
                         text=True, check=True).stdout
    vals = np.array(out.split(), dtype=float).reshape(X.shape[0], 2, nq, d, d)
    assert np.abs(vals[:, 0] - so).max() < 1e-11 * np.abs(so).max()
    if not sz["lowest"]:
        wo = np.einsum("ej,eqjab->eqab", om, E.W)
        assert np.abs(vals[:, 1] - wo).max() < 1e-10 * np.abs(wo).max()


@pytest.mark.parametrize("d,k", [(2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3), (3, 4)])
def test_load_rule_is_the_oracle_rule(harness, d, k):
    """The load quadrature of the dof contract (collapsed Gauss-Jacobi, k + 8 points per direction) is
    implemented on both sides independently: the library's points and weights equal the oracle's
    (SciPy Gauss-Jacobi nodes) to rounding, so both load vectors agree to rounding too."""
    from oracle import polys
    out = subprocess.run([harness, "loadrule", str(d), str(k), "0", "0"], capture_output=True, text=True,
                         check=True).stdout
    got = np.array(out.split(), dtype=float).reshape(-1, d + 1)
    x, w = polys.quadrature(d, k + 8)
    assert got.shape[0] == len(w)
    assert np.abs(got[:, :d] - x).max() < 1e-14
    assert np.abs(got[:, d] - w).max() < 1e-15 * max(1.0, np.abs(w).max()) * 10
