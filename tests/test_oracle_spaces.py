"""Oracle pins: dimensions and defining properties of the spaces of Sec. 3."""
import os

import numpy as np
import pytest

from oracle import fem, mesh, polys

HERE = os.path.dirname(os.path.abspath(__file__))


def test_local_dimensions_match_space_definitions():
    # (d, k): n_sigma, n_omega, n_u (facet+bubble), n_hat, n_p
    table = {(2, 2): (15, 3, 12, 9, 6, 3), (2, 3): (27, 6, 20, 12, 9, 6),
             (3, 2): (56, 12, 30, 24, 24, 4), (3, 3): (128, 30, 60, 40, 48, 10),
             (3, 4): (240, 60, 105, 60, 80, 20), (3, 5): (400, 105, 168, 84, 120, 35),
             (3, 6): (616, 168, 252, 112, 168, 56)}
    for (d, k), (ns, nw, nu, ndd, nh, npp) in table.items():
        s = fem.local_sizes(d, k)
        assert (s["n_sigma"], s["n_omega"], s["n_u"], s["n_dd"], s["n_hat"], s["n_p"]) == (ns, nw, nu, ndd, nh, npp)


def test_paper_table_st_ws_dof_counts():
    """#D of Table ST_ws for k = 1, 2, 4 on one mesh must follow from one facet count."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table_st_ws_dims.txt"))
            if l.strip() and not l.startswith("#")]
    by = {}
    for k, T, D in rows:
        by.setdefault(int(T), {})[int(k)] = int(D)
    s2, s4 = fem.local_sizes(3, 2), fem.local_sizes(3, 4)
    for T, dd in by.items():
        per_f2 = s2["nF"] + s2["n_hatF"]
        F, rem = divmod(dd[2] - (s2["n_bub"] + s2["n_p"]) * T, per_f2)
        assert rem == 0
        # k = 1 (Sec. 6): BDM^1 3 + Vhat (P^0 tangential) 2 + W (one H(div) dof) 1 per facet, p: 1 per element
        assert 6 * F + T == dd[1]
        if 4 in dd:
            assert (s4["nF"] + s4["n_hatF"]) * F + (s4["n_bub"] + s4["n_p"]) * T == dd[4]


def test_mesh_counts():
    m = mesh.structured(2, 8)
    assert (len(m.elems), len(m.facets), m.n_int) == (128, 208, 176)
    m = mesh.structured(3, 4)
    assert len(m.elems) == 384
    # Euler-type count: each element has d+1 facets, interior shared by 2
    assert 2 * m.n_int + (len(m.facets) - m.n_int) == 4 * len(m.elems)


@pytest.mark.parametrize("d,k", [(2, 2), (2, 3), (3, 2)])
def test_bdm_basis_traces_and_continuity(d, k):
    m = mesh.structured(d, 2)
    X = m.coords[m.elems]
    D = fem.element_data(X, m.signs, k)
    s = fem.local_sizes(d, k)
    nF = s["nF"]
    for f in range(d + 1):
        un = np.einsum("eqia,ea->eqi", D.fU[:, f], D.fn[:, f])
        for g in range(d + 1):
            cols = np.arange(g * nF, (g + 1) * nF)
            if g != f:   # facet functions of other facets: zero normal trace on f
                assert np.abs(un[:, :, cols]).max() < 1e-11
        assert np.abs(un[:, :, (d + 1) * nF:]).max() < 1e-11   # bubbles
    # normal continuity of the global facet functions: same u.n_F from both elements
    for F in np.nonzero(m.interior)[0]:
        vals = []
        for T in m.facet_elems[F]:
            f = int(np.nonzero(m.elem_facets[T] == F)[0][0])
            un = np.einsum("qia,a->qi", D.fU[T, f][:, f * nF:(f + 1) * nF], m.normals[F])
            # quadrature points of local facet f follow the sorted facet vertices on both sides
            vals.append(un)
        assert np.allclose(vals[0], vals[1], atol=1e-10)
        # dual property: moment of mode j against q_i is delta_ij
        sq, ws = polys.quadrature(d - 1, k + 2)
        q = polys.dubiner(d - 1, k, sq)[0]
        T = m.facet_elems[F][0]
        f = int(np.nonzero(m.elem_facets[T] == F)[0][0])
        mom = np.einsum("q,qi,qj->ij", D.fw[T, f], vals[0], q)
        assert np.allclose(mom, np.eye(nF), atol=1e-11)


@pytest.mark.parametrize("d,k", [(2, 2), (2, 3), (3, 2)])
def test_sigma_space(d, k):
    m = mesh.structured(d, 1)
    X = m.coords[m.elems]
    D = fem.element_data(X, m.signs, k)
    tr = np.einsum("eqsaa->eqs", D.S)
    assert np.abs(tr).max() < 1e-12
    # nt trace has no degree-k part on any facet
    sq, ws = polys.quadrature(d - 1, k + 2)
    q = polys.dubiner(d - 1, k, sq)[0]
    top = polys.degrees(d - 1, k) == k
    for f in range(d + 1):
        Sn = np.einsum("eqsab,eb->eqsa", D.fS[:, f], D.fn[:, f])
        Snn = np.einsum("eqsa,ea->eqs", Sn, D.fn[:, f])
        Snt = Sn - Snn[..., None] * D.fn[:, f][:, None, None, :]
        mom = np.einsum("eq,qj,eqsa->ejsa", D.fw[:, f], q[:, top], Snt)
        assert np.abs(mom).max() < 1e-11
