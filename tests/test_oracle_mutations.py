"""The oracle's pins catch plausible mistakes: each test plants one in the oracle (CPU only)."""
import numpy as np
import pytest

from oracle import fem, manufactured, mesh, precond, system


def _embedding_defect(d=2, k=2, N=4, nu=0.7):
    m = mesh.structured(d, N)
    D = system.discretize(m, k, nu)
    A = system.condensed_system(D, system.condense(D))
    E = precond.embedding(D)
    Ab = precond.abar(m, nu).toarray()
    return np.abs((E.T @ A @ E).toarray() - Ab).max() / np.abs(Ab).max()


def _pressure_defect():
    m = mesh.structured(2, 4)
    D = system.discretize(m, 2, 0.3)
    phi = lambda x: x[..., 0] * x[..., 1] ** 2
    gphi = lambda x: np.stack([x[..., 1] ** 2, 2 * x[..., 0] * x[..., 1]], -1)
    x = system.mean_zero_pressure(D, system.solve_condensed(D, system.load(D, gphi)))
    X = m.coords[m.elems]
    Dd = fem.element_data(X, m.signs, 2, q=6)
    y = np.zeros(D.ndof)
    y[D.p_map] = np.einsum("eq,eq,eqi->ei", Dd.wq, phi(Dd.xq), Dd.P) / np.abs(Dd.detJ)[:, None]
    y = system.mean_zero_pressure(D, y)
    n = D.off_p
    return np.abs(x[n:] - y[n:]).max() / np.abs(y[n:]).max()


def _corrupt(monkeypatch, key, fn):
    orig = fem.element_matrices

    def bad(*a, **kw):
        out = orig(*a, **kw)
        out[key] = fn(out[key])
        return out
    monkeypatch.setattr(fem, "element_matrices", bad)


def test_unmutated_pins_pass():
    assert _embedding_defect() < 1e-12
    assert _pressure_defect() < 1e-10


@pytest.mark.parametrize("key,fn", [
    ("Bh", lambda B: -B),                       # sign of the nt coupling
    ("Adiv", lambda A: 2.0 * A),                # dropped 1/d
    ("M", lambda M: 1.1 * M),                   # wrong nu scaling of the stress mass
])
def test_embedding_pin_catches(monkeypatch, key, fn):
    _corrupt(monkeypatch, key, fn)
    assert _embedding_defect() > 1e-6


def test_dropped_boundary_term_is_caught(monkeypatch):
    """Bu without -(sigma_nn, u_n)_dT."""
    orig = fem.element_matrices

    def bad(X, signs, k, nu, *rest):
        out = orig(X, signs, k, nu, *rest)
        D = fem.element_data(X, signs, k)
        out["Bu"] = np.einsum("eq,eqja,eqia->eij", D.wq, D.divS, D.U)
        return out
    monkeypatch.setattr(fem, "element_matrices", bad)
    assert _embedding_defect() > 1e-6


def test_pressure_sign_is_caught(monkeypatch):
    _corrupt(monkeypatch, "Bp", lambda B: -B)
    assert _pressure_defect() > 1e-3


def test_abar_scale_is_caught(monkeypatch):
    """eq. (defAhat) as printed (nu^{-1}) contradicts Corollary embed unless nu = 1 (reading R1)."""
    orig = precond.abar
    monkeypatch.setattr(precond, "abar", lambda m, nu: orig(m, 1.0 / nu))
    assert _embedding_defect(nu=0.7) > 1e-3


def test_orientation_sign_is_caught(monkeypatch):
    orig = mesh.build

    def bad(*a):
        m = orig(*a)
        m.signs[:] = 1
        return m
    monkeypatch.setattr(mesh, "build", bad)
    m = mesh.structured(2, 4)
    D = system.discretize(m, 2, 1.0)
    ms = manufactured.Manufactured(2, 1.0)
    x = system.mean_zero_pressure(D, system.solve_condensed(D, system.load(D, ms.f)))
    X = m.coords[m.elems]
    Dd = fem.element_data(X, m.signs, 2, q=6)
    xu = np.where(D.u_map >= 0, x[np.maximum(D.u_map, 0)], 0.0)
    uh = np.einsum("eqia,ei->eqa", Dd.U, xu)
    err = np.sqrt(np.sum(Dd.wq * np.sum((uh - ms.u(Dd.xq)) ** 2, -1)))
    norm = np.sqrt(np.sum(Dd.wq * np.sum(ms.u(Dd.xq) ** 2, -1)))
    assert err > 0.1 * norm
