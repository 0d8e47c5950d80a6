"""The forward facet sweep with a maintained residual is the block Gauss-Seidel sweep of Corollary
aux_pc_mult written in another order of summation.

The row-product form updates facet F of colour c by x_F += D_F^{-1} (b - A^d x)_F.  The maintained-residual
form keeps, for every element T, q_T = -A^d_T x_T restricted to T's coupling dofs; a facet's residual is
b_F plus the q_T entries of its two elements at F's dofs, and after the block solve the update delta_F is
pushed into q_T of both elements (q_T -= A^d_T[:, F] delta_F).  Starting from x = 0 (q = 0) both forms give
the same x after every colour, and b + sum_T q_T is the residual b - A^d x the coarse correction needs.
The check runs on the oracle's element matrices A^d_T (FP64, CPU), independent of the library."""
import numpy as np
import pytest

from oracle import mesh, precond, system


def _setup(d, N, k, nu):
    D = system.discretize(mesh.structured(d, N), k, nu)
    AT = system.condense(D)
    asp = precond.ASP(D, AT, precond.GMG(d, N, 1, nu))
    return D, asp


def _facet_positions(asp):
    """For every interior facet: [(element, local coupling positions of the facet's dofs)] over its
    two elements."""
    where = {}
    for T, row in enumerate(asp.cmap):
        for pos, g in enumerate(row):
            if g >= 0:
                where.setdefault(int(g), []).append((T, pos))
    out = []
    for fd in asp.fdofs:
        per_elem = {}
        for g in fd:
            for T, pos in where[int(g)]:
                per_elem.setdefault(T, []).append(pos)
        out.append([(T, np.array(p)) for T, p in sorted(per_elem.items())])
    return out


def _push_sweeps(asp, b, sweeps):
    ne, nc = asp.cmap.shape
    q = np.zeros((ne, nc))
    x = np.zeros_like(b)
    fpos = _facet_positions(asp)
    for _ in range(sweeps):
        for c in range(asp.ncol):
            for i in np.nonzero(asp.colour == c)[0]:
                fd = asp.fdofs[i]
                r = b[fd].copy()
                for T, p in fpos[i]:
                    r += q[T, p]
                delta = asp.Dinv[i] @ r
                x[fd] += delta
                for T, p in fpos[i]:
                    q[T] -= asp.Ad[T][:, p] @ delta
    res = b.copy()
    for T in range(ne):
        ok = asp.cmap[T] >= 0
        np.add.at(res, asp.cmap[T][ok], q[T][ok])
    return x, res


@pytest.mark.parametrize("d,N,k,nu,sweeps", [(3, 2, 2, 0.7, 2), (2, 4, 3, 1.0, 1), (2, 3, 4, 0.3, 2)])
def test_push_form_equals_row_products(d, N, k, nu, sweeps):
    D, asp = _setup(d, N, k, nu)
    b = np.zeros(D.ndof)
    rng = np.random.default_rng(7)
    cd = np.concatenate([np.arange(D.n_dd), D.off_h + np.arange(D.n_hat)])
    b[cd] = rng.standard_normal(len(cd))
    x_rows = np.zeros_like(b)
    for _ in range(sweeps):
        x_rows = asp._sweep(x_rows, b, range(asp.ncol))
    r_rows = b - asp.Ad_glob @ x_rows
    x_push, r_push = _push_sweeps(asp, b, sweeps)
    assert np.abs(x_push - x_rows).max() <= 1e-12 * np.abs(x_rows).max()
    assert np.abs(r_push[cd] - r_rows[cd]).max() <= 1e-12 * np.abs(b).max()


def test_push_form_catches_a_dropped_own_slot():
    """Mutation: leaving out the facet's own elements' diagonal blocks when pushing breaks the identity."""
    D, asp = _setup(3, 2, 2, 1.0)
    b = np.zeros(D.ndof)
    cd = np.concatenate([np.arange(D.n_dd), D.off_h + np.arange(D.n_hat)])
    b[cd] = np.random.default_rng(8).standard_normal(len(cd))
    x_rows = np.zeros_like(b)
    for _ in range(2):   # the own slot is read again in the second sweep
        x_rows = asp._sweep(x_rows, b, range(asp.ncol))
    ne, nc = asp.cmap.shape
    q = np.zeros((ne, nc))
    x = np.zeros_like(b)
    fpos = _facet_positions(asp)
    for c in list(range(asp.ncol)) * 2:
        for i in np.nonzero(asp.colour == c)[0]:
            fd = asp.fdofs[i]
            r = b[fd].copy()
            for T, p in fpos[i]:
                r += q[T, p]
            delta = asp.Dinv[i] @ r
            x[fd] += delta
            for T, p in fpos[i]:
                upd = asp.Ad[T][:, p] @ delta
                upd[p] = 0.0            # the planted mistake: the facet's own rows are not updated
                q[T] -= upd
    assert np.abs(x - x_rows).max() > 1e-6 * np.abs(x_rows).max()
