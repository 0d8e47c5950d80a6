"""CPU FP64 oracle for the mass-conserving mixed-stress (MCS) Stokes method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import anything
from this package.  The product path (the ``libmcs`` C-ABI library and its
Python binding) never imports, links or executes it, and it shares no code,
tables or constants with that path.

The oracle is a plain, slow, literal restatement of arXiv 2207.08481:

* ``polys``         reference-simplex polynomials and quadrature (library
                    Gauss-Jacobi rules from SciPy).
* ``mesh``          structured simplicial meshes, facets, orientation, the dof
                    numbering contract and the facet colouring.
* ``fem``           the spaces of Sec. 3, eqs. (fes_V)-(fes_Vbar), and the
                    element matrices of eq. (bigfemSPmat), computed by physical
                    quadrature of the printed bilinear forms.
* ``system``        global assembly of the uncondensed saddle-point system and
                    its direct solve; the condensed system of eq. (femSPmat)
                    and the bubble ("double Schur") condensation, Sec. 4.2.
* ``precond``       the conforming auxiliary space (eq. defAhat, eq. defE,
                    eq. defED), the geometric multigrid V-cycle used as C, the
                    facet-block Gauss-Seidel smoother, the multiplicative ASP of
                    Sec. 5.2 and the block preconditioner of eq. (mhatinvfactor).
* ``krylov``        textbook preconditioned MinRes, and GMRES (the paper's solver) for comparison.
* ``hdg``           the HDG norm eq. (nhdg_eps) on one element and the constant gamma of
                    Corollary schur_SPD (the single-element experiment the paper mentions).
* ``manufactured``  manufactured solutions and their right-hand sides (one with the outflow
                    condition of eq. (stokes_NT) on x = 1).

Outflow: ``mesh.with_outflow`` marks the face x_1 = 1 as Gamma_Ntilde; ``system`` then keeps BDM
dofs but no uhat on it and imposes no pressure mean, and ``precond`` adds the tangential penalty of
Lemma outflow to Abar and frees the conforming space on that face.
"""
