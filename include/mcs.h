/*
 * libmcs — GB300-native hot path of the mass-conserving mixed-stress (MCS)
 * Stokes method of arXiv 2207.08481 ("A conforming auxiliary space
 * preconditioner for the mass conserving mixed stress method").
 *
 * The library performs the two data-parallel steps of the method on one GPU:
 *   1. static condensation of the element-local stress sigma and rotation
 *      omega (Sec. 4.2, eq. femSPmat), followed by the bubble ("double Schur")
 *      condensation (eqs. Hcoeffs, factorSsigma);
 *   2. the preconditioned Krylov solve of the condensed saddle-point system
 *      K = [[A, B^T], [B, 0]] with the block preconditioner of eq.
 *      (mhatinvfactor), Shat_p = M_p (Sec. 5.1), and the multiplicative
 *      auxiliary-space preconditioner on the condensed velocity block
 *      (Sec. 6.1, Theorem aux_pc_schur, Corollary aux_pc_mult): facet-block
 *      Gauss-Seidel, the embedding E^d of conforming P1 vector fields (eq.
 *      defED) and one geometric-multigrid V-cycle as the solver C for
 *      abar(u, v) = nu (eps u, eps v) (eq. defAhat).
 *
 * Conventions
 *   - Every function returns an int status: MCS_OK (0) or a negative MCS_ERR_*.
 *     mcs_last_error() returns a thread-local message for the last failure.
 *     No C++ exception, abort or device trap crosses this interface.
 *   - "device" pointers are CUDA global-memory pointers on the handle's device
 *     (e.g. from torch); "host" pointers are ordinary CPU memory.  The caller
 *     owns every buffer it passes; the library owns the handle and the
 *     operators it keeps resident on the device.
 *   - Calls are asynchronous on the handle's stream unless stated otherwise.
 *   - Threads: one handle must not be used by two host threads at once; different handles are
 *     independent and may be used concurrently, each on its own stream (the serving loop does so).
 *   - Vectors of the condensed system have length ndof, layout
 *       [u_d | u_o | uhat | p]
 *     u_d: BDM facet moments (interior facet rank r, mode j) at r*nF + j;
 *     u_o: BDM bubbles (element T, m) at off_o + T*n_bub + m;
 *     uhat: tangential facet dofs (r, tangent m, mode j) at off_h + r*nhF + m*dimP^{k-1}(F) + j;
 *     p: pressure (T, mode j) at off_p + T*n_p + j.
 *     Lowest-order variant (k = 1, Sec. 7, dim = 3): no bubbles; the rotation omega lies in
 *     H(div) (P^0(T, R^3) + x P^0(T)), is kept after condensation, and its dof on facet r, the
 *     flux int_F omega.n_F, follows the two tangential uhat dofs: nhF = 3, uhat block of r =
 *     (t_1, t_2, omega flux).  The weak form uses kappa(omega) and adds nu (div omega, div eta).
 *   - Dof contract (the paper leaves bases and orientations open):
 *     * facets are the distinct sorted vertex tuples in lexicographic order; interior
 *       facets keep that order (rank r); local facet f of an element is opposite its
 *       local vertex f; the unit normal n_F satisfies det[e_1..e_{d-1}, n_F] > 0 for
 *       the edge vectors e_m = x_{w_m} - x_{w_0} of the sorted facet vertices w, and
 *       s_{T,f} = +1 where n_F points out of T;
 *     * orthonormal Dubiner polynomials (homogeneous Jacobi products, total degree
 *       ascending) on the reference simplex and on the facet parameter simplex;
 *     * V_h = BDM^k as the dual basis of the facet moments int_F u.n_F q_j and of
 *       interior moments of the Piola pull-back against the list psi_a e_c (deg <= k-2),
 *       then the Nedelec-type functions (-y, x) x^a y^b (2D) or x cross (x^alpha e_c) (3D),
 *       |alpha| = k-2, made L2-orthonormal on the reference simplex in list order;
 *     * uhat: q_j(s) e_m on each interior facet, deg q_j <= k-1; p: Dubiner, deg <= k-1;
 *     * structured meshes: the Kuhn split of N^dim cells, vertex (i,j[,l]) has id
 *       i + (N+1)(j + (N+1) l); element cell*dim! + (permutation index).
 *     All boundary facets are Dirichlet (u = 0) and carry no dofs; the pressure is
 *     fixed by a zero mean.
 */
#ifndef MCS_H
#define MCS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MCS_OK = 0,
  MCS_ERR_INVALID_ARG = -1,
  MCS_ERR_OOM = -2,
  MCS_ERR_CUDA = -3,
  MCS_ERR_NOT_CONVERGED = -4,
  MCS_ERR_BREAKDOWN = -5,
  MCS_ERR_TIMEOUT = -6,
  MCS_ERR_UNSUPPORTED = -7
};

enum { MCS_FP64 = 0, MCS_MIXED = 1 };

typedef struct mcs_handle mcs_handle;

typedef struct {
  int precision;      /* MCS_FP64: preconditioner in FP64; MCS_MIXED: preconditioner (smoother,
                         E^d, V-cycle, bubble solves) in FP32, outer Krylov and K in FP64 */
  int smooth_steps;   /* facet-block Gauss-Seidel sweeps before and after the coarse correction (2) */
  int gmg_levels;     /* multigrid levels incl. the coarsest (-1: auto, coarsest 16^2 / 4^3 cells) */
  int gmg_smooth;     /* l1-Jacobi sweeps before and after each coarse-grid correction (2) */
  double rtol;        /* stop when ||r||_{Khat^{-1}} <= rtol * ||F - K x0||_{Khat^{-1}} (1e-8) */
  int maxit;          /* total MinRes iterations (1000) */
  int max_refine;     /* outer refinement cycles after the first (8); MCS_FP64 uses at most 2 of them */
  double inner_rtol;  /* MCS_MIXED, and both forms with etol > 0: relative reduction per refinement cycle (1e-5) */
  int residual_dd;    /* residual of each refinement cycle in double-double: 1 always, 0 never (plain
                         FP64 K x, whose rounding floors the attainable residual near 1e-12 relative
                         for k = 4), -1 auto: when rtol < 1e-10 or etol > 0 (-1) */
  int asp;            /* auxiliary-space preconditioner for the condensed velocity block (Sec. 6.1):
                         0 multiplicative (smoother, coarse correction, adjoint smoother; default),
                         1 additive (facet-block Jacobi plus E^d C^{-1} E^d^T) */
  int lo_stab;        /* k = 1 only (Sec. 7), coefficient of (div omega, div eta)_T: 0 nu (default),
                         1 nu h_T^2 with h_T the element diameter (keeps the iteration count
                         bounded under refinement; see Table ST_ws) */
  int outflow;        /* mcs_setup_structured, k >= 2 only: 1 makes the face x_1 = 1 an outflow
                         boundary Gamma_Ntilde (eq. stokes_NT: u_t = 0, ((sigma + p I) n).n = 0);
                         0 (default): all faces Dirichlet.  See "Outflow" below. */
  double etol;        /* > 0: stop on the solution's error as well as on the residual (0 = off, the
                         default).  Then both forms run refinement cycles, each restarted from the exact
                         (double-double) residual: the correction d_c of cycle c (relative size rho_c =
                         max(|d_u|/|x_u|, |d_p|/|x_p|), 2-norms of the u and p blocks) estimates the error
                         entering it, and the error leaving it is bounded by est_c = 3 lag R_c rho_c with
                         R_c the cycle's achieved residual reduction and lag = max(1, (rho_c/rho_{c-1}) /
                         R_{c-1}) (from the third cycle on; else 1) how much less the previous cycle reduced
                         the error than its residual.  The first cycle runs to rtol (mixed form: to
                         inner_rtol); each later one ends as soon as that bound, evaluated on its
                         correction so far every 4 iterations, is <= etol.  The solve ends at the first
                         cycle start after est_c <= etol whose recomputed residual meets rtol; the bound is
                         returned in mcs_solve_info.err_est.  With a pressure-dominated right-hand side
                         (nu << 1) the velocity error exceeds the relative residual by orders of magnitude,
                         which the residual test alone does not see. */
  int tune;           /* 1: at the first mcs_condense of the handle, time the candidate launch shapes of the
                         batched facet step (2D) and of the staged K apply on the handle's own data and keep
                         the fastest (results are bitwise the same for every shape); 0 (default): the
                         shared-memory formulas */
  const char* tune_cache;  /* tune = 1: optional path of a text file of tuned shapes, one line per
                         (dim, k, precision, element count); read before tuning, appended after (NULL: none) */
  int facet_push;     /* multiplicative ASP: 1 (default) runs the facet sweeps before the coarse correction
                         with a maintained residual where the warp-per-facet smoother applies (facet blocks of
                         at least 4 KB with 2 m_F <= 32: 3D k = 2 and 2D k = 6 in both forms, 2D k = 4, 5 in
                         the FP64 form; mcs_sizes_t.push_warps > 0 when it is in use), so that
                         the residual for E^d^T needs no pass of its own; 0: row products and a residual
                         pass.  Both compute the same block Gauss-Seidel sweep (Corollary aux_pc_mult) and
                         differ only in rounding. */
} mcs_options;

typedef struct {
  int64_t ndof, n_dd, n_oo, n_hat, n_pres;  /* condensed system and its blocks */
  int64_t off_o, off_h, off_p;
  int64_t ne, nint, nfacets, nvertices;     /* mesh */
  int64_t np1;                              /* conforming P1 dofs (interior vertices * d) */
  int32_t dim, k, nF, n_bub, nhF, n_p, n_A, n_c, mF;
  int32_t ncolours, gmg_levels;
  int32_t nq_load;                          /* load quadrature points per element */
  int64_t bytes_resident;                   /* device bytes held by the handle */
  int32_t facet_batch, facet_threads, apply_batch;   /* launch shapes in use (-1: formulas; see tune) */
  int32_t push_warps;                       /* warps per block of the maintained-residual forward sweep
                                               (0: not in use; see facet_push) */
} mcs_sizes_t;

typedef struct {
  int iterations;            /* MinRes iterations (all refinement cycles) */
  int refinements;           /* outer cycles (each restarts MinRes from the recomputed residual) */
  int status;                /* MCS_OK, MCS_ERR_NOT_CONVERGED or MCS_ERR_BREAKDOWN */
  double rel_res_precond;    /* ||F - K x||_{Khat^{-1}} / ||F - K x0||_{Khat^{-1}} */
  double rel_res_true;       /* ||F - K x||_2 / ||F||_2 (FP64) */
  double err_est;            /* opt.etol > 0: estimated relative error of x (see etol), else 0 */
} mcs_solve_info;

/* Version of the library (e.g. 100 = 0.1.0). */
int mcs_version(void);
/* Thread-local description of the last error (never NULL). */
const char* mcs_last_error(void);
/* Fills *o with the defaults listed above. */
int mcs_default_options(mcs_options* o);

/* Outflow (opt.outflow = 1, Sec. 6.2, Lemma outflow).  The facets on the face x_1 = 1 carry BDM dofs
 * (u_n is free there) and take a rank among the coupling facets, which are then the interior and the
 * outflow facets in facet order: u_d, uhat and the facet-interleaved vectors use that rank.  uhat is
 * zero on Gamma_Ntilde; its slots of outflow facets stay in the layout as phantom dofs whose rows and
 * columns of K are those of the identity (they remain 0 for a right-hand side that is 0 there).  The
 * pressure has no constant mode, so no mean is removed.  The conforming space is free inside the face,
 * Abar gains nu C k^2 / h_F int_F u_t v_t on it (C = 4, h_F the facet diameter) and E^d has no uhat
 * rows there (pi_0).  Not available with k = 1, mcs_setup_mesh or mcs_condense_noalloc. */

/* Set-up on the Kuhn triangulation of [0,1]^dim with N cells per direction
 * (Sec. 7 uses unstructured meshes; the synthetic workloads use this nested
 * family so that the conforming space has a geometric multigrid hierarchy).
 * dim in {2, 3}, k = 2..6 (Sec. 3), or k = 1 with dim = 3 (the lowest-order variant of Sec. 7),
 * nu > 0 as printed in eq. (stokes).  stream: a cudaStream_t (NULL = default).
 * Builds mesh, facets, dof maps, colouring and the multigrid hierarchy on the
 * host and uploads them; allocates the resident operators.  Synchronous.
 * Errors: INVALID_ARG (bad sizes, N not divisible for the requested levels),
 * UNSUPPORTED (dim/k out of range), OOM, CUDA. */
int mcs_setup_structured(int dim, int N, int k, double nu, const mcs_options* opt, void* stream,
                         mcs_handle** out);

/* Set-up on a general simplicial mesh (host arrays, copied): coords [nv][dim],
 * elems [ne][dim+1] with ascending vertex ids per element.  The conforming
 * solver C is then an exact solve on the mesh's own P1 space (single level),
 * so this is meant for small meshes.  Errors as above. */
int mcs_setup_mesh(int dim, int64_t nv, const double* coords, int64_t ne, const int32_t* elems, int k,
                   double nu, const mcs_options* opt, void* stream, mcs_handle** out);

/* Sizes, offsets and resident bytes of a handle. */
int mcs_sizes(const mcs_handle* h, mcs_sizes_t* s);

/* Mesh and numbering export (host buffers, for bit-exact checks of the dof contract):
 * facets [nfacets][dim] sorted vertex ids; elem_facets [ne][dim+1]; signs [ne][dim+1]
 * orientation s_{T,f}; colour [nint] facet colour per interior rank.  NULL skips an array. */
int mcs_export_mesh(const mcs_handle* h, int32_t* facets, int32_t* elem_facets, int8_t* signs, int32_t* colour);
/* elem_dofs [ne][n_A + n_p]: global index of every local dof (local order u_d(f,j) | u_o |
 * uhat(f,m,j) | p), -1 on Dirichlet facets.  Host buffer. */
int mcs_export_dofmap(const mcs_handle* h, int64_t* elem_dofs);
/* CSR sparsity pattern of K (host).  rowptr [ndof+1]; col [rowptr[ndof]] ascending per
 * row, or NULL to query rowptr only. */
int mcs_export_pattern(const mcs_handle* h, int64_t* rowptr, int32_t* col);

/* Static condensation (Sec. 4.2): per element A_T (FP64), then A^d_T, G_T = A_oo^{-1} A_od,
 * A_oo^{-1} and the inverted facet blocks of the smoother in the preconditioner's
 * precision.  Asynchronous; idempotent. */
int mcs_condense(mcs_handle* h);
/* Static condensation of several problems in one persistent launch (elements of different meshes
 * and degrees k interleaved over the blocks); the same arithmetic as mcs_condense per handle, so the
 * results are identical.  handles: host array of count handles on the current device, all of the same
 * precision.  Runs on the stream of handles[0]; it waits for the work already enqueued on the other
 * handles' streams and their streams wait for it (events, no host synchronisation).  Takes a
 * temporary workspace from the stream-ordered allocator (largest element workspace x 4 blocks per
 * SM, fewer where that exceeds 2 GiB).  Errors: INVALID_ARG (NULL, count < 1, mixed precisions or devices), OOM, CUDA. */
int mcs_condense_batch(mcs_handle* const* handles, int count);

/* Copies the packed lower triangle of A_T (FP64, [count][n_A(n_A+1)/2], row-major
 * packing i(i+1)/2 + j, local order u_d | u_o | uhat, orientation signs applied) of
 * elements T0 .. T0+count-1 to a host buffer.  Synchronous. */
int mcs_copy_element_matrices(const mcs_handle* h, int64_t T0, int64_t count, double* AT_host);
/* Copies A^d_T ([count][n_c][n_c]) and G_T ([count][n_bub][n_c]) as FP64 to host buffers;
 * coupling dofs in facet-major order (facet f: nF facet moments then nhF tangential dofs).
 * The rows of A^d_T that belong to boundary facets are not kept on the device (those dofs are
 * eliminated by the Dirichlet condition) and come back as NaN.  Synchronous. */
int mcs_copy_schur(const mcs_handle* h, int64_t T0, int64_t count, double* Ad_host, double* G_host);

/* Physical load quadrature points, device buffer xq [ne*nq_load][dim]. */
int mcs_load_points(mcs_handle* h, double* xq);
/* F = (f, phi^u) for f given at the load points (device fq [ne*nq_load][dim]); F device [ndof],
 * zero outside the velocity block. */
int mcs_load_vector(mcs_handle* h, const double* fq, double* F);
/* F = M_u c: velocity mass matrix times the coefficient vector c (device [ndof]; only the
 * velocity blocks u_d, u_o are read); used for random right-hand sides f = sum c_j phi_j. */
int mcs_mass_velocity(mcs_handle* h, const double* c, double* F);

/* y = K x (eq. femSPmat), FP64, device vectors [ndof]. */
int mcs_apply(mcs_handle* h, const double* x, double* y);
/* r = F - K x, device vectors [ndof], with every element product and the sum of a facet dof's
 * two element contributions carried in double-double and rounded once, so r is accurate to a
 * few units in its own last place even where F and K x cancel.  MCS_MIXED: K uses the stored
 * float pairs hi + lo of A_T, taken as exact.  r may alias F, not x.  Uses a workspace of the
 * handle (calls on one handle are serialised by its stream). */
int mcs_residual(mcs_handle* h, const double* F, const double* x, double* r);
/* z = Khat^{-1} r (eq. mhatinvfactor applied with two Ahat^{-1}), device vectors [ndof];
 * the pressure part of z is not mean-corrected. */
int mcs_precond(mcs_handle* h, const double* r, double* z);
/* Solves K x = F by preconditioned MinRes (FP64 recurrence) inside outer refinement cycles:
 * each cycle recomputes r = F - K x (in double-double as mcs_residual when residual_dd selects
 * it, so the attainable accuracy is not limited by the rounding of K x); MCS_MIXED runs
 * FP32-preconditioned cycles, each asked for at least inner_rtol reduction.
 * x: in = initial guess, out = solution with mean-zero pressure.  Device vectors.  Synchronises
 * with the stream to read the convergence state.  info may be NULL.  Returns MCS_OK, or
 * MCS_ERR_NOT_CONVERGED / MCS_ERR_BREAKDOWN (x then holds the last iterate). */
int mcs_solve(mcs_handle* h, const double* F, double* x, mcs_solve_info* info);
/* Same as mcs_solve with HOST vectors F, x [ndof]: copies F and x in, solves, copies x out. */
int mcs_solve_host(mcs_handle* h, const double* F_host, double* x_host, mcs_solve_info* info);

/* Local recovery of the stress and rotation (eq. projection): for the solution x (device [ndof],
 * layout above), per element the element-local problem of eq. (bigfemSPmat) is solved for
 * (sigma_T, omega_T) given the element's (u, uhat), and both fields are evaluated at nq reference
 * points xhat_host (host [nq][dim], coordinates on the reference simplex with vertices 0, e_1..e_dim;
 * the physical point is x_0 + J xhat with J's columns x_i - x_0).  sigma, omega: device
 * [ne][nq][dim][dim] (physical tensors; omega may be NULL).  Recomputes the condensation workspace of
 * every element (about the cost of mcs_condense).  Asynchronous; takes a small temporary from the
 * stream-ordered allocator.  For k = 1 the rotation is a global unknown (its flux dofs are part of
 * x), only sigma is recovered and omega must be NULL (else UNSUPPORTED).
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
int mcs_recover_stress(mcs_handle* h, const double* x, int nq, const double* xhat_host, double* sigma,
                       double* omega);

/* Kernel timing (diagnostics): when enabled, the library brackets its main kernel classes
 * with CUDA events on the handle's stream during mcs_condense / mcs_apply / mcs_precond /
 * mcs_solve.  mcs_profile(h, 1) enables and clears, 0 disables.  mcs_profile_read fills up
 * to max_n entries (one per kernel class: name, launches, total device ms, algorithmic bytes
 * and flops of those launches) and returns their number; it synchronises the stream. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
  double bytes;
  double flops;
} mcs_kernel_stat;
int mcs_profile(mcs_handle* h, int enable);
int mcs_profile_read(mcs_handle* h, mcs_kernel_stat* out, int max_n);

/* Kernel-launch accounting (diagnostics): *count receives the number of kernels this library
 * has launched in this process, over all handles and threads, since it was loaded.  A kernel
 * that runs as a node of one of the library's CUDA graphs counts once per graph launch;
 * launches recorded while a graph is being captured do not count.  Copies and memsets are not
 * kernels and do not count.  Host-only; never fails except for a NULL count (INVALID_ARG). */
int mcs_launch_count(uint64_t* count);

/* Condensed element matrices without any device allocation, for callers that cannot let the
 * library allocate at call time: applications that own the whole device through their own pool
 * or run under a fixed memory budget, and code paths that must not block on the allocator
 * (cudaMalloc / cudaFree can synchronise the device).  The paper has no counterpart: this is a
 * deployment variant of the condensation of Sec. 4.2.
 *   AT_out: device buffer [count][n_A][n_A] (FP64, full symmetric, local order u_d | u_o | uhat,
 *           orientation signs applied) receiving A_T of elements T0 .. T0+count-1 of the handle.
 * Workspace: a file-scope 4 MiB device array, held by every GPU that loads the library until
 * the process exits; one element's workspace must fit in it (3D k = 4 needs 1.1 MiB and 3D k = 5
 * 2.8 MiB; 3D k = 6, 6 MiB, is refused), else MCS_ERR_UNSUPPORTED.  Nothing is allocated or freed: no cudaMalloc, no allocating library
 * routine.  The first call on a device looks up the array's device address (with that device
 * current); make that first call before any stream capture.  All calls share the array, so
 * calls whose kernels overlap on the GPU (other streams, other host threads) race: order them
 * on one stream.  The current device must be the handle's device.  Asynchronous on the handle's
 * stream.  Errors: INVALID_ARG (NULL, range, wrong device), UNSUPPORTED, CUDA. */
int mcs_condense_noalloc(mcs_handle* h, int64_t T0, int64_t count, double* AT_out);

/* Releases the handle and its device memory (synchronises its stream). */
int mcs_destroy(mcs_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* MCS_H */
