/*
 * bddc.h -- C ABI of the GB300 (sm_103a) adaptive BDDC library.
 *
 * The library computes the data-parallel hot path of adaptive BDDC in three
 * dimensions (Mandel, Sousedik, Sistek, "Adaptive BDDC in three
 * dimensions"): substructure Schur complements by batched dense Cholesky
 * (Section 2, eq. (reduced-problem)), the pairwise face generalized
 * eigenproblems and the adaptive face constraints (Section 3, eq.
 * (eig-matrix), (d-def), Algorithm 3.1), and PCG with the BDDC preconditioner
 * of Lemma 2.1 (eqs. (BDDC-prec)-(BDDC-Dc)) on one GPU.
 *
 * Conventions shared by every call
 *  - Every call returns a bddc_status; nothing aborts, traps or throws across
 *    the ABI.  bddc_last_error() gives a one-line reason for the last failure.
 *  - Pointers are plain host or device addresses; ``mem`` says which
 *    (BDDC_MEM_HOST / BDDC_MEM_DEVICE).  Inputs are copied during the call;
 *    the caller keeps ownership of every buffer it passes.
 *  - One handle serves one thread and one CUDA stream (bddc_options.stream,
 *    NULL = the legacy default stream).  Calls on one handle are not
 *    re-entrant.
 *  - Free degrees of freedom ("global dofs") are numbered node-major over the
 *    non-Dirichlet nodes in increasing node id, ncomp consecutive dofs per
 *    node.  Interface dofs (dofs of nodes in more than one substructure)
 *    are numbered by increasing global dof.
 *  - Device memory is allocated by the handle (cudaMalloc, or the caller's
 *    allocator of bddc_options) and released by bddc_destroy.
 */
#ifndef BDDC_H
#define BDDC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BDDC_API __attribute__((visibility("default")))
#else
#define BDDC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BDDC_OK = 0,
    BDDC_EINVAL = 1,       /* bad argument or size */
    BDDC_ENOMEM = 2,       /* device or host allocation failed */
    BDDC_ENOTSPD = 3,      /* non-positive pivot in a Cholesky factorization */
    BDDC_EASSUMPTION = 4,  /* Assumption 1 or 2 of the paper violated (too few corners) */
    BDDC_ENOCONV = 5,      /* PCG reached maxit; the best iterate is returned */
    BDDC_ETIMEOUT = 6,     /* a bounded device wait gave up; the context stays usable */
    BDDC_ECUDA = 7,        /* a CUDA runtime error */
    BDDC_ESTATE = 8        /* call out of order (e.g. solve before setup) */
} bddc_status;

typedef enum { BDDC_MEM_HOST = 0, BDDC_MEM_DEVICE = 1 } bddc_mem;

typedef enum {
    BDDC_FP64 = 0,         /* every dense factorization in FP64 */
    BDDC_MIXED = 1,        /* interior elimination: FP32 factorization + FP64 refinement (S_i to
                              1e-11 relative); the local saddle and coarse inverses and the pair
                              condensations in double-float (unit roundoff 2^-48), their trailing
                              updates on the bf16 tensor cores by exact digit slicing
                              (mixed_updates = 0); face eigenproblems in double-float with FP64
                              Sturm counts and Rayleigh quotients; PCG in FP64.  The
                              preconditioner matches the FP64 one to ~1e-9. */
    BDDC_MIXED_FP32_SADDLE = 2  /* as BDDC_MIXED, and the local saddle operators of the
                              preconditioner (Lemma 2.1) from an equilibrated FP32
                              factorization (rebuilt in FP64 if a pivot falls below 1e-5).
                              The preconditioner is then exact only to ~1e-5, which spreads
                              the eigenvalue cluster of M S at 1: PCG may need more
                              iterations than in FP64 (observed up to +33%). */
} bddc_precision;

enum { BDDC_AVG_EDGE = 1, BDDC_AVG_FACE = 2 };

typedef struct {
    int precision;         /* bddc_precision, default BDDC_FP64 */
    double tol;            /* PCG relative residual tolerance, default 1e-8 */
    int maxit;             /* PCG iteration limit, default 1000 */
    double drop_rel;       /* per-face rank drop of adaptive rows, default 1e-10 */
    double timeout_s;      /* limit of every bounded device wait, default 10 s */
    void *stream;          /* cudaStream_t; NULL = default stream */
    /* Device memory of the handle.  NULL (default) = cudaMalloc / cudaFree.
     * Otherwise every device buffer the handle owns comes from dev_alloc(bytes,
     * alloc_ctx) (it must return device memory usable on ``stream``, 256-byte
     * aligned, or NULL on failure -> BDDC_ENOMEM) and goes back through
     * dev_free(ptr, bytes, alloc_ctx).  Buffers are freed only after the
     * handle's stream is synchronized, so a stream-ordered allocator
     * (cudaMallocAsync on the same stream, a caching allocator keyed on the
     * stream) is safe.  Both callbacks or neither must be given. */
    void *(*dev_alloc)(size_t bytes, void *alloc_ctx);
    void (*dev_free)(void *ptr, size_t bytes, void *alloc_ctx);
    void *alloc_ctx;
    /* Mixed modes: the refinement of X = A_II^-1 A_IG stops at the first step with
     * ||A_IG - A_II X|| <= refine_tol ||A_IG|| per substructure (S_i is then formed
     * in the energy form, whose error R^T A_II^-1 R is second order in that residual,
     * so the default 1e-8 already gives S_i to ~1e-13 relative). */
    double refine_tol;
    /* Pair eigenproblems (Section 3).  By default every face is solved densely
     * (Householder reduction, by several CTAs per face above order 200, then Sturm
     * counts, bisection and inverse iteration).  Faces whose reduced problem has
     * order above eig_large_n (default -1: none) are instead solved by batched LOBPCG
     * (the eigensolver the paper names for them):
     * blocks of 16 (then 32) Ritz vectors, FP64 products and Rayleigh-Ritz, until every
     * selected pair and the largest rejected one has ||C x - theta x|| <= eig_tol |theta|
     * (default 1e-8) or eig_maxit iterations (default 240) have run.  The number of
     * eigenvalues above tau is then certified by a Cholesky factorization (see
     * bddc_adapt); a face that does not converge or fails the certificate is solved by
     * the dense kernel.  Both paths select the same constraints. */
    int eig_large_n;
    double eig_tol;
    int eig_maxit;
    /* Mixed modes: the double-float factorizations (pair condensations, local saddle and
     * coarse inverses).  0 (default): in block columns of 128 whose triangular solves
     * (against the inverse of the diagonal block's factor) and trailing updates run on the
     * tensor cores, by exact bf16 slicing (7 digit planes of 7 bits, FP32 accumulation of
     * integer digit products, double-float combination; ~2^-49 per product);
     * 1: double-float on the FP32 pipe. */
    int mixed_updates;
} bddc_options;

/* One substructure of an algebraic problem (bddc_set_problem): its local matrix
 * A_i (Section 2: A_i is the subassembly of the substructure's part of the
 * bilinear form, so A = sum_i R_i^T A_i R_i) in CSR over local dofs. */
typedef struct {
    int32_t n_local;       /* local dofs (rows of A_i) */
    const int64_t *l2g;    /* (n_local) local dof -> global dof, 0 <= g < n_global */
    const int64_t *rowptr; /* (n_local + 1) CSR row pointers, rowptr[0] = 0 */
    const int32_t *col;    /* (rowptr[n_local]) local column indices */
    const double *val;     /* (rowptr[n_local]) values; both triangles of the symmetric A_i,
                              duplicate (row, col) entries are summed */
} bddc_subdomain;

typedef struct bddc_handle bddc_handle;

typedef struct {
    int n_faces;           /* face pairs examined */
    int n_added;           /* adaptive constraints added (after rank drop) */
    int n_ties;            /* eigenvalues within 1e-6 relative of tau */
    double omega;          /* condition number indicator max_ij lambda_ij,1 (eq. (cond-ind)) */
    int n_lobpcg;          /* faces solved by LOBPCG (order above bddc_options.eig_large_n) */
    int lobpcg_iters;      /* the most LOBPCG iterations any of them needed */
    int n_dense_fallback;  /* of those, faces handed to the dense kernel (no convergence,
                              block too small, or a failed count certificate) */
} bddc_adapt_info;

typedef struct {
    int iters;             /* PCG iterations */
    int converged;         /* 1 if ||r_k|| <= tol ||r_0|| */
    double relres;         /* true relative residual ||g - S u_G|| / ||g|| of the condensed
                              interface problem (eq. (reduced-problem)), recomputed on the
                              device from the local S_i after PCG */
    double kappa;          /* Lanczos estimate lambda_max / lambda_min */
    double setup_ms;       /* last bddc_setup + bddc_adapt, device time */
    double solve_ms;       /* this solve, device time */
    int interior_fp32;     /* 1: S_i came from the FP32 factorization + FP64 refinement */
    int coarse_fp32;       /* 1: the local saddle operators came from the FP32 factorization */
    int refine_steps;      /* mixed modes: corrections of the interior refinement */
    double refine_relres;  /* mixed modes: its final largest relative residual */
    double relres_recurrence; /* ||r_k|| / ||r_0|| of the PCG recurrence (the stopping test) */
} bddc_solve_info;

/* Fills *opt with the defaults above. */
BDDC_API void bddc_default_options(bddc_options *opt);

/* Creates a handle.  opt may be NULL (defaults).  *out receives the handle.
 * Errors: BDDC_ENOMEM, BDDC_ECUDA (no device). */
BDDC_API bddc_status bddc_create(const bddc_options *opt, bddc_handle **out);

/* Releases every host and device buffer of the handle.  NULL is allowed. */
BDDC_API void bddc_destroy(bddc_handle *h);

/* Defines the problem from a trilinear hexahedral (Q1) mesh (Section 2: each
 * substructure is a union of elements and A_i is the subassembly of its
 * element matrices).
 *   ncomp      1 = scalar diffusion -div(k grad u), 3 = linear elasticity
 *   nn, xyz    nodes, xyz row-major (nn x 3) float64
 *   ne, elems  elements, row-major (ne x 8) int64 node ids, local node
 *              a = ax + 2 ay + 4 az for the reference corner (ax, ay, az)
 *   coef       (ne) float64: k_e (ncomp 1) or Young modulus E_e (ncomp 3)
 *   nu         Poisson ratio (ncomp 3; ignored for ncomp 1)
 *   elem_sub   (ne) int32 substructure of each element, 0 <= s < nsub
 *   dirichlet  (nn) uint8, non-zero = every component of the node fixed to 0
 *   mem        where the arrays live
 * Classifies the interface into faces, edges and corners (Section 2; corner
 * = a one-node edge set, or an edge-set node with at most one element-edge
 * neighbour in its own set and no neighbour whose set is a strict superset),
 * on the full mesh, then drops Dirichlet nodes.  Resets constraints to
 * corners only.  Errors: BDDC_EINVAL (sizes, ids out of range), BDDC_ENOMEM. */
BDDC_API bddc_status bddc_set_mesh_q1(bddc_handle *h, int ncomp, int64_t nn, const double *xyz, int64_t ne,
                             const int64_t *elems, const double *coef, double nu, const int32_t *elem_sub,
                             int32_t nsub, const uint8_t *dirichlet, int mem);

/* Defines the problem algebraically from the substructure matrices A_i
 * (Section 2: A = sum_i R_i^T A_i R_i).  Dirichlet dofs are already
 * eliminated by the caller, so every global dof is free and the global dof
 * numbering is the caller's, 0 <= g < n_global.  Node of dof g = g / ncomp:
 * the ncomp dofs of a node are consecutive, and a substructure holds either
 * all or none of them.
 *   ncomp      1 = scalar, 3 = elasticity (rigid modes from node_xyz)
 *   subs       (n_sub) CSR matrices; arrays in memory ``mem``
 *   node_xyz   (n_global / ncomp) x 3 row-major coordinates; required for
 *              ncomp = 3 (rigid body modes, corner augmentation), may be NULL
 *              for ncomp = 1
 * Globs follow Section 2 (faces: nodes of exactly two substructures; edges:
 * nodes of one set of three or more).  Corners are chosen by the rule of
 * bddc_set_mesh_q1 with "neighbour" read as a node coupled to it in some A_i
 * (the element-edge graph is not known here), on the free nodes only; then
 * face pairs with a floating member receive augmented corners (Assumptions 1
 * and 2).  A substructure floats when A_i annihilates the rigid modes (the
 * constant, or the six rigid body motions of node_xyz) to 1e-8 relative.
 * bddc_set_corners replaces the corner choice.  Resets constraints to corners
 * only.  Inputs are copied.  Errors: BDDC_EINVAL (sizes, indices, a dof in no
 * substructure, a node split between substructures, missing node_xyz for
 * ncomp = 3), BDDC_EASSUMPTION, BDDC_ENOMEM. */
BDDC_API bddc_status bddc_set_problem(bddc_handle *h, int64_t n_global, int ncomp, int32_t n_sub,
                                      const bddc_subdomain *subs, const double *node_xyz, int mem);

/* Host-only mesh analysis: the classification that bddc_set_mesh_q1 performs
 * (Section 2: faces, edges, corners by the same rule; Assumptions 1 and 2:
 * floating substructures and face pairs, corner augmentation), run on the
 * host without a handle, a GPU or any device memory.  Inputs as in
 * bddc_set_mesh_q1 (host memory only; coef and nu are not needed).
 * Outputs (each may be NULL):
 *   n_free, n_interface   free dofs and interface dofs
 *   n_corners, n_edges, n_faces   glob counts after Dirichlet nodes are dropped
 *                         and corners augmented (faces that lost every node
 *                         to augmentation are not counted)
 *   n_augmented           face nodes promoted to corners
 *   corners[corners_cap]  corner node ids, ascending (the first corners_cap)
 * Errors: BDDC_EINVAL (sizes, ids out of range), BDDC_EASSUMPTION (a
 * floating substructure whose corners cannot fix its rigid modes). */
BDDC_API bddc_status bddc_classify_q1(int ncomp, int64_t nn, const double *xyz, int64_t ne, const int64_t *elems,
                                      const int32_t *elem_sub, int32_t nsub, const uint8_t *dirichlet,
                                      int64_t *n_free, int64_t *n_interface, int *n_corners, int *n_edges,
                                      int *n_faces, int *n_augmented, int64_t *corners, int corners_cap);

/* Replaces the corners (Section 2: the coarse point constraints, W^c of the
 * paper's Fig. 3) by the n given node ids (host memory, any order, duplicates
 * ignored); no rule and no augmentation is applied.  Every node must be an
 * interface node.  Edges and faces are re-derived without those nodes.
 * Resets constraints to corners only.  Must follow bddc_set_problem or
 * bddc_set_mesh_q1 and precede bddc_setup.  Errors: BDDC_ESTATE, BDDC_EINVAL
 * (node out of range or not on the interface), BDDC_EASSUMPTION (the corners
 * do not fix the rigid modes of a floating substructure or face pair). */
BDDC_API bddc_status bddc_set_corners(bddc_handle *h, int64_t n, const int64_t *nodes);

/* Re-applies the default corner rule and augmentation (undoing
 * bddc_set_corners); *n_out (may be NULL) receives the number of corners.
 * Resets constraints to corners only.  Errors: BDDC_ESTATE, BDDC_EASSUMPTION. */
BDDC_API bddc_status bddc_select_corners(bddc_handle *h, int64_t *n_out);

/* Adds arithmetic averages as initial constraints (Section 2, eq. (Wtilde);
 * one coarse dof per glob and component): flags = BDDC_AVG_EDGE | BDDC_AVG_FACE.
 * Must follow bddc_set_mesh_q1 or bddc_set_problem and precede bddc_setup. */
BDDC_API bddc_status bddc_set_averages(bddc_handle *h, int flags);

/* Numeric setup: assembles A_i on the device, factors A_II and forms
 * S_i = A_GG - A_GI A_II^{-1} A_IG (Section 2), the averaging weights
 * delta_i = diag(A_i) / sum_k diag(A_k) (Section 7), and the local saddle
 * and coarse operators of the preconditioner for the current constraints.
 * Errors: BDDC_ESTATE (no mesh), BDDC_ENOTSPD, BDDC_EASSUMPTION, BDDC_ECUDA. */
BDDC_API bddc_status bddc_setup(bddc_handle *h);

/* Algorithm 3.1: for every pair of substructures sharing a face solves the
 * pair eigenproblem (eq. (eig-matrix)) and adds, for every eigenvalue
 * lambda > tau, the face part of d = w^T (I-E)^T S^c (I-E) (eq. (d-def))
 * as a weighted-average face constraint (edge parts dropped, Remark of
 * Section 3, unless bddc_set_edge_rows keeps them), then rebuilds the
 * preconditioner.  info may be NULL.
 * Errors: BDDC_ESTATE (no setup), BDDC_ENOTSPD, BDDC_EASSUMPTION. */
BDDC_API bddc_status bddc_adapt(bddc_handle *h, double tau, bddc_adapt_info *info);

/* As bddc_adapt, but every face gets the constraints of the n_per_face largest
 * eigenvalues of its pair problem (all of them when there are fewer) instead of
 * those above a threshold: the "c+e+f (3eigv)" constraints of Section 7 with
 * n_per_face = 3 after bddc_set_averages(h, BDDC_AVG_EDGE).  info->n_ties counts
 * faces whose last selected and first rejected eigenvalues agree to 1e-6
 * (the selected subspace is then not unique).  Errors: BDDC_ESTATE (no setup),
 * BDDC_EINVAL (n_per_face outside 1..48), BDDC_ENOTSPD, BDDC_EASSUMPTION. */
BDDC_API bddc_status bddc_adapt_fixed(bddc_handle *h, int n_per_face, bddc_adapt_info *info);

/* keep = 1: every later bddc_adapt / bddc_adapt_fixed also keeps the edge parts of the
 * selected rows d (Section 3 splits each d into one row on the face and one row per edge,
 * so that every row stays on one glob; the paper's experiments drop the edge rows, the
 * Remark closing Section 3, which is the default keep = 0).  Per edge, the edge parts
 * of every face pair's rows on it (each normalised; a part below drop_rel * sqrt(2) |d|
 * is left out) are orthonormalised with row pivoting, keeping rows while the pivot
 * exceeds drop_rel of the first (BDDC_FP64), or max(drop_rel, 1e-6) in the mixed modes
 * (the pairs' rows on one edge overlap in exact arithmetic, and below 1e-6 the mixed
 * modes' eigenvectors cannot tell a rounding direction from a real one), and the basis
 * becomes a constraint on all substructures sharing the edge.  That is a stronger
 * constraint set than the pairwise split rows, and with it every face pair's largest
 * eigenvalue on the constrained space is still at most its lambda_{k+1} <= tau, so
 * omega~ <= tau (the Courant-Fisher-Weyl principle with Algorithm 3.1); unlike the
 * pairwise rows, the rows of every substructure stay independent, as the primal
 * coarse space (Remark 5.1) needs.  Errors: BDDC_EINVAL (keep not 0 or 1); the adapt
 * call fails with BDDC_EINVAL when an edge is shared by more than 8 face pairs. */
BDDC_API bddc_status bddc_set_edge_rows(bddc_handle *h, int keep);

/* Edge rows kept by the last adapt in total, and the number of edges that got rows
 * (both 0 when bddc_set_edge_rows is off).  Either pointer may be NULL.
 * Errors: BDDC_EINVAL (null handle). */
BDDC_API bddc_status bddc_get_edge_rows(const bddc_handle *h, int *n_rows, int *n_edges);

/* Solves sum_i R_i^T A_i R_i u = f: condensed right-hand side, PCG with the
 * BDDC preconditioner to ||r|| <= tol ||r_0|| from x_0 = 0, interior
 * recovery.  f and u are global free-dof vectors (length n_free) in memory
 * ``mem``.  info may be NULL.  f = 0 gives u = 0 with no iteration (iters 0,
 * relres 0, condition estimate 1).  Errors: BDDC_ESTATE, BDDC_EINVAL (a load with
 * non-finite entries), BDDC_ENOCONV (maxit reached: u holds the solution recovered
 * from the last iterate, info is filled), BDDC_ETIMEOUT, BDDC_ECUDA. */
BDDC_API bddc_status bddc_solve(bddc_handle *h, const double *f, double *u, int mem, bddc_solve_info *info);

/* Extreme eigenvalues of the Lanczos matrix built from the last solve's PCG
 * coefficients alpha_k, beta_k (caption of Table 1 of the paper). */
BDDC_API bddc_status bddc_condition_estimate(const bddc_handle *h, double *lmin, double *lmax);

/* Sizes after bddc_set_mesh_q1 or bddc_set_problem (any pointer may be NULL). */
BDDC_API bddc_status bddc_get_sizes(const bddc_handle *h, int64_t *n_free, int64_t *n_interface, int *n_corners,
                           int *n_edges, int *n_faces, int *n_coarse);

/* Corner node ids (ascending) into nodes[cap]; *n = count. */
BDDC_API bddc_status bddc_get_corners(const bddc_handle *h, int64_t *nodes, int cap, int *n);

/* Self-test of the bounded device waits that the PCG kernel relies on (the
 * paper has no counterpart: it is failure detection for this library).  One
 * cooperative launch of a block per SM meets at the grid barrier of the PCG
 * kernel, told to wait for `extra` blocks more than exist.  extra = 0: every
 * block passes, *n_passed = the number of SMs, BDDC_OK.  extra > 0: nothing
 * releases the barrier, the wait gives up after timeout_s seconds, every
 * block returns, and the call reports BDDC_ETIMEOUT with *n_passed = 0; the
 * CUDA context stays usable.  Uses the handle's stream and status word only.
 * Errors: BDDC_ESTATE (null handle), BDDC_EINVAL (timeout_s <= 0 or > 60),
 * BDDC_ECUDA. */
BDDC_API bddc_status bddc_barrier_selftest(bddc_handle *h, int extra, double timeout_s, int *n_passed);

/* The adaptive constraint rows of face f kept by the last bddc_adapt
 * (eq. (d-def) restricted to the face dofs, normalised and orthogonalised
 * with row pivoting; the Remark at the end of Section 3 drops the edge
 * parts).  gdofs[n_dofs]: the face's global free dofs (ascending); rows:
 * row-major n_rows x n_dofs, host memory.  With cap_rows * cap_dofs too small
 * (or NULL buffers) only *n_rows and *n_dofs are set.  Errors: BDDC_ESTATE
 * (no mesh), BDDC_EINVAL (f out of range). */
BDDC_API bddc_status bddc_get_face_rows(const bddc_handle *h, int f, int64_t *gdofs, double *rows, int cap_rows,
                                        int cap_dofs, int *n_rows, int *n_dofs);

/* Face f (0 <= f < n_faces, faces ordered by (i, j), i < j): the pair, the
 * eigenvalues computed by the last bddc_adapt in descending order (the
 * selected ones plus the largest rejected one; at most cap) and the number
 * selected (lambda > tau) and kept after the rank drop. */
BDDC_API bddc_status bddc_get_face_eigs(const bddc_handle *h, int f, int32_t *i, int32_t *j, double *lam, int cap,
                               int *n_lam, int *n_selected, int *n_kept);

/* Interface dofs (global dof ids, ascending) of substructure s into gdofs[cap]. */
BDDC_API bddc_status bddc_get_interface_dofs(const bddc_handle *h, int s, int64_t *gdofs, int cap, int *n);

/* S_s after bddc_setup, n x n column-major into S (ld >= n), ordered as
 * bddc_get_interface_dofs; mem = where S lives. */
BDDC_API bddc_status bddc_get_schur(const bddc_handle *h, int s, double *S, int ld, int mem);

/* The assembled local stiffness matrix A_s (n x n, column-major into A, ld >= n),
 * ordered [interior dofs ascending; interface dofs ascending], as assembled by
 * the last bddc_setup.  In BDDC_FP64 mode the factorization overwrites the
 * lower triangle in place, so the call returns BDDC_ESTATE after a setup in
 * that mode; in the mixed modes the assembled matrix is kept. */
BDDC_API bddc_status bddc_get_local_matrix(const bddc_handle *h, int s, double *A, int ld, int mem);

/* One application of the preconditioner (z = M r) or of the assembled Schur
 * operator (y = S x) to an interface vector (length n_interface). */
BDDC_API bddc_status bddc_apply_preconditioner(bddc_handle *h, const double *r, double *z, int mem);
BDDC_API bddc_status bddc_apply_schur(bddc_handle *h, const double *x, double *y, int mem);

/* Device time (CUDA events on the handle's stream) and algorithmic FLOPs of
 * the phases of the last setup / adapt / solve, in this order:
 *   0 Q1 assembly + weights          1 interior elimination (partial Cholesky of A_i)
 *   2 coarse operators (built before the first solve or apply after a setup
 *     or adapt changed the constraints)
 *   3 pair condensations (adapt)     4 face eigenproblems (adapt)
 *   5 analysis of bddc_set_mesh_q1 (host wall time: classification, index maps, uploads)
 *   6 condensed right-hand side      7 PCG                       8 interior recovery
 * FLOPs of phase 1 are the dense count sum_i n_I^3/3 + n_I^2 n_G + n_I n_G^2;
 * phase 3 reports m^3/3 + m^2 (n-m) + m (n-m)^2 summed over its partial
 * Cholesky factorizations (order n, m columns eliminated); other phases
 * report 0 FLOPs.  ms[cap], flop[cap] may be NULL; *n = 9. */
BDDC_API bddc_status bddc_get_phase_times(const bddc_handle *h, double *ms, double *flop, int cap, int *n);

/* Kernel timers for roofline measurements.  on = 1 starts them (and clears the
 * totals), on = 0 stops them.  While on, every launch of the kernels below is
 * bracketed by CUDA events on the handle's stream.  Errors: BDDC_EINVAL. */
BDDC_API bddc_status bddc_set_kernel_timing(bddc_handle *h, int on);

/* Totals since the last bddc_set_kernel_timing(h, 1), one entry per class:
 *   0 trailing updates of the double-float partial Cholesky (pchol_update_kernel<ff>)
 *   1 trailing updates of the FP64 partial Cholesky
 *   2 trailing updates of the FP32 partial Cholesky
 *   3 tensor-core 3xTF32 GEMMs (tc_gemm_kernel)
 *   4 the persistent PCG kernel (solve launches)
 *   5 the face reductions (face_eig_kernel, tridiag_multi_kernel)
 *   6 tensor-core trailing updates of the double-float factorizations (oz_syrk_kernel;
 *     work = 2 x the multiply-adds of the block update, computed as 28 bf16 digit products)
 *   7 the digit splitting of their block columns (oz_split_kernel; work 0)
 *   8 the panel steps of every partial Cholesky (pchol_panel_kernel; work 0)
 * ms: summed device time of the launches; work: their algorithmic flop (partial
 * Cholesky updates: 2 x the multiply-adds of the lower-triangle tiles launched;
 * GEMMs: 2 M N K, one of the three TF32 products; reductions: 4/3 n^3 per face;
 * PCG: 0); launches: their count.  *n = 9; cap limits the entries written.  The call
 * waits for the recorded events.  Errors: BDDC_EINVAL (NULL handle). */
BDDC_API bddc_status bddc_get_kernel_times(bddc_handle *h, double *ms, double *work, int64_t *launches, int cap,
                                           int *n);

/* Number of kernel launches made by the handle so far (all phases). */
BDDC_API int64_t bddc_launch_count(const bddc_handle *h);

/* Schur complement of ONE dense symmetric matrix, for callers that cannot
 * allocate device memory (the paper has no counterpart; it is a service
 * entry point).  Callers that run under a fixed memory budget, own the device
 * memory through their own allocator, or must not allocate after start-up can
 * still use the interior elimination kernels through this call: it makes no
 * cudaMalloc, cudaFree or other allocating call.  Its scratch (a working copy
 * of A plus the kernels' work lists) is a static device array of about 8.5 MB
 * that every GPU loading the library holds until the process exits.
 *   n, n_int  order of A and number of leading (interior) rows to eliminate,
 *             0 <= n_int < n <= 1024 (larger n is rejected with BDDC_EINVAL)
 *   A, lda    device pointer, column-major, lower triangle read, not modified
 *   S, lds    device pointer: S = A_GG - A_GI A_II^{-1} A_IG written in full
 *             ((n - n_int) x (n - n_int), column-major, lds >= n - n_int)
 *   stream    cudaStream_t (NULL = default stream); the call synchronizes it
 *   msg       optional buffer (msg_cap bytes) for a one-line error reason
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (once per device, with that device current).  The CUDA
 * runtime loads device code lazily, so that first call is also when the array's
 * memory is taken on that device: make it at start-up (and before any stream
 * capture); later calls allocate nothing.  All calls share the one array:
 * calls whose work overlaps on the GPU (other threads or streams) race and
 * must be serialized by the caller.  Errors: BDDC_EINVAL (sizes, null
 * pointers, n > 1024), BDDC_ENOTSPD (A_II not positive definite), BDDC_ECUDA. */
BDDC_API bddc_status bddc_schur_dense_static(int n, int n_int, const double *A, int lda, double *S, int lds,
                                             void *stream, char *msg, int msg_cap);

BDDC_API const char *bddc_status_str(bddc_status s);
BDDC_API const char *bddc_last_error(const bddc_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* BDDC_H */
