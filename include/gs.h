/*
 * gs.h -- C ABI of the GB300 matrix-free generalized Stokes solver.
 *
 * Problem (Wichrowski et al., Sec. 3.1.2 predictor mode, Eqs. "form_a_j" and "form_b";
 * matrix form Eq. "stokes-discrete-block"):
 *
 *     alpha u - div(2 eta eps(u)) + grad p = f,   div u = g_p,
 *
 * discretised with Q2-Q1 Taylor-Hood elements (Sec. 3.2, Eq. "spaces", p1 = 2, p2 = 1) on a
 * structured Cartesian quad (dim = 2) or hex (dim = 3) mesh with one viscosity value per
 * cell.  The saddle matrix is K = [A B^T; B 0] with
 *     A[i a, j b] = sum_K alpha int phi_i phi_j delta_ab + eta_K int 2 eps(phi_j e_b):eps(phi_i e_a)
 *     B[q, j b]   = - sum_K int psi_q d phi_j / d x_b      (physical pressure sign).
 *
 * Solver (Sec. 4 and Sec. 5 "Linear solver settings"): FGMRES(m) with classical Gram-Schmidt
 * applied twice, right-preconditioned by the block upper-triangular operator
 *     z_p = -S^{-1} r_p,   z_u = V(r_u - B^T z_p),
 * where V is a velocity geometric-multigrid V-cycle with Chebyshev-Jacobi smoothing
 * (Cheb(A, diag(A), k_A)) and S = M_p(1/eta) is the 1/eta-weighted Q1 pressure mass matrix,
 * inverted approximately by Chebyshev-Jacobi iterations on Wathen's interval [2^-d, (3/2)^d].
 *
 * Vector layout (every vector argument): full length N = d*N_v + N_p, component-blocked,
 *     [u_x | u_y | (u_z) | p],
 * velocity nodes on the (2n_x+1) x (2n_y+1) [x (2n_z+1)] grid, pressure nodes on the
 * (n_x+1) x (n_y+1) [x (n_z+1)] grid, both lexicographic with x fastest.  Velocity-only
 * vectors (gs_vmult_A, gs_vcycle) have length d*N_v.
 *
 * Constraints: velocity nodes on a Dirichlet face (bit set in dirichlet_faces) or touching an
 * obstacle cell are constrained (all components); pressure nodes touched by no active cell
 * are constrained.  Constrained rows of K are identity rows and constrained columns are zero,
 * so a right-hand side holds the Dirichlet value at constrained entries (gs_lift_rhs builds
 * it).  With every face Dirichlet the constant pressure is in the kernel: the solver keeps
 * the Euclidean mean of the free pressure entries at zero.
 *
 * Memory and streams: all vector pointers are DEVICE pointers owned by the caller.  The
 * context owns no device allocation: the caller passes one device workspace of
 * gs_footprint_bytes() bytes (256-byte aligned) to gs_create and keeps it alive until
 * gs_destroy.  All work is enqueued on the stream given to gs_create (a cudaStream_t cast
 * to void*, NULL = legacy default stream).  gs_vmult, gs_vmult_A, gs_vcycle, gs_lift_rhs
 * and gs_apply_level only enqueue work; gs_create and gs_solve synchronise that stream.
 * A context is not thread-safe; use one context per stream.
 *
 * Errors: every call returns a gs_status; no exception crosses the ABI.  GS_EINVAL for bad
 * arguments (null pointers, sizes, unsupported dim, non-coarsenable mesh), GS_ECUDA when a
 * CUDA call fails (gs_last_error() gives the CUDA message), GS_ENOCONV when FGMRES stops at
 * max_iter or cannot reach tol (the best iterate and its residual are still written),
 * GS_EBREAKDOWN on a non-finite residual (NaN/Inf inputs).
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_ctx gs_ctx; /* opaque; level hierarchy + Krylov workspace */

typedef enum {
  GS_OK = 0,
  GS_EINVAL = 1,
  GS_ENOMEM = 2, /* workspace smaller than gs_footprint_bytes() */
  GS_ECUDA = 3,
  GS_ENOCONV = 4,
  GS_EBREAKDOWN = 5, /* a non-finite right-hand side, initial guess, residual or Krylov vector */
  GS_ETIMEOUT = 6,   /* a kernel's bounded wait for its staged data (an mbarrier of the bulk copies
                        of the 2D strip kernel) gave up after about a second; the launch completed
                        with unusable results.  Reported by gs_solve / gs_solve_A for any launch of
                        the context since the previous report. */
  GS_EBUSY = 7 /* batching engine: every slot is occupied */
} gs_status;

/* Dirichlet face bits */
#define GS_FACE_XM 1u
#define GS_FACE_XP 2u
#define GS_FACE_YM 4u
#define GS_FACE_YP 8u
#define GS_FACE_ZM 16u
#define GS_FACE_ZP 32u

typedef struct {
  int dim;                  /* 2 or 3 */
  int n[3];                 /* cells per axis on the FINEST level (n[2] ignored for dim 2) */
  double len[3];            /* domain extent per axis; origin at 0 */
  const uint8_t* cell_void; /* HOST array of N_c flags (1 = obstacle cell, excluded) or NULL */
  uint32_t dirichlet_faces; /* GS_FACE_* bits; faces without a bit are do-nothing (natural) */
} gs_mesh;

typedef struct {            /* zero-initialised = defaults */
  int cheb_degree;          /* k_A of Cheb(A, diag A, k_A); 0 -> 4 (Table NS-solver-parameters-1) */
  int smooth_steps;         /* Chebyshev calls before and after the coarse correction; 0 -> 1 */
  int restart;              /* FGMRES restart length m; 0 -> 50 */
  int max_iter;             /* total FGMRES iterations; 0 -> 1000 */
  int mg_precision;         /* 0 or 32: V-cycle + Schur step in FP32; 64: all FP64 */
  int schur_degree;         /* Chebyshev steps for S^{-1}; 0 -> 4 */
  int lanczos_steps;        /* eigenvalue-estimate steps per level; 0 -> 12 */
  int seed;                 /* SplitMix64 seed of the Lanczos start vectors */
  int coarse_mode;          /* 0: exact dense FP64 solve on level 0 (default);
                               1: Chebyshev smoothing only on level 0 (for meshes whose coarsest
                                  level is too large for a dense factorisation, e.g. 1280 x 210) */
  int schur_kind;           /* 0: Cahouet-Chabard when alpha > 0, else pressure mass (default);
                               1: 1/eta-weighted pressure mass M_p(1/eta) only;
                               2: Cahouet-Chabard S^{-1} ~ M_p(1/eta)^{-1} + alpha K_p^{-1}, K_p the
                                  Q1 pressure Laplacian (p = 0 on faces without a velocity
                                  Dirichlet condition), inverted by one multigrid V-cycle */
  int orth;                 /* 0 (default) or 2: CGS2 through the Gram matrix G = V^T V of the cycle:
                                  one pass over V for h1 = V^T w and the newest column of G, the
                                  coefficients c = h1 + (h1 - G h1) (CGS2's coefficients
                                  h1 + V^T (w - V h1) in exact arithmetic), one update pass w -= V c;
                                  3 instead of 4 FP64 FMAs per basis entry;
                               1: second pass only when the new vector's norm drops below
                                  1/sqrt(2) of its value before the projection (single solves
                                  only: the engine needs a fixed number of passes);
                               3: CGS2 with an explicit second pass (three passes over V) */
  int graphs;               /* 0: replay the preconditioner's fixed launch sequence as a CUDA graph
                                  captured at its second application (default); 1: plain launches */
  int plap_degree;          /* Chebyshev degree of the pressure-Laplacian V-cycle of the
                               Cahouet-Chabard term; 0 -> 2 */
  int krylov_fp64;          /* 0 (default) or 1: FGMRES basis V and the Gram-Schmidt products and
                                  updates in IEEE FP64;
                               2: basis stored as double-float pairs (hi + lo, ~48 significant
                                  bits, the same 8 bytes), Gram-Schmidt products on the FP32 pipes
                                  with FP64 sums of the partial results */
  int tile_autotune;        /* 2D meshes: 0 -> at gs_create, time each compiled variant of the
                                  velocity-block kernel on every level (cell tiles of 32 x 16,
                                  32 x 17, 32 x 8 evaluated cells; the strip kernel, 31-cell column
                                  strips marching up row segments) and keep the fastest (default);
                                  1 / 2 / 3 -> always the 32 x 16 / 32 x 17 / 32 x 8 tile; 4 -> always
                                  the strip kernel (the FP64 saddle operator then uses 32 x 8 tiles);
                                  5 -> by size, the strip kernel on levels of at least 32,768 cells
                                  and 32 x 8 tiles below (no timing at gs_create).
                               3D meshes: 0 -> time the cell tiles of 8 x 8 x 8 and 8 x 8 x 4
                                  evaluated cells per level and keep the faster (default);
                                  2 -> always 8 x 8 x 4; any other value -> always 8 x 8 x 8.
                                  Every variant sums a node's cell contributions in the same order,
                                  so the results do not depend on the choice. */
  int deflate;              /* 1: rigid-body deflation of stiff inclusions in the V-cycle's finest
                                  level (not part of the paper's method; for stiff inclusions
                                  smaller than a coarse cell, whose near-rigid motions no coarse
                                  level represents): inclusions = node-connected components of
                                  cells with eta >= sqrt(eta_min eta_max) when eta_max >= 1e3
                                  eta_min, at most 256; Z = their rigid motions on their cells'
                                  nodes; the finest level adds Z (Z^T A Z)^-1 Z^T r to its coarse
                                  correction.  0: off (default). */
  int precond_kind;         /* 0: block upper-triangular preconditioner (velocity V-cycle + Schur
                                  approximation, the default);
                               1: the preconditioner of Sec. 4 itself: mono_cycles V-cycles of
                                  multigrid on the whole saddle matrix M_j = [A_j B_j^T; B_j 0] with
                                  mono_smooth steps of the block smoother of Eq. "smoother",
                                  K_j = [Ahat B^T; B B Ahat^{-1} B^T - Shat]^{-1}, before and after
                                  the coarse correction; Ahat^{-1} = Cheb(A, diag A, cheb_degree);
                                  Shat^{-1} = ChebMINRES(1, 1): one MINRES step on
                                  S = B Ahat^{-1} B^T preconditioned by one Chebyshev step with
                                  diag(B diag(A)^{-1} B^T) (n_S = k_S = 1, Table
                                  NS-solver-parameters-1); dense saddle solve on level 0 (or, with
                                  coarse_mode = 1, mono_smooth smoothing steps).  smooth_steps,
                                  schur_*, plap_degree and deflate do not apply. */
  int mono_smooth;          /* m of precond_kind 1; 0 -> 2 (Table NS-solver-parameters-1) */
  int mono_cycles;          /* n of precond_kind 1; 0 -> 1 */
  int corrector;            /* 1: reserve the per-level fields of the corrector stage (see
                               gs_set_corrector); 0 -> none */
} gs_options;

/* Bytes of device workspace gs_create needs for this mesh / levels / options (0 on bad input):
 * the multigrid hierarchy of Sec. 4 and the FGMRES basis of Sec. 5 ("Linear solver settings"). */
size_t gs_footprint_bytes(const gs_mesh* mesh, int levels, const gs_options* opts);

/* Build the hierarchy of the generalized Stokes problem alpha u - div(2 eta eps(u)) + grad p = f,
 * div u = g_p (Sec. 3.1.2, Eq. "ggce:implicit"; Q2-Q1 spaces of Eq. "spaces"; eta per cell as in the
 * viscosity splitting, Eq. "viscosity-splitting"; nested meshes of Sec. 4): levels l = 0
 * (coarsest, n / 2^(levels-1) cells per axis) ... levels-1 (finest, mesh->n).  eta_per_cell: HOST
 * array of N_c positive finite values (finest level, cell-lexicographic, x fastest); coarse eta =
 * mean of the active children.  alpha >= 0 (alpha = rho / (gamma tau)).  opts may be NULL.
 * stream: cudaStream_t or NULL.  workspace: device pointer of at least gs_footprint_bytes() bytes,
 * owned by the caller and used by the context until gs_destroy.  On success *out receives the
 * context; on GS_EINVAL (bad sizes, non-finite eta, too small a workspace) or GS_ECUDA nothing is
 * kept (gs_last_error() says why). */
gs_status gs_create(const gs_mesh* mesh, int levels, const double* eta_per_cell, double alpha,
                    const gs_options* opts, void* stream, void* workspace, size_t workspace_bytes,
                    gs_ctx** out);

/* gs_create with alpha = rho / (gamma tau) given per cell (the solid's density differs from the
 * fluid's, e.g. rho_s = 10 rho_f in FSI2i, Sec. 5): the mass term of A becomes
 * sum_K alpha_K int_K phi_i phi_j.  alpha_per_cell: HOST array of N_c finite values >= 0 (finest
 * level; coarse alpha = mean of the active children, like eta).  The Cahouet-Chabard Schur term
 * becomes K_p(1/alpha)^{-1}, the pressure Laplacian with cell weights 1/alpha_K, applied as
 * abar V(K_p^w) with w_K = abar / alpha_K and abar = max alpha_K (cells with alpha_K = 0 get
 * w_K = 1); it is active when abar > 0 (schur_kind 0).  Everything else as gs_create; the
 * workspace size is the same (gs_footprint_bytes reserves the per-cell arrays). */
gs_status gs_create_ex(const gs_mesh* mesh, int levels, const double* eta_per_cell, const double* alpha_per_cell,
                       const gs_options* opts, void* stream, void* workspace, size_t workspace_bytes,
                       gs_ctx** out);

/* y = K x on the finest level, FP64 (Eq. "stokes-discrete-block" with constraints; the blocks
 * are the forms of Eq. "form_a_j" and Eq. "form_b").  x, y: device, length N, must not alias.
 * GS_EINVAL on a null pointer. */
gs_status gs_vmult(gs_ctx* ctx, const double* x, double* y);

/* y = A x (velocity block, constrained) on the finest level.  fp32 = 0: x, y are double*;
 * fp32 = 1: x, y are float* (the operator the FP32 multigrid uses).  Length d*N_v. */
gs_status gs_vmult_A(gs_ctx* ctx, const void* x, void* y, int fp32);

/* z = V(r): one velocity V-cycle of Sec. 4 (Chebyshev-Jacobi smoothing of degree k_A, Table
 * "NS-solver-parameters-1"; FP64 in/out, inside in the context's mg_precision).  Length d*N_v,
 * device.  Constrained rows act as identity rows inside the smoother and never couple to free
 * entries; the block preconditioner overwrites them with r.  GS_EINVAL on a null pointer. */
gs_status gs_vcycle(gs_ctx* ctx, const double* r, double* z);

/* Solve K x = rhs with FGMRES (Sec. 5, "Linear solver settings") preconditioned as in Sec. 4, to
 * ||rhs - K x|| / ||rhs|| <= tol (explicit residual).  x: in = initial guess, out = solution
 * (device, length N).  *iterations and *rel_residual receive the FGMRES iteration count and the
 * explicit relative residual (either may be NULL).  Returns GS_ENOCONV if tol was not reached
 * within max_iter (x holds the last iterate), GS_EBREAKDOWN on a non-finite right-hand side,
 * initial guess or Krylov scalar, GS_ETIMEOUT when a kernel's bounded wait gave up (the context
 * stays usable). */
gs_status gs_solve(gs_ctx* ctx, const double* rhs, double* x, double tol, int* iterations,
                   double* rel_residual);

/* Mesh-extension solve (Eq. "extenstion"; Sec. 5: CG preconditioned by a matrix-free multigrid
 * with a fourth-order Chebyshev smoother): A x = rhs on the velocity block of the finest level,
 * where A is this context's velocity block (create it with alpha = 0 and eta = mu_A / 2 per cell:
 * A then carries int mu_A eps(u) : eps(v); solid cells are obstacle cells whose nodes hold the
 * solid displacement as Dirichlet data).  Flexible (Polak-Ribiere) preconditioned CG, one velocity
 * V-cycle (gs_vcycle, the context's mg_precision) per iteration, FP64 vectors; stops when
 * ||rhs - A x|| / ||rhs|| <= tol or after max_iter iterations.  rhs: device, d*N_v, holding the
 * Dirichlet values on constrained entries and -A_raw g elsewhere (the velocity part of
 * gs_lift_rhs with f = 0).  x: device, d*N_v; in = initial guess on free entries (constrained
 * entries are overwritten with rhs), out = solution.  Uses the context's Krylov workspace (not
 * concurrently with gs_solve on the same context).  GS_ENOCONV / GS_EBREAKDOWN leave the last
 * iterate in x; *iterations and *rel_residual (either may be NULL) receive the CG iteration count
 * and the explicit relative residual. */
gs_status gs_solve_A(gs_ctx* ctx, const double* rhs, double* x, double tol, int* iterations,
                     double* rel_residual);

/* Right-hand side of Eq. "stokes-discrete-block" with the Dirichlet data lifted (Sec. 3.1.2):
 * rhs = [M_u f_u ; M_p f_p] - K_raw g on free entries, rhs = g on constrained entries, where
 * f is a nodal load field (full layout) and g holds Dirichlet values (full layout; only its
 * constrained entries are used).  K_raw is the saddle matrix without constraint elimination.
 * All pointers device, length N; rhs must not alias f or g. */
gs_status gs_lift_rhs(gs_ctx* ctx, const double* f, const double* g, double* rhs);

/* Switch the context to the corrector stage of the time step (Sec. 3.1.2, Eq. "v_star"): the
 * convective velocity is the unknown and v° = v# - w# is given, so the velocity block becomes
 *   A_c = alpha M + 2 eta eps:eps + rho C(v°) + rho S(v°, r),
 *   C: (phi_i, (v° . grad) phi_j) on each component,  S: the streamline diffusion of Eq. "a_stab",
 *   sum_K r_K ((v° . grad) phi_i, (v° . grad) phi_j)_K with the Brooks-Hughes parameter
 *   r_K = h_K / (2 |v°|_K p1) (coth Pe_K - 1 / Pe_K), Pe_K = rho |v°|_K h_K / (2 eta_K p1), p1 = 2,
 *   |v°|_K at the cell centre, h_K the cell diameter, r_K = 0 where Pe_K < 1;
 * both integrated with the 3-point Gauss rule per axis.  Every later gs_vmult / gs_vmult_A / gs_solve /
 * gs_vcycle / gs_lift_rhs uses A_c (non-symmetric; B and B^T unchanged): the V-cycle smooths with
 * A_c, its Chebyshev bounds come from 12 Lanczos steps on the symmetric part (A_c + A_c^T) / 2, the
 * coarse levels take v° by injection (coarse node I = fine node 2 I) and the dense coarse solve
 * factors A_c,0 (Gauss-Jordan; its symmetric part is positive definite).
 * vcirc: host, d N_v doubles of the finest level (component-blocked, like a velocity vector);
 * With the saddle-point multigrid (precond_kind = 1) every level's velocity block is A_c and the
 * Schur solve of the block smoother is ChebBiCGStab(1, 1) (one BiCGStab step preconditioned by
 * diag(B diag(A_c)^-1 B^T)^-1, shadow residual = the right-hand side) in place of ChebMINRES.
 * NULL switches back to the predictor stage (rho ignored).  rho >= 0.  2D and 3D meshes, contexts
 * created with gs_options.corrector = 1, no deflation; synchronises the context stream (setup work:
 * diagonals, Lanczos, coarse factorisations).  Not while the context is in a batching engine. */
gs_status gs_set_corrector(gs_ctx* ctx, const double* vcirc, double rho);

/* Solve `count` independent systems; ctxs[i] with rhs[i] -> x[i] (device pointers).
 * iterations / rel_residuals: host arrays of `count` entries or NULL.  Returns the first
 * non-OK status (all systems are still attempted).  When every context uses a fixed number of
 * Gram-Schmidt passes (orth != 1) and no profiling, the systems run together through a batching
 * engine on ctxs[0]'s stream (one launch per kernel per FGMRES iteration for all of them, see
 * gs_engine_*).  Otherwise they run one after the other through gs_solve. */
gs_status gs_batch_solve(gs_ctx* const* ctxs, int count, const double* const* rhs,
                         double* const* x, double tol, int* iterations, double* rel_residuals);

/* ---- level operators (the individual kernels of the path, for checking and profiling) ---- */
typedef enum {
  GS_OP_A = 0,           /* y = A_l x            (velocity, constrained)            */
  GS_OP_RESIDUAL_A = 1,  /* y = b - A_l x        (aux = b)                          */
  GS_OP_DIAG_A = 2,      /* y = diag(A_l)        (x ignored; velocity length)       */
  GS_OP_SMOOTH = 3,      /* y = Cheb(A_l, diag, k_A) from x0 = aux (NULL -> 0), rhs x */
  GS_OP_RESTRICT = 4,    /* y (level l-1) = P_l^T x (level l)                       */
  GS_OP_PROLONGATE = 5,  /* y (level l) += P_l x (level l-1)                        */
  GS_OP_B = 6,           /* y (pressure, N_p) = B x (velocity)      finest level only */
  GS_OP_BT = 7,          /* y (velocity) = B^T x (pressure)         finest level only */
  GS_OP_SCHUR_MASS = 8,  /* y = M_p(1/eta) x     (pressure)         finest level only */
  GS_OP_SCHUR_INV = 9,   /* y = Cheb(M_p(1/eta), diag, schur_degree) x, from 0       */
  GS_OP_COARSE = 10,     /* y = A_0^{-1} x       (level 0, dense FP64)               */
  GS_OP_PRECOND = 11,    /* y = P^{-1} x         (full block preconditioner)         */
  GS_OP_A_RAW = 12,      /* y = A_l x without constraint elimination                 */
  GS_OP_PLAP = 13,       /* y = K_p,l x          (pressure Laplacian of level l)     */
  GS_OP_PLAP_INV = 14,   /* y = V_p(x) ~ K_p^{-1} x (finest level, MG precision)    */
  GS_OP_PRESTRICT = 15,  /* y (level l-1) = P_p,l^T x (Q1 restriction)               */
  GS_OP_PPROLONGATE = 16,/* y (level l) += P_p,l x (level l-1) (Q1 interpolation)    */
  /* precond_kind = 1 only; "level vector" = [u (d N_v,l) | p (N_p,l)] of level l, MG precision: */
  GS_OP_SCHUR_DIAG = 17, /* y = diag(B_l diag(A_l)^{-1} B_l^T) (pressure, N_p,l; 0 on
                            constrained nodes), the ChebMINRES preconditioner of Sec. 4 */
  GS_OP_SADDLE_SMOOTH = 18, /* y = K_j x: one block-smoother application (Eq. "smoother") to
                            the level vector x; level >= 1 (or level 0 with coarse_mode 1) */
  GS_OP_SADDLE_VCYCLE = 19, /* y = V_l(x): one saddle-point V-cycle on level l, level vectors */
  GS_OP_SADDLE_COARSE = 20, /* y = M_0^{-1} x: dense saddle solve of level 0 (FP64 level
                            vectors, free unknowns; constrained entries of y are 0) */
  GS_OP_CHEB_STEP = 21,  /* one fused Chebyshev-Jacobi step on the caller's vectors (the kernel
                            the smoother of Sec. 4 launches k_A - 1 times per call): with
                            aux = [b | d | D^-1] (3 x d N_v,l contiguous entries), r = b - A_l x,
                            d <- c1 d + c2 D^-1 r (in place in aux), y = x + d, where c1, c2 are
                            the coefficients of the level's second Chebyshev step (Saad's
                            recurrence on [lambda_hi / 15, lambda_hi]); x and y must not alias;
                            levels with Chebyshev bounds only (not level 0 with the dense
                            coarse solve).  Lets a caller time the step on vectors of its own,
                            e.g. several copies that together exceed L2. */
  GS_OP_WAIT_PROBE = 22  /* fault-path check (no paper counterpart): one CTA waits, with the
                            bounded wait of the staged kernels, on an mbarrier phase that nothing
                            completes; after about a second it gives up and sets the context's
                            error word, so the next gs_solve / gs_solve_A returns GS_ETIMEOUT (and
                            clears it).  x, y, aux ignored (y must be non-NULL). */
} gs_op;

/* Apply one operator of level `level` (0 = coarsest).  prec = 64: x, y, aux are double*;
 * prec = 32: float* (GS_OP_COARSE, GS_OP_SADDLE_COARSE and GS_OP_PRECOND take double* always;
 * the saddle operators 17-19 need prec = the context's mg_precision).  Enqueue only. */
gs_status gs_apply_level(gs_ctx* ctx, int level, gs_op op, int prec, const void* x, void* y,
                         const void* aux);

/* Introspection: sizes and eigenvalue bounds. */
typedef struct {
  int levels;
  int dim;
  long long n_total;       /* N of the finest level */
  long long n_u;           /* d * N_v of the finest level */
  long long n_p;           /* N_p of the finest level */
  int pressure_nullspace;  /* 1 if every face is Dirichlet */
  int last_iterations;
  double last_rel_residual;
  double lambda_max[16];   /* Chebyshev upper bound (1.2 x Lanczos estimate) per level */
  long long level_n_u[16];
  int coarse_free;         /* unknowns of the dense coarse solve */
  size_t footprint_bytes;
  long long kernel_launches; /* kernels this library has launched in this process (all contexts) */
  int schur_cc;            /* 1 if the Cahouet-Chabard term is active */
  int pressure_coarse_free;/* unknowns of the dense coarse pressure-Laplacian solve */
  double plambda_max[16];  /* Chebyshev upper bound of the pressure Laplacian per level */
  int tile_rows[16];       /* 2D: evaluated cell rows per tile chosen for each level's multigrid kernels
                              (0: the strip kernel); 3D: evaluated cell layers along z per 8 x 8 x k
                              tile (8 or 4) */
  int saddle_tile_rows;    /* the same for the FP64 saddle operator */
  int deflation_inclusions;/* stiff inclusions in the deflation space (option deflate) */
  int deflation_modes;     /* rigid modes kept (modes vanishing on unconstrained nodes dropped) */
  int precond_kind;        /* the preconditioner in use (gs_options.precond_kind) */
  int saddle_coarse_free;  /* unknowns of the dense coarse saddle solve (precond_kind 1) */
} gs_info;
gs_status gs_get_info(const gs_ctx* ctx, gs_info* out);

/* Per-kernel-class timing of the work a context enqueues (tracing aid, no paper counterpart in
 * the method itself; the paper reports time per unknown, Sec. 5).  gs_profile(ctx, 1) starts
 * recording a CUDA event pair around every launch of gs_solve / gs_vcycle / gs_vmult work;
 * gs_profile(ctx, 0) stops.  gs_profile_read synchronises the stream and fills up to `max`
 * entries (one per class: launches and summed device milliseconds); returns the count. */
typedef struct {
  const char* name;        /* static string */
  long long launches;
  double total_ms;
} gs_kernel_stat;
gs_status gs_profile(gs_ctx* ctx, int enable);
int gs_profile_read(gs_ctx* ctx, gs_kernel_stat* out, int max);
/* The same, restricted to the launches recorded on multigrid level `level` (0 = coarsest; the
 * velocity and pressure-Laplacian cycles and the saddle-point cycle tag their launches with
 * the level they run on; -1 selects the launches tied to no level: FGMRES kernels, the FP64
 * saddle operator).  Lets a caller weight a class's algorithmic bytes by level. */
int gs_profile_read_level(gs_ctx* ctx, int level, gs_kernel_stat* out, int max);

/* Coarse-level solve y = A_0^{-1} b that allocates nothing and uses no workspace scratch.
 * The paper has no counterpart: this is a service entry point for callers that cannot
 * allocate device memory at the point of the call -- for example a multigrid code that uses
 * this library's dense coarse solve as its bottom solver from inside a CUDA-graph capture or
 * a latency-critical loop where cudaMalloc (and any allocating library routine) is not
 * allowed, and that must not touch the context workspace another stream may be using.  It
 * computes exactly what gs_apply_level(ctx, 0, GS_OP_COARSE, 64, b, y, NULL) computes.
 * b, y: device, length d*N_v of level 0, FP64, must not alias.  The gathered right-hand side
 * lives in one file-scope device array of GS_NOALLOC_COARSE_MAX doubles (128 KiB), which every
 * GPU that loads the library holds until the process exits; contexts whose coarse level has
 * more free unknowns than that are rejected with GS_EINVAL (see gs_get_info().coarse_free), as
 * are contexts built with coarse_mode = 1.  Call it with the context's device current.  The
 * first call on each device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array and it keeps the last
 * call's contents (every call rewrites the entries it reads, so nothing needs clearing): calls
 * that overlap on the GPU -- on different streams, or from different threads -- race.  Enqueue
 * only, on the context's stream. */
#define GS_NOALLOC_COARSE_MAX 16384
gs_status gs_coarse_solve_noalloc(gs_ctx* ctx, const double* b, double* y);

/* ---- Batching engine (many solves in lockstep; continuous batching) --------------------------
 * The paper solves one system at a time; this engine runs many independent solves together on
 * one GPU.  Each solve is a context of its own (hierarchy and Krylov state resident on the
 * device).  gs_engine_step advances every solve in the engine by one FGMRES iteration (right
 * preconditioned, restart m, classical Gram-Schmidt twice, Sec. 5): the launches all solves
 * need for that iteration are merged so that each kernel runs once for all of them (a work
 * list of (solve, block) pairs), the block preconditioners of all solves replay as one captured
 * CUDA graph, and the host synchronises once per step.  Each solve runs the launches gs_solve
 * issues for it (same kernel bodies, arguments and order) through the batched entry points: its
 * result is bitwise the same whoever else is in the engine, and agrees with gs_solve's to
 * rounding (the single-instance entry points are compiled separately, and the compiler may
 * contract multiply-adds differently there).  Solves join with gs_engine_add and leave when they
 * finish, between steps.
 *
 * gs_engine_create: max_slots solves at most at a time; max_restart >= the restart length of
 * every context added (0: 50); stream: cudaStream_t or NULL; all engine work is enqueued there.
 * The engine allocates its own staging buffers (device and pinned host memory, a few hundred
 * bytes per slot plus the argument tables of one step).
 * gs_engine_add: ctx must use orth != 1 and no profiling and must not be in the engine already;
 * rhs, x: device, full length, x holds the initial guess and receives the solution; they and the
 * context stay in use until the solve is reported by gs_engine_poll.  Synchronises ctx's stream.
 * GS_EBUSY when every slot is taken.
 * gs_engine_step: one iteration of every solve in the engine; *active (may be NULL) = solves
 * still running afterwards.  A failing solve (GS_ENOCONV, GS_EBREAKDOWN) finishes with that
 * status; the return value reports engine failures only (GS_ECUDA).
 * gs_engine_poll: copies up to max finished solves (oldest first) and forgets them.
 * t_added / t_done: host steady-clock seconds at gs_engine_add and at the end of the step that
 * finished the solve. */
typedef struct gs_engine gs_engine;
typedef struct {
  long long tag;
  gs_status status;
  int iterations;
  double rel_residual;
  double t_added, t_done;
} gs_engine_result;
typedef struct {
  long long steps;
  long long batched_launches; /* per-step merged launches (outside the plan graph) */
  long long plan_builds;
  long long plan_kernels;     /* kernels in the current plan graph */
  long long completed;
} gs_engine_stats;
gs_status gs_engine_create(int max_slots, int max_restart, void* stream, gs_engine** out);
gs_status gs_engine_add(gs_engine* eng, gs_ctx* ctx, const double* rhs, double* x, double tol, long long tag);
gs_status gs_engine_step(gs_engine* eng, int* active);
int gs_engine_poll(gs_engine* eng, gs_engine_result* out, int max);
int gs_engine_active(const gs_engine* eng);
gs_status gs_engine_get_stats(const gs_engine* eng, gs_engine_stats* out);
void gs_engine_destroy(gs_engine* eng);

/* Change the stream work is enqueued on. */
gs_status gs_set_stream(gs_ctx* ctx, void* stream);

void gs_destroy(gs_ctx* ctx);
const char* gs_strerror(gs_status s);
const char* gs_last_error(void); /* thread-local text of the last GS_ECUDA / GS_EINVAL cause */

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
