/*
 * ldgmg — GB300-native multigrid for high-order LDG discretisations.
 *
 * C ABI of the hot path of the multigrid solvers in arXiv 2412.12506 (Saye,
 * "A comparative study of efficient multigrid solvers for high-order local
 * discontinuous Galerkin methods"): the element-block-sparse LDG operator,
 * block-Jacobi and balanced block-SAI smoothers, the per-level residual,
 * restriction and prolongation of the V-cycle (Algorithm 1), the bottom
 * pseudo-inverse, and multigrid-preconditioned CG; and the same hierarchy for
 * the LDG Stokes saddle-point system (Sec. 3) with restarted GMRES.
 *
 * Conventions shared by every call
 *   - Mesh: uniform periodic Cartesian n^dim mesh of the unit square/cube
 *     (dim = 2 or 3), h = 1/n.  Elements are numbered lexicographically with x
 *     fastest: e = ix + n*iy (+ n*n*iz).
 *   - Basis: tensor-product orthonormal Legendre modes (Sec. 2.1), b = (p+1)^dim
 *     coefficients per element, mode m = kx + (p+1)*ky (+ (p+1)^2*kz).
 *     A Stokes operator (ldgmg_assemble_stokes) has dim + 1 fields per element
 *     in the order u_1, .., u_dim, p, each with (p+1)^dim modes: block size
 *     b = (dim+1)(p+1)^dim, dof (field f, mode m) at f*(p+1)^dim + m.
 *   - Vector layout: a vector is N*b contiguous values [element][mode]; calls
 *     taking nrhs > 1 right-hand sides take nrhs such vectors one after another
 *     ([rhs][element][mode]).  FP64 vectors are double; V-cycle level vectors
 *     are double (FP64 hierarchy) or float (FP32/BF16 hierarchy); batched level
 *     vectors (ldgmg_level_apply_batched) are float [element][rhs][mode].
 *   - Pointers named *_dev are device pointers owned by the caller; *_host are
 *     host pointers owned by the caller.  Handles (ldgmg_op, ldgmg_hier) are
 *     opaque; the library owns every allocation made behind them and releases
 *     it in the matching *_free.
 *   - Every call takes a cudaStream_t passed as void* (NULL = legacy default
 *     stream) and enqueues its work on it; calls that return host results
 *     synchronise that stream.
 *   - Errors: every call returns an ldgmg_status and never aborts, traps or
 *     exits.  On failure ldgmg_last_error() returns a thread-local message.
 *   - Threading: a handle must not be used from two host threads at once.
 */
#ifndef LDGMG_H
#define LDGMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LDGMG_OK = 0,
  LDGMG_EINVAL = 1,        /* bad argument (null pointer, size, NaN/Inf input) */
  LDGMG_ENOMEM = 2,        /* device or host allocation failed */
  LDGMG_ECUDA = 3,         /* a CUDA runtime / library call failed */
  LDGMG_ENOTCONV = 4,      /* Krylov solve hit max_iter; the iterate is still written */
  LDGMG_ETIMEOUT = 5,      /* a bounded device wait gave up */
  LDGMG_EUNSUPPORTED = 6   /* valid request outside what this build implements */
} ldgmg_status;

enum { LDGMG_JACOBI = 0, LDGMG_SAI = 1, LDGMG_GS = 2 };   /* smoother kind */
enum { LDGMG_FORM_B1 = 0, LDGMG_FORM_BT = 1 };            /* SAI smoother form, Eqs. B1 / BT */
enum { LDGMG_FP64 = 0, LDGMG_FP32 = 1, LDGMG_BF16 = 2, LDGMG_FP16 = 3 };   /* V-cycle precision */
enum { LDGMG_MAT_A = 0, LDGMG_MAT_B = 1, LDGMG_MAT_BT = 2, LDGMG_MAT_D = 3 }; /* level matrices */
enum { LDGMG_OUTER_AUTO = 0, LDGMG_OUTER_FP64 = 1, LDGMG_OUTER_DF = 2 };  /* batched outer apply */
enum { LDGMG_KRYLOV_AUTO = 0, LDGMG_KRYLOV_CG = 1, LDGMG_KRYLOV_GMRES = 2, LDGMG_KRYLOV_FGMRES = 3 };
                                                          /* outer Krylov method */

typedef struct {
  int dim;          /* 2 or 3 */
  int n;            /* elements per axis, >= 1 */
  int periodic;     /* must be 1 (periodic boundaries); 0 -> LDGMG_EUNSUPPORTED */
} ldgmg_mesh;

typedef struct {
  int smoother;          /* LDGMG_JACOBI (Sec. 2.3.1), LDGMG_SAI (Sec. 2.3.3), or LDGMG_GS:
                            multi-coloured block Gauss-Seidel, undamped, greedy colouring of
                            A's block pattern (Sec. 2.3.2; pre_form / post_form B1 = forward,
                            BT = backward colour order) */
  int sai_level;         /* ell: B has the block pattern of A^ell (Sec. 2.3.3); 0..2 */
  int balance;           /* 1: balanced SAI, alpha_i = ||A_ii||_F^{-1/2} (Sec. 2.3.3) */
  int nu1, nu2;          /* pre / post sweeps of Algorithm 1 (paper: 3 / 3, Sec. 2.2) */
  double omega;          /* Jacobi damping (paper: 0.8, Eq. Jsmooth) */
  int pre_form;          /* SAI form of the pre-sweeps  (B1 = Eq. B1) */
  int post_form;         /* SAI form of the post-sweeps (BT = Eq. BT); B1/BT is symmetric */
  int vcycle_precision;  /* V-cycle matrix storage, FP32 accumulate: LDGMG_FP64, LDGMG_FP32,
                            LDGMG_BF16, or LDGMG_FP16 (each level matrix scaled by a power of
                            two so its largest entry is in [2^14, 2^15)) */
  int max_iter;          /* Krylov iteration cap for ldgmg_solve */
  int max_rhs;           /* right-hand sides per call, 1..128 (scalar operators; Stokes: 1).
                            With b = 16 or 64, vcycle_precision LDGMG_BF16 (BF16 blocks) or
                            LDGMG_FP32 (FP32 blocks split into two BF16 parts on the fly) and
                            Jacobi or SAI, > 1 builds the batched tensor-core hierarchy; else
                            the CUDA-core kernels run one grid row per right-hand side */
  int outer_apply;       /* operator apply of the outer CG of reduced-precision or batched
                            hierarchies with b = 16 or 64: LDGMG_OUTER_FP64, or
                            LDGMG_OUTER_DF = double-FP32 arithmetic (FP32 pairs, ~2^-44 of
                            sum |a x|, on the fast FP32 pipes), or LDGMG_OUTER_AUTO = DF.
                            With DF and max mu / min mu > 10 (cancellation across the jump
                            costs DF accuracy) CG runs to 1e-8 of the residual it starts
                            from and is restarted from the FP64 residual b - A x until tol
                            is met (iterative refinement).  FP64 hierarchies always use
                            FP64.  The final residual that ldgmg_solve reports is always
                            computed in FP64. */
  int krylov;            /* ldgmg_solve's method: LDGMG_KRYLOV_CG (SPD scalar problems),
                            LDGMG_KRYLOV_GMRES (left preconditioned, the paper's form; Stokes:
                            A and V are symmetric indefinite, Sec. 3.4), LDGMG_KRYLOV_FGMRES
                            (flexible, right preconditioned, stops on the true residual), or
                            LDGMG_KRYLOV_AUTO = CG for scalar operators; for Stokes GMRES with
                            an FP64 V-cycle and FGMRES with a reduced-precision one */
  int restart;           /* GMRES restart length m, 1..200 (Krylov vectors kept on the device) */
  double zeta;           /* Stokes SAI balancing (Sec. 3.3); <= 0 takes Table tab:zeta for
                            (gamma, dim, p), 0.1 where the table has no entry */
} ldgmg_setup_opts;

typedef struct ldgmg_op ldgmg_op;
typedef struct ldgmg_hier ldgmg_hier;

/* Fill *o with the paper's defaults: SAI, ell = 1, balanced, nu1 = nu2 = 3,
 * omega = 0.8, B1 pre / BT post, FP64, max_iter = 200, max_rhs = 1,
 * outer_apply = LDGMG_OUTER_AUTO, krylov = LDGMG_KRYLOV_AUTO, restart = 50,
 * zeta = 0 (table). */
void ldgmg_default_opts(ldgmg_setup_opts* o);

/* Assemble the LDG Laplacian A = sum_a G_a^T M_mu G_a + E of Sec. 2.1 (display
 * after Eq. scalar3) on the device, FP64.
 *   mesh         uniform periodic mesh (see conventions).
 *   p            polynomial degree, 1 <= p <= 5 (b = (p+1)^dim must be one of
 *                4, 8, 9, 16, 25, 27, 36, 64).
 *   mu_host      host array of N = n^dim per-element coefficients (> 0, finite),
 *                or NULL for mu == 1.  Copied; the caller keeps ownership.
 *   tau0         penalty constant: tau_f = tau0 * min(mu_L, mu_U) / h (> 0).
 *   out          receives the handle; free with ldgmg_op_free.
 * Fluxes are viscosity-upwinded one-sided (Sec. 2.1): u_hat from the element with
 * the larger mu, from the lower element on ties.  Errors: EINVAL, EUNSUPPORTED,
 * ENOMEM, ECUDA. */
ldgmg_status ldgmg_assemble(const ldgmg_mesh* mesh, int p, const double* mu_host, double tau0,
                            ldgmg_op** out);

/* Assemble the LDG Stokes saddle-point operator of Sec. 3.1 (Eq. components)
 * on the device, FP64, block size b = (dim+1)(p+1)^dim with fields
 * (u_1, .., u_dim, p) per element:
 *   (u_f, u_g) = delta_fg (sum_a G_a^T M_mu G_a + E) + gamma G_g^T M_mu G_f
 *   (u_f, p) = -G_f^T M,   (p, u_g) = -M G_g,   (p, p) = -E_p
 * with G, M_mu, E those of ldgmg_assemble and M the unweighted mass.
 *   gamma        0: standard form, 1: stress form (Sec. 3.1).
 *   tau0         velocity penalty constant as in ldgmg_assemble (> 0).
 *   taup         pressure penalty: E_p = sum_faces tau_p int_f [p][q] with
 *                tau_p = taup * h / min(mu_L, mu_U) (>= 0; 0 disables it).
 *                The paper takes its values from [flame]; 0.05 puts the
 *                balanced E_p sub-block at 0.2-0.7 zeta as Sec. 3.3 reports.
 * The operator is symmetric indefinite; on the periodic mesh its kernel is the
 * constant velocities and the constant pressure (dim + 1 modes).  b must be a
 * supported block size (2D: p = 1, 2, 3; 3D: p = 1).  Errors: EINVAL,
 * EUNSUPPORTED, ENOMEM, ECUDA. */
ldgmg_status ldgmg_assemble_stokes(const ldgmg_mesh* mesh, int p, const double* mu_host, int gamma,
                                   double tau0, double taup, ldgmg_op** out);

/* Sizes of an assembled operator: N elements, b dofs per element, nnzb stored blocks. */
ldgmg_status ldgmg_op_info(const ldgmg_op* op, int64_t* N, int* b, int64_t* nnzb);

/* Device memory held by a handle: the operator (FP64 A, its double-FP32 copy
 * once a hierarchy asked for it, scratch) or a hierarchy (level matrices and
 * vectors, bottom pseudo-inverse, Krylov work space), in bytes.  Scratch used
 * only while a call runs is not included.  For HBM budgeting (e.g. admission
 * of requests by footprint). */
ldgmg_status ldgmg_op_device_bytes(const ldgmg_op* op, size_t* bytes);
ldgmg_status ldgmg_hier_device_bytes(const ldgmg_hier* h, size_t* bytes);

/* Launch shape chosen by the setup-time autotuner of the tensor-core apply
 * (batched hierarchies): CTAs per SM of the per-use kernel (0 when that
 * kernel is not tuned: every matrix runs the cached kernel below) and the
 * level-0 smoother apply's time with max_rhs right-hand sides at the chosen
 * shape (ms).  The apply's result does not depend on the shape. */
ldgmg_status ldgmg_hier_tuning(const ldgmg_hier* h, int* tc_ctas_per_sm, double* tc_ms);

/* The cached tensor-core apply of batched 2D hierarchies with b = 16 and
 * max_rhs <= 64 (one CTA per SM; rows in strips of `strip` element columns
 * walked along y; converted x_j kept in shared-memory slots): the autotuned
 * strip width (0 when the hierarchy does not use this kernel), the x slots
 * per CTA and the x_j loads per block row of one level-0 smoother apply
 * (each load reads x_j from HBM or L2 once). */
ldgmg_status ldgmg_hier_tc_schedule(const ldgmg_hier* h, int* strip, int* x_slots, double* loads_per_row);

/* Field structure: nfields = 1 (scalar) or dim + 1 (Stokes), field_b = (p+1)^dim
 * dofs per field and element (b = nfields * field_b). */
ldgmg_status ldgmg_op_fields(const ldgmg_op* op, int* nfields, int* field_b);

/* y = A x in FP64 (Sec. 2.3: y_i = sum_j A_ij x_j) for nrhs >= 1 stacked
 * vectors.  x_dev, y_dev: device arrays of N*b*nrhs doubles, must not overlap. */
ldgmg_status ldgmg_apply(ldgmg_op* op, const double* x_dev, double* y_dev, int nrhs, void* stream);

/* Remove the kernel component (constant functions, Sec. 2.2 "Bottom solver"):
 * v <- v - (c^T v / c^T c) c with c the coefficients of u == 1, for each of the
 * nrhs stacked vectors; for a Stokes operator, once per field (constant
 * velocity components and constant pressure).  In place. */
ldgmg_status ldgmg_project_kernel(ldgmg_op* op, double* v_dev, int nrhs, void* stream);

/* Build the multigrid hierarchy (Sec. 2.2): levels n, n/2, ... while n is even
 * and > 1, coarse operators by operator coarsening, the smoother of every
 * level but the last (block-Jacobi inverse blocks or balanced SAI by
 * Householder-QR least squares), and the bottom pseudo-inverse from a
 * symmetric eigendecomposition.  Everything stays resident on the device.
 * The op must outlive the hierarchy.  Errors: EINVAL, EUNSUPPORTED (e.g. a
 * rank-deficient SAI least-squares column), ENOMEM, ECUDA. */
ldgmg_status ldgmg_setup(ldgmg_op* op, const ldgmg_setup_opts* opts, void* stream,
                         ldgmg_hier** out);

/* Number of levels and, for level l, n, N, b and stored blocks of A_l and of the
 * smoother matrix (B_l for SAI, D_l for Jacobi; 0 on the bottom level). */
ldgmg_status ldgmg_hier_info(const ldgmg_hier* h, int level, int* nlevels, int* n, int64_t* N,
                             int* b, int64_t* nnzb_A, int64_t* nnzb_S);

/* x = V b: one V-cycle of Algorithm 1 with zero initial guess (the
 * preconditioner V of Sec. 2.2), FP64 in and out; internally in the
 * hierarchy's precision.  b_dev, x_dev: nrhs stacked vectors (nrhs <=
 * max_rhs of the setup), may not overlap. */
ldgmg_status ldgmg_vcycle(ldgmg_hier* h, const double* b_dev, double* x_dev, int nrhs,
                          void* stream);

/* Solve A x = rhs from x0 = 0 with the V-cycle as preconditioner.
 * CG (Sec. 2.2, last paragraph; flexible Polak-Ribiere form when the V-cycle
 * runs in reduced precision) stops when ||rhs - A x||_2 <= tol ||rhs||_2, for
 * nrhs <= max_rhs stacked right-hand sides at once (batched hierarchy when
 * nrhs > 1).  GMRES (Stokes, Sec. 3.4; nrhs = 1; restarted every `restart`
 * steps, modified Gram-Schmidt Arnoldi, Givens rotations, FP64 Krylov
 * vectors) is left preconditioned as in the paper and stops when
 * ||V (rhs - A x)||_2 <= tol ||V rhs||_2; with a reduced-precision V-cycle
 * (linear only to its rounding) that test is confirmed on the recomputed
 * preconditioned residual and the iteration restarts from it when it fails.
 * FGMRES (right preconditioned, preconditioned directions kept) stops when
 * ||rhs - A x||_2 <= tol ||rhs||_2.  With a coefficient jump the two tests
 * differ by orders of magnitude (V weights the residual by about 1/mu);
 * relres always reports the true residual.  Every right-hand side keeps
 * its own CG scalars and stops updating once it has converged, so its result
 * is the same whether it is solved alone or in a batch.  rhs and x may be
 * device pointers or host pointers (pinned or pageable); host buffers are
 * staged through device memory owned by the hierarchy.  rhs must be
 * consistent (orthogonal to the constants, see ldgmg_project_kernel).
 * iters[r] and relres[r] (host arrays of nrhs entries, may be NULL) receive
 * the iteration count and the true final relative residual of right-hand side
 * r.  Returns ENOTCONV (with x written) if max_iter is hit, EINVAL for
 * non-finite rhs, ETIMEOUT if a bounded device wait gave up. */
ldgmg_status ldgmg_solve(ldgmg_hier* h, const double* rhs, double tol, double* x, int nrhs,
                         int* iters, double* relres, void* stream);

/* Residual history of the last ldgmg_solve on this hierarchy for right-hand
 * side `rhs` (0-based): relres[k] for k = 0 .. count-1 (relres[0] = 1), the
 * norm the method tests, relative to its value at x = 0 -- CG: the recurrence
 * residual ||r_k|| / ||b||; GMRES: ||V r_k|| / ||V b|| (Givens estimate);
 * FGMRES: ||r_k|| / ||b||.  This is the history the paper's speed
 * eta = log 0.1 / log rho (Eq. eta) is measured on.  *count receives the
 * length; at most cap values are written (relres may be NULL). */
ldgmg_status ldgmg_solve_history(const ldgmg_hier* h, int rhs, double* relres, int cap, int* count);

/* ---- grouped solve: many small problems in one launch --------------------
 * A group workspace holds the device and pinned host memory of grouped
 * solves (grown on demand, kept between calls).  Use it from one thread at a
 * time; free with ldgmg_group_free. */
typedef struct ldgmg_group ldgmg_group;
ldgmg_status ldgmg_group_create(ldgmg_group** out);
void ldgmg_group_free(ldgmg_group* g);

/* Solve `count` independent single-right-hand-side problems A_i x_i = rhs_i,
 * each on its own hierarchy h[i] (hierarchies may differ in mesh, degree,
 * coefficient field, smoother and V-cycle precision, and may repeat), with
 * one kernel launch per cluster size (at most four launches, the second to
 * fourth on side streams the workspace owns, ordered after the work queued
 * on `stream` and joined back into it): every problem
 * is a whole CG solve (Sec. 2.2, the V-cycle of Algorithm 1 as the
 * preconditioner) run on the device by one thread-block cluster of 1, 2, 4
 * or 8 CTAs (ldgmg_group_cluster), with no host round trip inside it.  The
 * method, stopping test (||rhs - A x|| <= tol[i] ||rhs||, FP64 residual
 * confirmation with a reduced-precision V-cycle) and max_iter are those of
 * ldgmg_solve on h[i] with one right-hand side; results agree with it to
 * rounding (sums are taken in another order).  Eligible hierarchies: scalar
 * operators solved by CG whose blocks are not tensor-core images (max_rhs =
 * 1, or a block size / precision without the batched path), at most 12
 * levels; others -> EUNSUPPORTED.  The call reads the hierarchies' matrices
 * only (never their vectors), so several group calls may share a hierarchy.
 *   rhs[i], x[i]  N_i*b_i doubles each, device or host pointers (host ones are
 *                 staged through the workspace); the x[i] must not overlap.
 *   tol[i] > 0.
 *   iters, relres, status  host arrays of count entries (may be NULL): the
 *                 iteration count, the true final relative residual and the
 *                 status of problem i (OK; ENOTCONV at max_iter or on a
 *                 non-finite residual, x written; EINVAL for non-finite rhs).
 * Returns OK when every problem converged, else the status of the failing
 * problem with the lowest index (the others are still solved).  Synchronises
 * `stream`. */
ldgmg_status ldgmg_solve_group(ldgmg_group* g, int count, ldgmg_hier* const* h, const double* const* rhs,
                               double* const* x, const double* tol, int* iters, double* relres,
                               ldgmg_status* status, void* stream);

/* Cluster size (CTAs) a grouped solve gives hierarchy h: 1, 2, 4 or 8, about
 * 1024 finest-level unknowns per CTA; 0 if h is not eligible for grouped
 * solves. */
ldgmg_status ldgmg_group_cluster(const ldgmg_hier* h, int* cluster);

/* y = A x with the operator apply of the outer CG (Sec. 2.2: the residual
 * update q = A p of every CG iteration), exactly as ldgmg_solve runs it on this
 * hierarchy: the double-FP32 kernels (outer_apply DF; one right-hand side or
 * several, b = 16 / 64), the FP64 block-reuse kernel (several right-hand sides,
 * b = 16 / 64) or the FP64 CUDA-core kernel (every other case).  x_dev, y_dev:
 * device arrays of N*b*nrhs doubles in the layout the batched CG keeps,
 * [element][rhs][mode] (the stacked layout when nrhs = 1); must not overlap.
 * 1 <= nrhs <= max_rhs.  GMRES hierarchies -> EUNSUPPORTED (their apply is
 * ldgmg_apply).  Enqueues on `stream`; does not synchronise. */
ldgmg_status ldgmg_krylov_apply(ldgmg_hier* h, int nrhs, const double* x_dev, double* y_dev, void* stream);

/* ---- per-level entry points (one step of the hot path each) --------------
 * Level vectors are in the hierarchy's working type: double for an FP64
 * hierarchy, float for FP32/BF16.  All pointers are device pointers. */

/* y = M x for M in {A_l, B_l, B_l^T, D_l} (LDGMG_MAT_*; D_l for Jacobi and Gauss-Seidel). */
ldgmg_status ldgmg_level_apply(ldgmg_hier* h, int level, int which, const void* x_dev,
                               void* y_dev, void* stream);

/* Batched block-row apply on level l: y = M x for nrhs right-hand sides, float
 * vectors laid out [element][rhs][mode] (N*b*nrhs floats).  On a batched
 * tensor-core hierarchy (see max_rhs) this is the tensor-core kernel;
 * otherwise the CUDA-core kernel (FP32/BF16/FP16 hierarchies).  nrhs <= 128. */
ldgmg_status ldgmg_level_apply_batched(ldgmg_hier* h, int level, int which, int nrhs, const float* x_dev,
                                       float* y_dev, void* stream);

/* One smoother sweep on level l (Eq. Jsmooth, Eq. B1 or Eq. BT by `form`;
 * Gauss-Seidel: forward / backward colour order; Jacobi ignores form).  x_out may equal x_in.  x_is_zero != 0 treats x_in as
 * zero without reading it (first pre-sweep of a coarse level). */
ldgmg_status ldgmg_level_smooth(ldgmg_hier* h, int level, int form, const void* rhs_dev,
                                const void* x_in_dev, void* x_out_dev, int x_is_zero,
                                void* stream);

/* Restricted residual of Algorithm 1: rc = I_l^T (rhs - A_l x) onto level l+1. */
ldgmg_status ldgmg_level_restrict(ldgmg_hier* h, int level, const void* rhs_dev,
                                  const void* x_dev, void* rc_dev, void* stream);

/* Interpolate and correct (Algorithm 1): x += I_l xc, xc on level l+1. */
ldgmg_status ldgmg_level_prolong(ldgmg_hier* h, int level, const void* xc_dev, void* x_dev,
                                 void* stream);

/* Bottom solve: x = A_bottom^+ rhs (FP64 pseudo-inverse, Sec. 2.2 "Bottom solver"). */
ldgmg_status ldgmg_bottom_solve(ldgmg_hier* h, const void* rhs_dev, void* x_dev, void* stream);

/* Copy a level matrix to host memory as FP64 block-CSR (values as stored on the
 * device, converted to double and divided by the storage scale; FP32 levels of
 * a tensor-core hierarchy are stored as BF16 pairs hi + lo, |a - hi - lo| <=
 * 2^-17 |a|, and exported as hi + lo).  row_ptr: N+1 int64, col: nnzb int32, vals:
 * nnzb*b*b doubles, block (r, c) at vals[nz*b*b + r*b + c].  Any of the three
 * may be NULL to skip it.  Test/inspection entry point. */
ldgmg_status ldgmg_export_level(ldgmg_hier* h, int level, int which, int64_t* row_ptr,
                                int32_t* col, double* vals);

void ldgmg_op_free(ldgmg_op* op);
void ldgmg_hier_free(ldgmg_hier* h);

/* ---- allocation-free entry point ------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that must
 * not call cudaMalloc: code whose device memory is wholly owned by another
 * allocator (e.g. a framework's caching allocator that has reserved the GPU),
 * or a latency-critical loop that cannot take cudaMalloc's implicit device
 * synchronisation.  Such callers cannot create an ldgmg_op either, so this
 * call takes plain sizes.
 *
 * Removes the constant mode of ONE field in place: subtracts the mean of the
 * values v_dev[e*b] over the N elements e from each of them (the mode-0
 * coefficients when v_dev points at an element's first mode).  For a scalar
 * operator (one field, b = (p+1)^dim) that is ldgmg_project_kernel's result up
 * to summation order.  A Stokes vector has dim + 1 fields per element; b alone
 * cannot tell it from a scalar one (b = 27 is both), so this call does not try:
 * project a Stokes vector with one call per field f, passing v_dev + f*field_b
 * and the full block size b as the stride (ldgmg_op_fields gives field_b).
 * v_dev must hold at least (N-1)*b + 1 doubles; the library cannot check its
 * length.  N must satisfy 1 <= N <= LDGMG_NOALLOC_MAX_ELEMENTS, else EINVAL.
 * It allocates nothing: its reduction scratch is a fixed file-scope device
 * array of (LDGMG_NOALLOC_MAX_ELEMENTS / 4096 + 1) doubles (about 32 KB) that
 * every GPU which loads the library holds until the process exits.  The first
 * call on a device looks up that array's device address once (with the device
 * current); make that first call before any stream capture.  All calls share
 * the array: calls that overlap on the GPU (unordered streams, concurrent host
 * threads) race.  Each call writes every scratch word it reads, so nothing
 * carries over between calls.  Enqueues on `stream`; does not synchronise. */
#define LDGMG_NOALLOC_MAX_ELEMENTS 16777216
ldgmg_status ldgmg_project_kernel_noalloc(int64_t N, int b, double* v_dev, void* stream);

/* Self-test of the error path of the library's bounded device waits (the
 * paper has no counterpart): one kernel waits on an mbarrier that nothing
 * arrives on, with the spin limit of the tensor-core kernel's waits, then
 * records the timeout and returns.  Returns LDGMG_ETIMEOUT when the wait gave
 * up as designed (the context stays usable), ECUDA on a CUDA error. */
ldgmg_status ldgmg_selftest_bounded_wait(void* stream);

/* Number of CUDA kernels this library has enqueued since it was loaded (all
 * handles, streams and devices; setup-only kernels included).  For counting
 * the launches of a timed region: read before and after it. */
unsigned long long ldgmg_kernel_launches(void);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* ldgmg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LDGMG_H */
