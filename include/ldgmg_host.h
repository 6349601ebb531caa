/*
 * ldgmg host-setup inspection API (no GPU needed).
 *
 * Runs the library's host-side setup -- LDG assembly (Sec. 2.1), operator
 * coarsening (Sec. 2.2) and smoother construction (block Jacobi, Eq. Jsmooth;
 * balanced block SAI, Sec. 2.3.3) -- exactly as ldgmg_setup does before it
 * uploads the level matrices, and lets the caller read every level matrix
 * back.  Intended for tests and inspection on machines without a GPU.
 *
 * Conventions are those of ldgmg.h (mesh, basis, element and mode order).
 * Returned arrays are written into caller-owned host buffers.  Every call
 * returns an ldgmg_status; messages via ldgmg_last_error().
 */
#ifndef LDGMG_HOST_H
#define LDGMG_HOST_H

#include "ldgmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ldgmg_host_hier ldgmg_host_hier;

/* Assemble on the mesh (mu_host: N values or NULL for mu == 1) and build the
 * whole host hierarchy with the smoother options in *opts (precision ignored).
 * Errors: EINVAL for bad arguments, EUNSUPPORTED for rank-deficient SAI columns. */
ldgmg_status ldgmg_host_build(const ldgmg_mesh* mesh, int p, const double* mu_host, double tau0,
                              const ldgmg_setup_opts* opts, ldgmg_host_hier** out);

/* Same for the Stokes operator of ldgmg_assemble_stokes (gamma, tau0, taup as
 * there); Stokes-balanced SAI with opts->zeta (Sec. 3.3). */
ldgmg_status ldgmg_host_build_stokes(const ldgmg_mesh* mesh, int p, const double* mu_host, int gamma,
                                     double tau0, double taup, const ldgmg_setup_opts* opts,
                                     ldgmg_host_hier** out);

/* Level count and, for level l, n, N, b, stored blocks of A_l and of the
 * smoother matrix (B_l for SAI, D_l for Jacobi; 0 on the bottom level), and the
 * number of distinct blocks held for A_l (the size of its block pool). */
ldgmg_status ldgmg_host_level_info(const ldgmg_host_hier* h, int level, int* nlevels, int* n,
                                   int64_t* N, int* b, int64_t* nnzb_A, int64_t* nnzb_S,
                                   int64_t* distinct_A);

/* FP64 block-CSR copy of A_l / B_l / B_l^T / D_l (LDGMG_MAT_*): row_ptr N+1,
 * col nnzb, vals nnzb*b*b with block (r, c) at vals[nz*b*b + r*b + c].  Any
 * pointer may be NULL. */
ldgmg_status ldgmg_host_export(const ldgmg_host_hier* h, int level, int which, int64_t* row_ptr,
                               int32_t* col, double* vals);

/* Multi-coloured Gauss-Seidel hierarchies (smoother LDGMG_GS): the colour of
 * every element of level l (colour: N ints, may be NULL) and the number of
 * colours.  EINVAL on the bottom level or for other smoothers. */
ldgmg_status ldgmg_host_colours(const ldgmg_host_hier* h, int level, int* colour, int* ncolours);

/* Schedule of the cached tensor-core apply (2D meshes, b = 16) that the
 * library builds for a block pattern (row_ptr: n*n + 1 entries, col), for
 * rcap right-hand sides, storage prec (LDGMG_FP32 or LDGMG_BF16), `ctas` SMs
 * (two CTAs each) and strip width `strip`.  info[0..3] = CTAs used, x slots per CTA, strip
 * width, most blocks in a row; *nloads = x_j loads of one apply.  rec (n*n
 * records of 16 int32 in processing order: row, first block, first load,
 * nnz | nld << 16, then 16 bytes of block slots and 16 bytes of load slots,
 * 16 bytes unused), seg (CTAs + 1 step offsets) and ld_elem (nloads element
 * indices) may be NULL.  EUNSUPPORTED with the reason when no schedule fits
 * (the library then uses the per-use tensor-core kernel).  For tests. */
ldgmg_status ldgmg_host_tc_plan(int n, const int64_t* row_ptr, const int32_t* col, int rcap, int prec, int ctas,
                                int strip, int* info, int64_t* nloads, int32_t* rec, int32_t* seg,
                                int32_t* ld_elem);

void ldgmg_host_free(ldgmg_host_hier* h);

#ifdef __cplusplus
}
#endif

#endif /* LDGMG_HOST_H */
