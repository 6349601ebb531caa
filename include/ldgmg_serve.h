/*
 * ldgmg serving engine: continuous batching of multigrid solves on one GPU.
 *
 * The paper solves one problem at a time; this layer has no counterpart in it.
 * It serves a stream of independent solve requests (different meshes,
 * degrees, coefficient fields and right-hand sides) with the solvers of
 * ldgmg.h:
 *   - Problem classes.  Requests with the same (dim, n, p, stokes form,
 *     coefficient field, penalties) share one operator + hierarchy, built on
 *     first use by a builder thread and then kept resident on the device.
 *   - Admission by HBM footprint.  A class is built only when its estimated
 *     device footprint fits the budget; idle classes (nothing queued, nothing
 *     running) are evicted least-recently-used first to make room.  Requests
 *     of a class that does not fit yet wait in its queue.  A class whose
 *     estimated footprint alone exceeds the budget is refused: it is never
 *     built and its requests complete with status LDGMG_ENOMEM.
 *   - Continuous batching.  Worker threads, each with its own CUDA stream,
 *     take the oldest waiting class that is built and not running, and solve
 *     as many of its queued requests as one call takes: for scalar operators
 *     up to max_batch right-hand sides (fewer for large classes: at most 2^22
 *     dofs per call), on the tensor cores where the hierarchy supports them;
 *     one for Stokes (GMRES).  Requests that arrive while a class is running
 *     join its next call.  Different classes run concurrently on different
 *     streams.
 *   - Grouped small problems.  Scalar classes with at most group_dofs
 *     unknowns are built with one right-hand side per call and solved
 *     together with the queued requests of every other such class: one
 *     ldgmg_solve_group call (one kernel launch per cluster size, each
 *     problem a whole solve on one thread-block cluster) takes up to
 *     group_max of the oldest small requests, whatever their class.  Several
 *     grouped calls may read the same class at once.  With grouped calls on,
 *     the server runs one more worker (index `workers`) that takes grouped
 *     calls only, so small requests never wait behind large solves.
 *   - Precision fallback.  When a solve of a class with a reduced-precision
 *     V-cycle ends with LDGMG_ENOTCONV (the V-cycle too inexact for the
 *     class, e.g. a large coefficient contrast in 3D), the class is rebuilt
 *     once with an FP64 V-cycle and its requests are solved again.
 *   - Determinism.  Every right-hand side of a batched solve keeps its own
 *     Krylov scalars and its arithmetic does not depend on the other
 *     right-hand sides (ldgmg_solve), so a request's result is the same
 *     whether it was served alone or in a mix.
 *
 * Threading: all calls are thread safe.  The server owns copies of the
 * request inputs; the caller keeps x_host alive until ldgmg_server_wait
 * returns for that ticket.  Errors as in ldgmg.h.
 */
#ifndef LDGMG_SERVE_H
#define LDGMG_SERVE_H

#include "ldgmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ldgmg_server ldgmg_server;

typedef struct {
  size_t hbm_budget;        /* device bytes the server may hold in cached classes; 0 = 90% of the
                               device memory free at creation */
  int workers;              /* concurrent solves: host threads with one CUDA stream each, 1..16 */
  int max_batch;            /* right-hand sides per batched solve call, 1..64 */
  int simulate;             /* 1: no device work at all -- builds and solves are timed stand-ins
                               (results carry iters = 0, relres = NaN, x_host untouched).  For
                               testing the scheduler on machines without a GPU. */
  double simulate_solve_s;  /* simulate = 1: seconds per simulated solve call */
  ldgmg_setup_opts setup;   /* options of every hierarchy (max_rhs is set by the server) */
  size_t group_dofs;        /* scalar classes with N*b <= group_dofs are solved in grouped calls
                               (ldgmg_solve_group); 0 = none */
  int group_max;            /* requests per grouped call, 1..65536; 0 = 512 */
  int simulate_notconv_n;   /* simulate = 1 only: solves of classes with mesh size n equal to this value end
                               with LDGMG_ENOTCONV while their V-cycle runs in reduced precision, which
                               exercises the precision fallback without a GPU (0: never) */
} ldgmg_server_opts;

typedef struct {
  int dim, n, p;
  int stokes;               /* -1: scalar operator (ldgmg_assemble); 0 / 1: Stokes standard / stress */
  const double* mu_host;    /* N = n^dim coefficients or NULL (mu == 1); copied at submit */
  double tau0;              /* penalty constants as in ldgmg_assemble(_stokes) */
  double taup;
  const double* rhs_host;   /* N*b values; copied at submit */
  double* x_host;           /* receives the solution; must stay valid until the ticket is waited on */
  double tol;               /* relative residual target of ldgmg_solve */
} ldgmg_request;

typedef struct {
  ldgmg_status status;      /* status of the solve, or of the class build when that failed */
  int iters;
  double relres;            /* true final relative residual (ldgmg_solve) */
  double t_submit, t_start, t_end;   /* seconds on the server clock (ldgmg_server_clock) */
  int batch;                /* right-hand sides (grouped calls: problems) in the call that served it */
  int worker;               /* worker (stream) index that ran it */
} ldgmg_result;

typedef struct {
  uint64_t submitted, completed;
  uint64_t builds, evictions;
  uint64_t build_failures;  /* classes whose build failed or that admission refused (too large) */
  uint64_t solve_calls;     /* ldgmg_solve and ldgmg_solve_group calls; completed / solve_calls = mean batch */
  int max_batch_seen;
  int classes_resident;
  size_t bytes_resident;    /* device bytes of resident classes (measured after build) */
  size_t bytes_peak;
  size_t hbm_budget;
  uint64_t precision_fallbacks;   /* classes rebuilt with an FP64 V-cycle after a reduced-precision ENOTCONV */
  uint64_t group_calls;     /* ldgmg_solve_group calls (counted in solve_calls too) */
  uint64_t group_requests;  /* requests served by them */
} ldgmg_server_stats;

/* Start the server's scheduler, builder and worker threads.  Errors: EINVAL,
 * ENOMEM, ECUDA. */
ldgmg_status ldgmg_server_create(const ldgmg_server_opts* opts, ldgmg_server** out);

/* Queue one request; *ticket identifies it.  Inputs are validated and copied
 * here (EINVAL on bad sizes or a NULL rhs / x). */
ldgmg_status ldgmg_server_submit(ldgmg_server* s, const ldgmg_request* req, uint64_t* ticket);

/* Block until the request is done, fill *out and release the ticket (a ticket
 * is waited on once).  Returns EINVAL for an unknown ticket, else OK; the
 * request's own outcome is in out->status. */
ldgmg_status ldgmg_server_wait(ldgmg_server* s, uint64_t ticket, ldgmg_result* out);

ldgmg_status ldgmg_server_get_stats(ldgmg_server* s, ldgmg_server_stats* out);

/* Seconds since the server was created (the clock of ldgmg_result). */
double ldgmg_server_clock(const ldgmg_server* s);

/* Finish queued and running work, join the threads, free every class. */
void ldgmg_server_destroy(ldgmg_server* s);

#ifdef __cplusplus
}
#endif

#endif /* LDGMG_SERVE_H */
