// C ABI of the LDG multigrid library (declared in include/ldgmg.h).
//
// Setup (assembly, operator coarsening, smoother construction) runs in host
// C++ on pooled block storage (host.cpp), then every level matrix is
// expanded on the device into explicit block-CSR in the requested precision
// (column-major blocks for the CUDA-core kernel, row-major BF16 blocks for
// the tensor-core batched kernel).  The bottom pseudo-inverse comes from a
// cuSOLVER FP64 eigendecomposition on the device.  Everything the V-cycle and
// CG touch afterwards is device resident; the host only enqueues kernels and
// reads the per-right-hand-side residual norms once per CG iteration for the
// stopping test.
#include "ldgmg.h"

#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "host.h"
#include "kernels.h"

using namespace ldgmg;

static thread_local std::string g_err;

// NVTX range over one C-ABI call (visible in Nsight tools; no cost without a tool)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

void ldgmg_set_error(const std::string& msg) { g_err = msg; }

static ldgmg_status fail(ldgmg_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? LDGMG_ENOMEM : LDGMG_ECUDA,           \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

#define CKS(call)                        \
  do {                                   \
    ldgmg_status s_ = (call);            \
    if (s_ != LDGMG_OK) return s_;       \
  } while (0)

static size_t esize(int prec) { return prec == P_FP64 ? 8 : (prec == P_FP32 ? 4 : 2); }

// Power-of-two storage scale for FP16 blocks: the largest entry lands in
// [2^14, 2^15), well inside the FP16 range (max 65504); 1 for other types.
static double storage_scale(const PBSR& H, int prec) {
  if (prec != P_FP16) return 1.0;
  double mx = 0.0;
  for (double v : H.pool.data) mx = std::max(mx, std::fabs(v));
  if (!(mx > 0.0)) return 1.0;
  int e = 0;
  std::frexp(mx, &e);            // mx in [2^(e-1), 2^e)
  return std::ldexp(1.0, 15 - e);
}

// Device bytes held by the handle being built on this thread (ldgmg_*_device_bytes).
static thread_local size_t* g_acct = nullptr;
struct AcctScope {
  size_t* prev;
  explicit AcctScope(size_t* target) : prev(g_acct) { g_acct = target; }
  ~AcctScope() { g_acct = prev; }
};

template <class T>
static ldgmg_status dalloc_impl(T** p, size_t bytes, bool persistent) {
  *p = nullptr;
  if (bytes == 0) return LDGMG_OK;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(LDGMG_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
  }
  if (persistent && g_acct) *g_acct += bytes;
  return LDGMG_OK;
}
// allocation owned by the handle under construction (counted)
template <class T>
static ldgmg_status dalloc(T** p, size_t bytes) { return dalloc_impl(p, bytes, true); }
// scratch freed before the building call returns (not counted)
template <class T>
static ldgmg_status dalloc_tmp(T** p, size_t bytes) { return dalloc_impl(p, bytes, false); }

static void free_sched(TcSched& S) {
  cudaFree(S.rec);
  cudaFree(S.seg);
  cudaFree(S.ld_elem);
  S = TcSched();
}

static void free_mat(DevMat& M) {
  cudaFree(M.row_ptr);
  cudaFree(M.col);
  cudaFree(M.vals);
  free_sched(M.sched);
  M = DevMat();
}

// Expand a pooled host matrix into an explicit device block-CSR.
static ldgmg_status upload(const PBSR& H, int b, int prec, int tc_image, DevMat& M, cudaStream_t st) {
  if (H.nnzb() >= (int64_t(1) << 31)) return fail(LDGMG_EUNSUPPORTED, "more than 2^31 blocks");
  M.nrows = H.nrows;
  M.nnzb = H.nnzb();
  M.b = b;
  M.prec = prec;
  M.tc_image = tc_image;
  M.scale = storage_scale(H, prec);
  M.cs = tc_image ? b : col_stride(b);
  std::vector<int> rp(H.row_ptr.begin(), H.row_ptr.end());
  CKS(dalloc(&M.row_ptr, rp.size() * sizeof(int)));
  CKS(dalloc(&M.col, H.col.size() * sizeof(int)));
  CKS(dalloc((char**)&M.vals, size_t(M.nnzb) * b * M.cs * esize(prec)));
  CK(cudaMemcpyAsync(M.row_ptr, rp.data(), rp.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (M.nnzb) CK(cudaMemcpyAsync(M.col, H.col.data(), H.col.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  uint32_t* d_ids = nullptr;
  double* d_pool = nullptr;
  CKS(dalloc_tmp(&d_ids, H.id.size() * sizeof(uint32_t)));
  CKS(dalloc_tmp(&d_pool, H.pool.data.size() * sizeof(double)));
  if (M.nnzb) {
    CK(cudaMemcpyAsync(d_ids, H.id.data(), H.id.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_pool, H.pool.data.data(), H.pool.data.size() * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    CK(expand_blocks(M.nnzb, b, M.cs, d_ids, d_pool, M.vals, prec, tc_image, M.scale, st));
  }
  CK(cudaStreamSynchronize(st));
  cudaFree(d_ids);
  cudaFree(d_pool);
  return LDGMG_OK;
}

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------

struct ldgmg_op {
  HostLevel host;
  DevMat A;              // FP64 finest-level operator (column-major blocks)
  void* A_pairs = nullptr;  // A's entries as (hi, lo) FP32 pairs, built for batched solves
  double tau0 = 1.0;
  double mu_contrast = 1.0; // max mu / min mu
  double* partials = nullptr;
  double* scal = nullptr;
  size_t dev_bytes = 0;     // device memory held by this handle
};

struct DevLevel {
  int n = 0;
  int64_t N = 0;
  int b = 0;
  DevMat A, S, ST;       // A_l; smoother matrix (B_l or D_l); B_l^T (SAI only)
  int* crows = nullptr;  // Gauss-Seidel: element indices grouped by colour
  std::vector<int64_t> cptr;   // colour c = crows[cptr[c] .. cptr[c+1])
  bool own_A = true;
  void* rhs = nullptr;   // level vectors, room for max_rhs right-hand sides
  void* x = nullptr;
  void* r = nullptr;
};

struct ldgmg_hier {
  ldgmg_op* op = nullptr;
  ldgmg_setup_opts o;
  int prec = P_FP64;
  int vprec = 0;         // 0: double level vectors, 1: float
  size_t vsz = 8;
  int Rmax = 1;          // right-hand sides per call
  bool batched = false;  // tensor-core hierarchy (blocks stored as operand images)
  bool use_df = false;   // batched outer apply in double-FP32 arithmetic
  std::vector<HostLevel> host;   // host[0] is unused (the op holds the finest level)
  std::vector<DevLevel> lv;
  double* P1d = nullptr;         // 2 * q * q injection matrices
  double* pinv = nullptr;        // bottom pseudo-inverse, nbot x nbot
  int64_t nbot = 0;
  // CG work space (FP64, Rmax right-hand sides, [element][rhs][mode])
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *bvec = nullptr, *xvec = nullptr;
  double *scal = nullptr, *partials = nullptr;
  double *stage_rhs = nullptr, *stage_x = nullptr;
  int* active = nullptr;         // device per-RHS CG state: active[Rmax], it[Rmax], flag[Rmax]
  int* err = nullptr;            // device flag set by bounded waits
  double* hscal = nullptr;       // pinned host mirror of per-RHS scalars
  int* hactive = nullptr;        // pinned host mirror of that state
  // GMRES (single right-hand side): Krylov basis Q (restart + 1 vectors),
  // preconditioned directions Z (flexible variant, restart vectors), device
  // Hessenberg column / coefficients, pinned host mirror
  bool gmres = false;
  double *gq = nullptr, *gz = nullptr, *gs = nullptr, *hgs = nullptr;
  size_t dev_bytes = 0;          // device memory held by this handle
  // autotuned launch shape of the tensor-core apply (CTAs per SM; 0 = all that fit)
  int tc_ctas = 0;
  void* ximg = nullptr;          // tensor-core path: operand images of the vector being applied
  size_t ximg_bytes = 0;         // its capacity (level 0 at max_rhs; grown for wider inspection applies)
  double tc_ms = 0.0;            // its measured time on level 0 with max_rhs right-hand sides
  int tc_L = 0;                  // cached tensor-core apply: autotuned strip width (0: not used)
  // residual history of the last solve: ||r_k||^2 of right-hand side r at
  // hist[k * R + r], k = 0..iters (device, CG) / host copy after the solve
  double* hist = nullptr;
  std::vector<double> hhist;
  int hist_R = 0;
  std::vector<int> hist_len;
  std::vector<double> hist_b2;   // ||b||^2 per right-hand side
  // CUDA graphs of the V-cycle body and of chunks of CG iterations, per
  // right-hand-side count: the first run of each runs eagerly (it also
  // performs one-time kernel configuration), the second is captured, later
  // ones replay it.
  struct VGraph {
    int uses = 0;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
  };
  std::map<int, VGraph> graphs;  // by (what, R, chunk): see run_graphed
  cudaStream_t cap_stream = nullptr;
};

static const HostLevel& host_level(const ldgmg_hier* h, int l) {
  return l == 0 ? h->op->host : h->host[l];
}

// y = M x (+ epilogue) on R right-hand sides in the [element][rhs][mode] layout
static ldgmg_status apply_mat(ldgmg_hier* h, const DevMat& M, int mode, const void* x, const void* rhs,
                              const void* xin, void* y, double s, int R, cudaStream_t st) {
  const int64_t b = M.b;
  if (M.tc_image) {
    BatchArgs a;
    a.nrows = M.nrows;
    a.row_ptr = M.row_ptr;
    a.col = M.col;
    a.vals = M.vals;
    if (!h) return fail(LDGMG_EINVAL, "tensor-core apply without its hierarchy");
    a.x = static_cast<const float*>(x);
    a.rhs = static_cast<const float*>(rhs);
    a.xin = static_cast<const float*>(xin);
    a.y = static_cast<float*>(y);
    a.s = s;
    a.mode = mode;
    a.R = R;
    a.es = R * b;
    a.rs = b;
    a.err = h->err;
    if (M.sched.rec && R <= M.sched.rcap) {
      // x operands converted inside the kernel, cached in shared memory (tc_cached.cu)
      a.ximg = nullptr;
      CK(bsr_apply_tc_cached(a, M.sched, M.prec, st));
      return LDGMG_OK;
    }
    const size_t need = x_image_bytes(M.nrows, R, int(b));
    if (need > h->ximg_bytes) {
      // only ldgmg_level_apply_batched can ask for more right-hand sides than
      // max_rhs; never inside a graph capture (V-cycles stay within max_rhs)
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return fail(LDGMG_EINVAL, "tensor-core image work space too small inside a capture");
      CK(cudaDeviceSynchronize());        // no queued work may still read the old space
      cudaFree(h->ximg);
      h->ximg = nullptr;
      h->dev_bytes -= h->ximg_bytes;
      h->ximg_bytes = 0;
      if (cudaMalloc(&h->ximg, need) != cudaSuccess) {
        h->ximg = nullptr;
        return fail(LDGMG_ENOMEM, "cudaMalloc(" + std::to_string(need) + " bytes) for tensor-core images");
      }
      h->ximg_bytes = need;
      h->dev_bytes += need;
    }
    CK(split_x_images(static_cast<const float*>(x), M.nrows, R, int(b), h->ximg, st));
    a.ximg = h->ximg;
    a.ctas_per_sm = h->tc_ctas;
    CK(bsr_apply_tc(a, M.b, M.prec, st));
    return LDGMG_OK;
  }
  CK(bsr_apply_strided(M, mode, x, rhs, xin, y, s, R, R * b, b, st));
  return LDGMG_OK;
}

extern "C" {

const char* ldgmg_last_error(void) { return g_err.c_str(); }

unsigned long long ldgmg_kernel_launches(void) { return launches(); }

void ldgmg_default_opts(ldgmg_setup_opts* o) {
  if (!o) return;
  o->smoother = LDGMG_SAI;
  o->sai_level = 1;
  o->balance = 1;
  o->nu1 = 3;
  o->nu2 = 3;
  o->omega = 0.8;
  o->pre_form = LDGMG_FORM_B1;
  o->post_form = LDGMG_FORM_BT;
  o->vcycle_precision = LDGMG_FP64;
  o->max_iter = 200;
  o->max_rhs = 1;
  o->outer_apply = LDGMG_OUTER_AUTO;
  o->krylov = LDGMG_KRYLOV_AUTO;
  o->restart = 50;
  o->zeta = 0.0;
}

void ldgmg_op_free(ldgmg_op* op) {
  if (!op) return;
  free_mat(op->A);
  cudaFree(op->A_pairs);
  cudaFree(op->partials);
  cudaFree(op->scal);
  delete op;
}

}  // extern "C"

// Common part of the assembly entry points: checks, host assembly by
// `assemble`, and the FP64 device copy of A.
template <class Assemble>
static ldgmg_status make_op(const ldgmg_mesh* mesh, int p, int nfields, const double* mu_host, double tau0,
                            ldgmg_op** out, Assemble assemble) {
  g_err.clear();
  if (!mesh || !out) return fail(LDGMG_EINVAL, "null argument");
  *out = nullptr;
  if (!mesh->periodic) return fail(LDGMG_EUNSUPPORTED, "only periodic meshes are supported");
  if (mesh->dim != 2 && mesh->dim != 3) return fail(LDGMG_EINVAL, "dim must be 2 or 3");
  if (mesh->n < 1 || mesh->n > 4096) return fail(LDGMG_EINVAL, "n out of range");
  int b = nfields;
  for (int t = 0; t < mesh->dim; ++t) b *= (p + 1);
  if (p < 1 || !block_size_supported(b)) return fail(LDGMG_EUNSUPPORTED, "unsupported block size");
  ldgmg_op* op = new (std::nothrow) ldgmg_op();
  if (!op) return fail(LDGMG_ENOMEM, "host allocation");
  std::string err = assemble(op->host);
  if (!err.empty()) {
    delete op;
    return fail(LDGMG_EINVAL, err);
  }
  AcctScope acct(&op->dev_bytes);
  op->tau0 = tau0;
  if (mu_host) {
    double lo = mu_host[0], hi = mu_host[0];
    for (int64_t e = 1; e < op->host.N; ++e) {
      lo = std::min(lo, mu_host[e]);
      hi = std::max(hi, mu_host[e]);
    }
    op->mu_contrast = hi / lo;
  }
  ldgmg_status s = upload(op->host.A, b, P_FP64, 0, op->A, 0);
  if (s == LDGMG_OK) s = dalloc(&op->partials, kDotBlocks * sizeof(double));
  if (s == LDGMG_OK) s = dalloc(&op->scal, kCgSlots * sizeof(double));
  if (s != LDGMG_OK) {
    ldgmg_op_free(op);
    return s;
  }
  *out = op;
  return LDGMG_OK;
}

extern "C" {

ldgmg_status ldgmg_assemble(const ldgmg_mesh* mesh, int p, const double* mu_host, double tau0,
                            ldgmg_op** out) {
  return make_op(mesh, p, 1, mu_host, tau0, out,
                 [&](HostLevel& L) { return assemble_fine(L, mesh->dim, mesh->n, p, mu_host, tau0); });
}

ldgmg_status ldgmg_assemble_stokes(const ldgmg_mesh* mesh, int p, const double* mu_host, int gamma,
                                   double tau0, double taup, ldgmg_op** out) {
  if (!mesh) return fail(LDGMG_EINVAL, "null argument");
  return make_op(mesh, p, mesh->dim + 1, mu_host, tau0, out, [&](HostLevel& L) {
    return assemble_stokes_fine(L, mesh->dim, mesh->n, p, mu_host, gamma, tau0, taup);
  });
}

ldgmg_status ldgmg_op_device_bytes(const ldgmg_op* op, size_t* bytes) {
  if (!op || !bytes) return fail(LDGMG_EINVAL, "null argument");
  *bytes = op->dev_bytes;
  return LDGMG_OK;
}

ldgmg_status ldgmg_solve_history(const ldgmg_hier* h, int rhs, double* relres, int cap, int* count) {
  if (!h || !count) return fail(LDGMG_EINVAL, "null argument");
  if (rhs < 0 || rhs >= h->hist_R) return fail(LDGMG_EINVAL, "no history for this right-hand side");
  const int len = h->hist_len[rhs];
  *count = len;
  const double b2 = h->hist_b2[rhs];
  for (int k = 0; k < len && k < cap && relres; ++k) {
    const double v = h->hhist[size_t(k) * h->hist_R + rhs];
    relres[k] = b2 > 0.0 ? std::sqrt(v / b2) : 0.0;
  }
  return LDGMG_OK;
}

ldgmg_status ldgmg_selftest_bounded_wait(void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int* d_err = nullptr;
  CK(cudaMalloc((void**)&d_err, sizeof(int)));
  int e = 0;
  cudaError_t c = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (c == cudaSuccess) c = bounded_wait_probe(d_err, st);
  if (c == cudaSuccess) c = cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (c == cudaSuccess) c = cudaStreamSynchronize(st);
  cudaFree(d_err);
  if (c != cudaSuccess) return fail(LDGMG_ECUDA, std::string("bounded-wait self-test: ") + cudaGetErrorString(c));
  if (e) return fail(LDGMG_ETIMEOUT, "bounded device wait gave up (self-test: expected)");
  return LDGMG_OK;
}

ldgmg_status ldgmg_hier_tc_schedule(const ldgmg_hier* h, int* strip, int* x_slots, double* loads_per_row) {
  if (!h) return fail(LDGMG_EINVAL, "null hierarchy");
  const TcSched& S = h->lv.size() > 1 ? h->lv[0].S.sched : TcSched();
  if (strip) *strip = S.rec ? h->tc_L : 0;
  if (x_slots) *x_slots = S.rec ? S.S : 0;
  if (loads_per_row) *loads_per_row = S.rec && h->lv[0].N ? double(S.nloads) / double(h->lv[0].N) : 0.0;
  return LDGMG_OK;
}

ldgmg_status ldgmg_hier_tuning(const ldgmg_hier* h, int* tc_ctas_per_sm, double* tc_ms) {
  if (!h) return fail(LDGMG_EINVAL, "null hierarchy");
  if (tc_ctas_per_sm) *tc_ctas_per_sm = h->tc_ctas;
  if (tc_ms) *tc_ms = h->tc_ms;
  return LDGMG_OK;
}

ldgmg_status ldgmg_hier_device_bytes(const ldgmg_hier* h, size_t* bytes) {
  if (!h || !bytes) return fail(LDGMG_EINVAL, "null argument");
  *bytes = h->dev_bytes;
  return LDGMG_OK;
}

ldgmg_status ldgmg_op_fields(const ldgmg_op* op, int* nfields, int* field_b) {
  if (!op) return fail(LDGMG_EINVAL, "null op");
  if (nfields) *nfields = op->host.nf;
  if (field_b) *field_b = op->host.bs;
  return LDGMG_OK;
}

ldgmg_status ldgmg_op_info(const ldgmg_op* op, int64_t* N, int* b, int64_t* nnzb) {
  if (!op) return fail(LDGMG_EINVAL, "null op");
  if (N) *N = op->host.N;
  if (b) *b = op->host.b;
  if (nnzb) *nnzb = op->A.nnzb;
  return LDGMG_OK;
}

ldgmg_status ldgmg_apply(ldgmg_op* op, const double* x, double* y, int nrhs, void* stream) {
  if (!op || !x || !y) return fail(LDGMG_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > 65535) return fail(LDGMG_EINVAL, "nrhs out of range");
  const int64_t b = op->host.b, N = op->host.N;
  // stacked vectors: element e of right-hand side r at (r*N + e)*b
  CK(bsr_apply_strided(op->A, M_Y, x, nullptr, nullptr, y, 1.0, nrhs, b, N * b, (cudaStream_t)stream));
  return LDGMG_OK;
}

ldgmg_status ldgmg_project_kernel(ldgmg_op* op, double* v, int nrhs, void* stream) {
  if (!op || !v) return fail(LDGMG_EINVAL, "null argument");
  if (nrhs < 1) return fail(LDGMG_EINVAL, "nrhs must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  // c has equal mode-0 entries and zeros elsewhere, so the projection
  // subtracts the mean of the mode-0 coefficients from each of them (per
  // field: the field's mode 0 sits at offset f * bs inside each block).
  const int64_t N = op->host.N, b = op->host.b, bs = op->host.bs;
  for (int r = 0; r < nrhs; ++r)
    for (int f = 0; f < op->host.nf; ++f) {
      CK(strided_sum(N, b, v + r * N * b + f * bs, op->partials, op->scal, st));
      CK(strided_sub_mean(N, b, v + r * N * b + f * bs, op->scal, st));
    }
  return LDGMG_OK;
}

void ldgmg_hier_free(ldgmg_hier* h) {
  if (!h) return;
  for (auto& L : h->lv) {
    if (L.own_A) free_mat(L.A);
    free_mat(L.S);
    free_mat(L.ST);
    cudaFree(L.crows);
    cudaFree(L.rhs);
    cudaFree(L.x);
    cudaFree(L.r);
  }
  cudaFree(h->P1d);
  cudaFree(h->pinv);
  for (double* v : {h->r, h->z, h->p, h->q, h->bvec, h->xvec, h->scal, h->partials, h->stage_rhs, h->stage_x})
    cudaFree(v);
  cudaFree(h->active);
  cudaFree(h->err);
  cudaFree(h->ximg);
  cudaFree(h->hist);
  cudaFree(h->gq);
  cudaFree(h->gz);
  cudaFree(h->gs);
  for (auto& kv : h->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->hgs) cudaFreeHost(h->hgs);
  if (h->hscal) cudaFreeHost(h->hscal);
  if (h->hactive) cudaFreeHost(h->hactive);
  delete h;
}

// bottom pseudo-inverse: FP64 symmetric eigendecomposition (cuSOLVER) on the device
__global__ void scale_columns(int64_t n, double* U, const double* inv) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n * n; t += int64_t(gridDim.x) * blockDim.x)
    U[t] *= inv[t / n];  // column-major: column t / n
}

static ldgmg_status bottom_pinv(ldgmg_hier* h, const HostLevel& L, cudaStream_t st) {
  std::vector<double> dense;
  dense_A(L, dense);
  const int64_t n = L.N * L.b;
  if (n > 20000) return fail(LDGMG_EUNSUPPORTED, "bottom level too large for a dense solve");
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      const double m = 0.5 * (dense[i * n + j] + dense[j * n + i]);
      dense[i * n + j] = dense[j * n + i] = m;
    }
  h->nbot = n;
  double *dA = nullptr, *dW = nullptr, *dWork = nullptr, *dU2 = nullptr, *dInv = nullptr;
  int* dInfo = nullptr;
  CKS(dalloc_tmp(&dA, size_t(n) * n * sizeof(double)));
  CKS(dalloc_tmp(&dU2, size_t(n) * n * sizeof(double)));
  CKS(dalloc_tmp(&dW, n * sizeof(double)));
  CKS(dalloc_tmp(&dInv, n * sizeof(double)));
  CKS(dalloc_tmp(&dInfo, sizeof(int)));
  CKS(dalloc(&h->pinv, size_t(n) * n * sizeof(double)));
  CK(cudaMemcpyAsync(dA, dense.data(), size_t(n) * n * sizeof(double), cudaMemcpyHostToDevice, st));
  cusolverDnHandle_t sh = nullptr;
  cublasHandle_t bh = nullptr;
  ldgmg_status status = LDGMG_OK;
  int lwork = 0, info = 0;
  std::vector<double> W(n), inv(n, 0.0);
  double lmax = 0.0;
  if (cusolverDnCreate(&sh) != CUSOLVER_STATUS_SUCCESS) { status = fail(LDGMG_ECUDA, "cusolverDnCreate"); goto done; }
  cusolverDnSetStream(sh, st);
  if (cusolverDnDsyevd_bufferSize(sh, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, int(n), dA, int(n), dW,
                                  &lwork) != CUSOLVER_STATUS_SUCCESS) {
    status = fail(LDGMG_ECUDA, "cusolverDnDsyevd_bufferSize");
    goto done;
  }
  if ((status = dalloc_tmp(&dWork, size_t(lwork) * sizeof(double))) != LDGMG_OK) goto done;
  if (cusolverDnDsyevd(sh, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, int(n), dA, int(n), dW, dWork, lwork,
                       dInfo) != CUSOLVER_STATUS_SUCCESS) {
    status = fail(LDGMG_ECUDA, "cusolverDnDsyevd");
    goto done;
  }
  if (cudaMemcpyAsync(W.data(), dW, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&info, dInfo, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    status = fail(LDGMG_ECUDA, "eigenvalue copy");
    goto done;
  }
  if (info != 0) { status = fail(LDGMG_ECUDA, "syevd info = " + std::to_string(info)); goto done; }
  for (double w : W) lmax = std::max(lmax, std::fabs(w));
  for (int64_t k = 0; k < n; ++k) inv[k] = std::fabs(W[k]) > 1e-12 * lmax ? 1.0 / W[k] : 0.0;
  if (cudaMemcpyAsync(dInv, inv.data(), n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dU2, dA, size_t(n) * n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    status = fail(LDGMG_ECUDA, "pinv copies");
    goto done;
  }
  scale_columns<<<256, 256, 0, st>>>(n, dU2, dInv);  // setup only, not counted
  if (cublasCreate(&bh) != CUBLAS_STATUS_SUCCESS) { status = fail(LDGMG_ECUDA, "cublasCreate"); goto done; }
  cublasSetStream(bh, st);
  {
    const double one = 1.0, zero = 0.0;
    // Pinv = (U Lambda^+) U^T, column-major; symmetric, so row-major is the same
    if (cublasDgemm(bh, CUBLAS_OP_N, CUBLAS_OP_T, int(n), int(n), int(n), &one, dU2, int(n), dA, int(n), &zero,
                    h->pinv, int(n)) != CUBLAS_STATUS_SUCCESS) {
      status = fail(LDGMG_ECUDA, "cublasDgemm");
      goto done;
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) status = fail(LDGMG_ECUDA, "bottom pinv");
done:
  if (bh) cublasDestroy(bh);
  if (sh) cusolverDnDestroy(sh);
  cudaFree(dA);
  cudaFree(dU2);
  cudaFree(dW);
  cudaFree(dInv);
  cudaFree(dInfo);
  cudaFree(dWork);
  return status;
}

// block-diagonal PBSR view of the Jacobi inverse blocks
static PBSR jacobi_pbsr(const HostLevel& L) {
  PBSR D;
  D.nrows = L.N;
  D.row_ptr.resize(L.N + 1);
  D.col.resize(L.N);
  for (int64_t i = 0; i <= L.N; ++i) D.row_ptr[i] = i;
  for (int64_t i = 0; i < L.N; ++i) D.col[i] = int32_t(i);
  D.id = L.dinv;
  D.pool = L.dinv_pool;
  return D;
}

static ldgmg_status check_err_flag(ldgmg_hier* h, cudaStream_t st);

// Autotuner of the tensor-core apply's launch shape: times the level-0
// smoother apply with max_rhs right-hand sides (on zeroed level vectors) for
// every CTAs-per-SM count that fits and keeps the fastest (median of 3).
// The result of the kernel does not depend on the launch shape.
static ldgmg_status tune_tc(ldgmg_hier* h, cudaStream_t st) {
  DevLevel& D = h->lv[0];
  if (h->lv.size() < 2 || !D.S.tc_image) return LDGMG_OK;
  const int R = h->Rmax;
  const int fit = tc_max_ctas_per_sm(D.b, h->prec, R);
  if (fit <= 1) return LDGMG_OK;
  const size_t bytes = size_t(D.N) * D.b * h->vsz * R;
  CK(cudaMemsetAsync(D.rhs, 0, bytes, st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e30;
  int best_c = 0;
  ldgmg_status status = LDGMG_OK;
  for (int c = 1; c <= fit && status == LDGMG_OK; ++c) {
    h->tc_ctas = c;
    std::vector<float> t;
    for (int rep = 0; rep < 4 && status == LDGMG_OK; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess) { status = fail(LDGMG_ECUDA, "tuner event"); break; }
      status = apply_mat(h, D.S, M_Y, D.rhs, nullptr, nullptr, D.x, 1.0, R, st);
      if (status != LDGMG_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        status = fail(LDGMG_ECUDA, "tuner timing");
        break;
      }
      if (rep > 0) t.push_back(ms);       // the first launch warms caches
    }
    if (status != LDGMG_OK) break;
    std::sort(t.begin(), t.end());
    const double med = t[t.size() / 2];
    if (med < best) {
      best = med;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tc_ctas = best_c;
  h->tc_ms = best;
  if (status == LDGMG_OK) status = check_err_flag(h, st);
  return status;
}

// Schedule of the cached tensor-core apply for M (2D, b = 16) with strip
// width L, halving L while the plan does not fit; *ok = false leaves M on the
// per-use kernel.  counted: the arrays belong to the hierarchy (false: a
// tuning probe, freed by the caller).
static ldgmg_status attach_sched(ldgmg_hier* h, DevMat& M, int dim, int n, int L, bool counted, cudaStream_t st,
                                 bool* ok) {
  *ok = false;
  free_sched(M.sched);
  if (!M.tc_image || M.b != 16 || h->Rmax > 64 || M.nrows == 0) return LDGMG_OK;
  std::vector<int> rp32(size_t(M.nrows) + 1);
  std::vector<int32_t> col(size_t(M.nnzb));
  CK(cudaMemcpyAsync(rp32.data(), M.row_ptr, rp32.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (M.nnzb) CK(cudaMemcpyAsync(col.data(), M.col, col.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const std::vector<int64_t> rp(rp32.begin(), rp32.end());
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  TcSchedHost H;
  bool planned = false;
  for (int l = L; l >= 1 && !planned; l /= 2)
    planned = tc_sched_plan(dim, n, M.nrows, rp.data(), col.data(), h->Rmax, M.prec, sms, l, &H).empty();
  if (!planned) return LDGMG_OK;
  TcSched& S = M.sched;
  auto alloc = [&](auto** p, size_t bytes) { return counted ? dalloc(p, bytes) : dalloc_tmp(p, bytes); };
  if (alloc(&S.rec, H.rec.size()) != LDGMG_OK || alloc(&S.seg, H.seg.size() * sizeof(int)) != LDGMG_OK ||
      alloc(&S.ld_elem, H.ld_elem.size() * sizeof(int)) != LDGMG_OK) {
    free_sched(S);
    return LDGMG_ENOMEM;
  }
  CK(cudaMemcpyAsync(S.rec, H.rec.data(), H.rec.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(S.seg, H.seg.data(), H.seg.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(S.ld_elem, H.ld_elem.data(), H.ld_elem.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  S.G = H.G;
  S.S = H.S;
  S.L = H.L;
  S.kmax = H.kmax;
  S.rcap = H.rcap;
  S.nloads = H.nloads;
  *ok = true;
  return LDGMG_OK;
}

static bool needs_x_images(const ldgmg_hier* h) {
  for (const DevLevel& D : h->lv)
    for (const DevMat* M : {&D.A, &D.S, &D.ST})
      if (M->tc_image && M->nrows > 0 && !M->sched.rec) return true;
  return false;
}

// Autotuner of the cached tensor-core apply: times the level-0 smoother apply
// with max_rhs right-hand sides (zeroed level vectors, median of 3 after one
// warm-up) for strip widths 4, 8 and 16 and keeps the fastest, then attaches
// the schedules of every tensor-core matrix at that width.  The result of
// the apply does not depend on the width (a block row's MMAs are the same).
static ldgmg_status setup_cached_tc(ldgmg_hier* h, cudaStream_t st) {
  DevLevel& D = h->lv[0];
  const int dim = h->op->host.dim;
  if (h->lv.size() < 2 || !D.S.tc_image || D.b != 16 || h->Rmax > 64 || dim != 2) return LDGMG_OK;
  const int R = h->Rmax;
  const size_t bytes = size_t(D.N) * D.b * h->vsz * R;
  CK(cudaMemsetAsync(D.rhs, 0, bytes, st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e30;
  int best_L = 0;
  ldgmg_status status = LDGMG_OK;
  for (int L : {4, 8, 16}) {
    bool ok = false;
    status = attach_sched(h, D.S, dim, D.n, L, false, st, &ok);
    if (status != LDGMG_OK) break;
    if (!ok || D.S.sched.L != std::min(L, D.n)) continue;
    std::vector<float> t;
    for (int rep = 0; rep < 4 && status == LDGMG_OK; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess) { status = fail(LDGMG_ECUDA, "tuner event"); break; }
      status = apply_mat(h, D.S, M_Y, D.rhs, nullptr, nullptr, D.x, 1.0, R, st);
      if (status != LDGMG_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        status = fail(LDGMG_ECUDA, "tuner timing");
        break;
      }
      if (rep > 0) t.push_back(ms);
    }
    if (status != LDGMG_OK) break;
    std::sort(t.begin(), t.end());
    if (t[t.size() / 2] < best) {
      best = t[t.size() / 2];
      best_L = L;
    }
  }
  free_sched(D.S.sched);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status == LDGMG_OK) status = check_err_flag(h, st);
  if (status != LDGMG_OK || best_L == 0) return status;
  h->tc_L = best_L;
  h->tc_ms = best;
  for (DevLevel& Dl : h->lv)
    for (DevMat* M : {&Dl.A, &Dl.S, &Dl.ST}) {
      bool ok = false;
      CKS(attach_sched(h, *M, dim, Dl.n, best_L, true, st, &ok));
    }
  return LDGMG_OK;
}

ldgmg_status ldgmg_setup(ldgmg_op* op, const ldgmg_setup_opts* o, void* stream, ldgmg_hier** out) {
  NvtxRange nvtx_("ldgmg_setup");
  g_err.clear();
  if (!op || !o || !out) return fail(LDGMG_EINVAL, "null argument");
  *out = nullptr;
  if (o->smoother != LDGMG_JACOBI && o->smoother != LDGMG_SAI && o->smoother != LDGMG_GS)
    return fail(LDGMG_EINVAL, "smoother");
  if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 > 64 || o->nu2 > 64) return fail(LDGMG_EINVAL, "nu1/nu2");
  if (o->vcycle_precision < 0 || o->vcycle_precision > 3) return fail(LDGMG_EINVAL, "precision");
  if (o->max_iter < 1) return fail(LDGMG_EINVAL, "max_iter");
  if (o->max_rhs < 1 || o->max_rhs > 128) return fail(LDGMG_EINVAL, "max_rhs must be in 1..128");
  if (o->outer_apply < 0 || o->outer_apply > 2) return fail(LDGMG_EINVAL, "outer_apply");
  if (o->smoother == LDGMG_JACOBI && !(o->omega > 0.0 && o->omega < 2.0)) return fail(LDGMG_EINVAL, "omega");
  if (o->krylov < 0 || o->krylov > 3) return fail(LDGMG_EINVAL, "krylov");
  if (o->restart < 1 || o->restart > 200) return fail(LDGMG_EINVAL, "restart must be in 1..200");
  if (!std::isfinite(o->zeta)) return fail(LDGMG_EINVAL, "zeta");
  // Several right-hand sides: the tensor-core hierarchy where it applies
  // (b = 16 / 64, BF16 or FP32 blocks, Jacobi or SAI), else the CUDA-core
  // kernels with one grid row per right-hand side.
  const bool multi_rhs = o->max_rhs > 1;
  if (multi_rhs && op->host.nf > 1) return fail(LDGMG_EUNSUPPORTED, "max_rhs > 1 is implemented for scalar operators");
  const bool batched = multi_rhs && tc_block_size_supported(op->host.b) && o->smoother != LDGMG_GS &&
                       (o->vcycle_precision == LDGMG_BF16 || o->vcycle_precision == LDGMG_FP32);
  cudaStream_t st = (cudaStream_t)stream;
  ldgmg_hier* h = new (std::nothrow) ldgmg_hier();
  if (!h) return fail(LDGMG_ENOMEM, "host allocation");
  AcctScope acct(&h->dev_bytes);
  h->op = op;
  h->o = *o;
  h->prec = o->vcycle_precision;
  h->vprec = h->prec == P_FP64 ? 0 : 1;
  h->vsz = h->vprec ? 4 : 8;
  h->Rmax = o->max_rhs;
  h->batched = batched;
  auto bail = [&](ldgmg_status s) {
    ldgmg_hier_free(h);
    return s;
  };
  // host hierarchy: n, n/2, ... while n is even and > 1 (host[0] stays empty)
  h->host.resize(1);
  {
    std::string err = build_coarse_levels(op->host, h->host);
    if (!err.empty()) return bail(fail(LDGMG_EINVAL, err));
  }
  const int nl = int(h->host.size());
  SetupParams sp;
  sp.smoother = o->smoother;
  sp.sai_level = o->sai_level;
  sp.balance = o->balance;
  sp.zeta = o->zeta;
  // the SAI least-squares problems (one per distinct balanced column) on the device
  sp.ls = [st](std::vector<LsProblem>& batch) { return sai_ls_device(batch, st); };
  const int nth = std::max(1u, std::thread::hardware_concurrency());
  for (int l = 0; l + 1 < nl; ++l) {
    HostLevel& L = l == 0 ? op->host : h->host[l];
    std::string err = setup_smoother(L, sp, nth);
    if (!err.empty()) return bail(fail(err.find("rank") != std::string::npos ? LDGMG_EUNSUPPORTED : LDGMG_EINVAL, err));
  }
  // device hierarchy
  const HostLevel& L0 = op->host;
  const int q = L0.p + 1;
  {
    Basis1D B = make_basis(L0.p);
    std::vector<double> P(2 * q * q);
    for (int s = 0; s < 2; ++s) std::copy(B.P[s].begin(), B.P[s].end(), P.begin() + s * q * q);
    ldgmg_status s = dalloc(&h->P1d, P.size() * sizeof(double));
    if (s != LDGMG_OK) return bail(s);
    if (cudaMemcpyAsync(h->P1d, P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return bail(fail(LDGMG_ECUDA, "P1d copy"));
  }
  const int rm = batched ? 1 : 0;
  h->lv.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const HostLevel& L = host_level(h, l);
    DevLevel& D = h->lv[l];
    D.n = L.n;
    D.N = L.N;
    D.b = L.b;
    ldgmg_status s = LDGMG_OK;
    if (l == 0 && h->prec == P_FP64) {
      D.A = op->A;
      D.own_A = false;
    } else {
      s = upload(L.A, L.b, h->prec, rm, D.A, st);
    }
    if (s == LDGMG_OK && l + 1 < nl) {
      if (o->smoother == LDGMG_SAI) {
        s = upload(L.B, L.b, h->prec, rm, D.S, st);
        if (s == LDGMG_OK) s = upload(L.BT, L.b, h->prec, rm, D.ST, st);
      } else {
        s = upload(jacobi_pbsr(L), L.b, h->prec, rm, D.S, st);
      }
      if (s == LDGMG_OK && o->smoother == LDGMG_GS) {
        D.cptr = L.colour_ptr;
        s = dalloc(&D.crows, L.colour_rows.size() * sizeof(int));
        if (s == LDGMG_OK &&
            cudaMemcpyAsync(D.crows, L.colour_rows.data(), L.colour_rows.size() * sizeof(int),
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
          s = fail(LDGMG_ECUDA, "colour rows copy");
        if (s == LDGMG_OK && cudaStreamSynchronize(st) != cudaSuccess) s = fail(LDGMG_ECUDA, "colour rows sync");
      }
    }
    const size_t vb = size_t(L.N) * L.b * h->vsz * h->Rmax;
    if (s == LDGMG_OK) s = dalloc((char**)&D.rhs, vb);
    if (s == LDGMG_OK) s = dalloc((char**)&D.x, vb);
    if (s == LDGMG_OK) s = dalloc((char**)&D.r, vb);
    if (s != LDGMG_OK) return bail(s);
  }
  {
    ldgmg_status s = bottom_pinv(h, host_level(h, nl - 1), st);
    if (s != LDGMG_OK) return bail(s);
  }
  // double-FP32 outer apply: batched hierarchies (b = 16 / 64), and the single
  // right-hand-side mixed-precision path for b = 16 / 64; the plain FP64
  // hierarchy always keeps the FP64 apply
  h->use_df = (batched || h->prec != P_FP64) && tc_block_size_supported(op->host.b) &&
              (o->outer_apply == LDGMG_OUTER_DF || o->outer_apply == LDGMG_OUTER_AUTO);
  if (h->use_df && !op->A_pairs) {
    // FP32-pair copy of the FP64 operator for the batched outer apply (df_apply.cu)
    const int64_t cnt = op->A.nnzb * int64_t(op->A.b) * op->A.b;
    AcctScope acct_op(&op->dev_bytes);       // owned (and freed) by the operator
    ldgmg_status s = dalloc((char**)&op->A_pairs, size_t(cnt) * 8);
    if (s != LDGMG_OK) return bail(s);
    if (split_to_float_pairs(cnt, static_cast<const double*>(op->A.vals), op->A_pairs, st) != cudaSuccess)
      return bail(fail(LDGMG_ECUDA, "split_to_float_pairs"));
  }
  const size_t n0 = size_t(L0.N) * L0.b * sizeof(double) * h->Rmax;
  for (double** v : {&h->r, &h->z, &h->p, &h->q, &h->bvec, &h->xvec, &h->stage_rhs, &h->stage_x}) {
    ldgmg_status s = dalloc(v, n0);
    if (s != LDGMG_OK) return bail(s);
  }
  if (dalloc(&h->hist, size_t(o->max_iter + 1) * h->Rmax * sizeof(double)) != LDGMG_OK ||
      dalloc(&h->scal, size_t(kCgSlots) * h->Rmax * sizeof(double)) != LDGMG_OK ||
      dalloc(&h->partials, size_t(std::max(kDotBlocks, kBatchDotBlocks)) * h->Rmax * sizeof(double)) != LDGMG_OK ||
      dalloc(&h->active, 3 * size_t(h->Rmax) * sizeof(int)) != LDGMG_OK || dalloc(&h->err, sizeof(int)) != LDGMG_OK)
    return bail(LDGMG_ENOMEM);
  if (cudaMallocHost((void**)&h->hscal, size_t(kCgSlots) * h->Rmax * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&h->hactive, 3 * size_t(h->Rmax) * sizeof(int)) != cudaSuccess)
    return bail(fail(LDGMG_ENOMEM, "cudaMallocHost"));
  h->gmres = o->krylov == LDGMG_KRYLOV_GMRES || o->krylov == LDGMG_KRYLOV_FGMRES ||
             (o->krylov == LDGMG_KRYLOV_AUTO && op->host.nf > 1);
  if (h->gmres) {
    const size_t nv = size_t(L0.N) * L0.b * sizeof(double);
    const int m = o->restart;
    const bool flexible = o->krylov == LDGMG_KRYLOV_FGMRES || (o->krylov == LDGMG_KRYLOV_AUTO && h->prec != P_FP64);
    if (dalloc(&h->gq, nv * (m + 1)) != LDGMG_OK || (flexible && dalloc(&h->gz, nv * m) != LDGMG_OK) ||
        dalloc(&h->gs, size_t(m + 2) * sizeof(double)) != LDGMG_OK)
      return bail(LDGMG_ENOMEM);
    if (cudaMallocHost((void**)&h->hgs, size_t(m + 2) * sizeof(double)) != cudaSuccess)
      return bail(fail(LDGMG_ENOMEM, "cudaMallocHost"));
  }
  if (cudaMemsetAsync(h->err, 0, sizeof(int), st) != cudaSuccess) return bail(fail(LDGMG_ECUDA, "memset"));
  if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(LDGMG_ECUDA, "setup sync"));
  if (batched) {
    // cached tensor-core apply where a schedule fits (2D, b = 16), autotuned
    // strip width; the per-use kernel with x images for every other matrix
    ldgmg_status s = setup_cached_tc(h, st);
    if (s != LDGMG_OK) return bail(s);
    if (needs_x_images(h)) {
      h->ximg_bytes = x_image_bytes(L0.N, h->Rmax, L0.b);
      if (dalloc(&h->ximg, h->ximg_bytes) != LDGMG_OK) return bail(LDGMG_ENOMEM);
      s = tune_tc(h, st);
      if (s != LDGMG_OK) return bail(s);
    }
  }
  *out = h;
  return LDGMG_OK;
}

ldgmg_status ldgmg_hier_info(const ldgmg_hier* h, int level, int* nlevels, int* n, int64_t* N, int* b,
                             int64_t* nnzb_A, int64_t* nnzb_S) {
  if (!h) return fail(LDGMG_EINVAL, "null hierarchy");
  if (nlevels) *nlevels = int(h->lv.size());
  if (level < 0 || level >= int(h->lv.size())) return fail(LDGMG_EINVAL, "level out of range");
  const DevLevel& D = h->lv[level];
  if (n) *n = D.n;
  if (N) *N = D.N;
  if (b) *b = D.b;
  if (nnzb_A) *nnzb_A = D.A.nnzb;
  if (nnzb_S) *nnzb_S = D.S.nnzb;
  return LDGMG_OK;
}

// ---------------------------------------------------------------------------
// V-cycle steps on R right-hand sides (level vectors [element][rhs][mode])
// ---------------------------------------------------------------------------

static ldgmg_status smooth(ldgmg_hier* h, int l, int form, const void* rhs, const void* xin, void* xout,
                           bool x_zero, int R, cudaStream_t st) {
  DevLevel& D = h->lv[l];
  if (h->o.smoother == LDGMG_GS) {
    // Multi-coloured block Gauss-Seidel (Sec. 2.3.2), omega = 1: colour by
    // colour, x_i += A_ii^{-1} (b_i - sum_j A_ij x_j) on that colour's rows
    // (the residual kernel reads the newest x of the other colours); forward
    // colour order for form B1, backward for BT.  CUDA-core kernels only.
    const int64_t b = D.b;
    const int64_t es = R * b, rs = b;
    const size_t bytes = size_t(D.N) * b * h->vsz * R;
    if (x_zero) CK(cudaMemsetAsync(xout, 0, bytes, st));
    else if (xin != xout) CK(cudaMemcpyAsync(xout, xin, bytes, cudaMemcpyDeviceToDevice, st));
    const int nc = int(D.cptr.size()) - 1;
    for (int k = 0; k < nc; ++k) {
      const int c = form == LDGMG_FORM_BT ? nc - 1 - k : k;
      const int* rows = D.crows + D.cptr[c];
      const int64_t cnt = D.cptr[c + 1] - D.cptr[c];
      if (x_zero && k == 0) {        // x = 0: the first colour's residual is b itself
        CK(bsr_apply_rows(D.S, rows, cnt, M_SCALE, rhs, nullptr, nullptr, xout, 1.0, R, es, rs, st));
        continue;
      }
      CK(bsr_apply_rows(D.A, rows, cnt, M_RES, xout, rhs, nullptr, D.r, 1.0, R, es, rs, st));
      CK(bsr_apply_rows(D.S, rows, cnt, M_AXPY, D.r, nullptr, xout, xout, 1.0, R, es, rs, st));
    }
    return LDGMG_OK;
  }
  if (h->o.smoother == LDGMG_JACOBI) {
    // Eq. Jsmooth written as x + omega D^{-1} (b - A x)
    if (x_zero) {
      CKS(apply_mat(h, D.S, M_SCALE, rhs, nullptr, nullptr, xout, h->o.omega, R, st));
    } else {
      CKS(apply_mat(h, D.A, M_RES, xin, rhs, nullptr, D.r, 1.0, R, st));
      CKS(apply_mat(h, D.S, M_AXPY, D.r, nullptr, xin, xout, h->o.omega, R, st));
    }
    return LDGMG_OK;
  }
  // Eq. B1: x - B (A x - b) = x + B (b - A x); Eq. BT with B^T
  const DevMat& M = form == LDGMG_FORM_BT ? D.ST : D.S;
  if (x_zero) {
    CKS(apply_mat(h, M, M_Y, rhs, nullptr, nullptr, xout, 1.0, R, st));
  } else {
    CKS(apply_mat(h, D.A, M_RES, xin, rhs, nullptr, D.r, 1.0, R, st));
    CKS(apply_mat(h, M, M_AXPY, D.r, nullptr, xin, xout, 1.0, R, st));
  }
  return LDGMG_OK;
}

static ldgmg_status restrict_residual(ldgmg_hier* h, int l, const void* rhs, const void* x, bool x_zero,
                                      void* rc, int R, cudaStream_t st) {
  DevLevel& D = h->lv[l];
  const void* r = rhs;
  if (!x_zero) {
    CKS(apply_mat(h, D.A, M_RES, x, rhs, nullptr, D.r, 1.0, R, st));
    r = D.r;
  }
  // fields transfer independently: R right-hand sides of nf fields are R * nf scalar vectors
  CK(restrict_apply(h->op->host.dim, h->op->host.p + 1, D.n, h->P1d, r, rc, h->vprec, R * h->op->host.nf, st));
  return LDGMG_OK;
}

// Algorithm 1 on level l with x_l = 0 initially; rhs in lv[l].rhs, result in lv[l].x
static ldgmg_status vcycle_level(ldgmg_hier* h, int l, int R, cudaStream_t st) {
  DevLevel& D = h->lv[l];
  const int nl = int(h->lv.size());
  if (l == nl - 1) {
    CK(dense_gemv(h->nbot, D.b, h->pinv, D.rhs, D.x, h->vprec, R, st));
    return LDGMG_OK;
  }
  bool xz = true;
  for (int s = 0; s < h->o.nu1; ++s) {
    CKS(smooth(h, l, h->o.pre_form, D.rhs, D.x, D.x, xz, R, st));
    xz = false;
  }
  CKS(restrict_residual(h, l, D.rhs, D.x, xz, h->lv[l + 1].rhs, R, st));
  CKS(vcycle_level(h, l + 1, R, st));
  if (xz) CK(cudaMemsetAsync(D.x, 0, size_t(D.N) * D.b * h->vsz * R, st));
  CK(prolong_apply(h->op->host.dim, h->op->host.p + 1, D.n, h->P1d, h->lv[l + 1].x, D.x, h->vprec,
                   R * h->op->host.nf, st));
  for (int s = 0; s < h->o.nu2; ++s) CKS(smooth(h, l, h->o.post_form, D.rhs, D.x, D.x, false, R, st));
  return LDGMG_OK;
}

}  // extern "C"

// Runs fn(stream) eagerly the first time `key` is seen, captures it into a
// CUDA graph the second time (on a private stream in thread-local capture
// mode, ordered after the work already queued on st), and replays the graph
// on st from then on.  fn must only enqueue work on the stream it is given
// and only touch buffers owned by the hierarchy.
template <class Fn>
static ldgmg_status run_graphed(ldgmg_hier* h, int key, cudaStream_t st, Fn fn) {
  auto& g = h->graphs[key];
  if (g.exec) {
    CK(cudaGraphLaunch(g.exec, st));
    CK(launched(g.kernels));
    return LDGMG_OK;
  }
  if (g.uses++ == 0) return fn(st);
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CK(cudaEventRecord(ev, st));
  CK(cudaStreamWaitEvent(h->cap_stream, ev, 0));
  CK(cudaEventDestroy(ev));
  const unsigned long long k0 = launches();
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  ldgmg_status s = fn(h->cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (s != LDGMG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(LDGMG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g.exec = nullptr;
    return fail(LDGMG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  g.kernels = int(launches() - k0);
  launched(-g.kernels);      // captured, not yet run
  CK(cudaGraphLaunch(g.exec, st));
  CK(launched(g.kernels));
  return LDGMG_OK;
}

extern "C" {

enum { G_VCYCLE = 1, G_CG = 2 };
static int graph_key(int what, int R, int chunk) { return (what << 24) | (R << 8) | chunk; }

// The V-cycle body on level 0's own buffers (lv[0].rhs -> lv[0].x)
static ldgmg_status vcycle_body(ldgmg_hier* h, int R, cudaStream_t st) {
  return run_graphed(h, graph_key(G_VCYCLE, R, 0), st, [&](cudaStream_t s) { return vcycle_level(h, 0, R, s); });
}

// x = V b on R right-hand sides, FP64 device vectors [element][rhs][mode];
// graphed = false inlines the V-cycle kernels (inside a larger capture).
static ldgmg_status apply_V(ldgmg_hier* h, const double* b, double* x, int R, cudaStream_t st,
                            bool graphed = true) {
  DevLevel& D = h->lv[0];
  const int64_t n = D.N * D.b * R;
  if (h->vprec == 0) CK(cudaMemcpyAsync(D.rhs, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else CK(cast_d2f(n, b, (float*)D.rhs, st));
  if (graphed) CKS(vcycle_body(h, R, st));
  else CKS(vcycle_level(h, 0, R, st));
  if (h->vprec == 0) CK(cudaMemcpyAsync(x, D.x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else CK(cast_f2d(n, (const float*)D.x, x, st));
  return LDGMG_OK;
}

static ldgmg_status check_err_flag(ldgmg_hier* h, cudaStream_t st) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (e) return fail(LDGMG_ETIMEOUT, "a bounded device wait in the tensor-core apply gave up");
  return LDGMG_OK;
}

ldgmg_status ldgmg_vcycle(ldgmg_hier* h, const double* b, double* x, int nrhs, void* stream) {
  NvtxRange nvtx_("ldgmg_vcycle");
  if (!h || !b || !x) return fail(LDGMG_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > h->Rmax) return fail(LDGMG_EINVAL, "nrhs must be in 1..max_rhs");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = h->op->host.N, bsz = h->op->host.b;
  if (nrhs == 1) {
    CKS(apply_V(h, b, x, 1, st));
  } else {
    CK(stack_to_batch(N, nrhs, int(bsz), b, h->bvec, st));
    CKS(apply_V(h, h->bvec, h->xvec, nrhs, st));
    CK(batch_to_stack(N, nrhs, int(bsz), h->xvec, x, st));
  }
  if (h->batched) return check_err_flag(h, st);
  return LDGMG_OK;
}

static bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// copy slot `slot` (R doubles) of the device scalars to the pinned host mirror
static ldgmg_status read_slot(ldgmg_hier* h, int slot, int R, cudaStream_t st) {
  CK(cudaMemcpyAsync(h->hscal + size_t(slot) * R, h->scal + size_t(slot) * R, R * sizeof(double),
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return LDGMG_OK;
}

// Restarted GMRES from x = 0 on one right-hand side b (FP64 device vectors),
// the outer solver for the symmetric indefinite Stokes system (Sec. 3.4).
// Arnoldi by modified Gram-Schmidt (dots and updates on the device, the
// Hessenberg column read back once per step), Givens rotations and the
// least-squares update on the host.
//   left (LDGMG_KRYLOV_GMRES, the paper's form): solves V A x = V b, stops when
//     ||V (b - A x)|| <= tol ||V b||.  With a reduced-precision V-cycle, V is
//     linear only to its rounding, so the Givens estimate is confirmed on the
//     recomputed preconditioned residual (FP64 residual, then V) before
//     stopping, and the iteration restarts from it otherwise: iterative
//     refinement with GMRES as the inner solver.
//   flexible (LDGMG_KRYLOV_FGMRES): right preconditioned with z_j = V q_j kept,
//     x = sum y_j z_j, stops when ||b - A x|| <= tol ||b|| (confirmed on the
//     recomputed true residual).
static ldgmg_status gmres_solve(ldgmg_hier* h, const double* b, double* x, double tol, int* iters,
                                cudaStream_t st) {
  const HostLevel& L0 = h->op->host;
  const int64_t n = L0.N * L0.b;
  const int m = h->o.restart;
  const bool flexible = h->o.krylov == LDGMG_KRYLOV_FGMRES ||
                        (h->o.krylov == LDGMG_KRYLOV_AUTO && h->prec != P_FP64);
  const bool exact_V = h->prec == P_FP64;
  double* Q = h->gq;
  auto q = [&](int i) { return Q + int64_t(i) * n; };
  auto zv = [&](int i) { return h->gz + int64_t(i) * n; };
  auto norm2 = [&](const double* v, double* out) -> ldgmg_status {
    CK(dot(n, v, v, h->partials, h->gs, st));
    CK(cudaMemcpyAsync(h->hgs, h->gs, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *out = std::sqrt(h->hgs[0]);
    return LDGMG_OK;
  };
  CK(cudaMemsetAsync(x, 0, size_t(n) * sizeof(double), st));
  // r0 = V b (left) or b (flexible), held in q_0
  if (flexible) CK(cudaMemcpyAsync(q(0), b, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else CKS(apply_V(h, b, q(0), 1, st));
  double beta0 = 0.0;
  CKS(norm2(q(0), &beta0));
  if (iters) *iters = 0;
  if (!std::isfinite(beta0)) return fail(LDGMG_EINVAL, "rhs contains NaN or Inf");
  h->hist_R = 1;
  h->hist_b2.assign(1, beta0 * beta0);
  h->hhist.assign(1, beta0 * beta0);
  h->hist_len.assign(1, 1);
  if (beta0 == 0.0) return LDGMG_OK;
  std::vector<double> H(size_t(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hij = [&](int i, int j) -> double& { return H[size_t(i) * m + j]; };
  double beta = beta0;
  int k = 0;
  bool converged = false;
  while (k < h->o.max_iter) {
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    CK(vec_div(n, beta, q(0), q(0), st));
    const int mm = std::min(m, h->o.max_iter - k);
    int jd = 0;
    for (int j = 0; j < mm; ++j) {
      double* w = q(j + 1);
      if (flexible) {
        CKS(apply_V(h, q(j), zv(j), 1, st));
        CK(bsr_apply_strided(h->op->A, M_Y, zv(j), nullptr, nullptr, w, 1.0, 1, L0.b, 0, st));
      } else {
        CK(bsr_apply_strided(h->op->A, M_Y, q(j), nullptr, nullptr, h->q, 1.0, 1, L0.b, 0, st));
        CKS(apply_V(h, h->q, w, 1, st));
      }
      for (int i = 0; i <= j; ++i) {     // modified Gram-Schmidt
        CK(dot(n, q(i), w, h->partials, h->gs + i, st));
        CK(axpy_dev(n, h->gs + i, -1.0, q(i), w, st));
      }
      CK(dot(n, w, w, h->partials, h->gs + j + 1, st));
      CK(cudaMemcpyAsync(h->hgs, h->gs, size_t(j + 2) * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i <= j; ++i) Hij(i, j) = h->hgs[i];
      Hij(j + 1, j) = std::sqrt(h->hgs[j + 1]);
      if (!std::isfinite(Hij(j + 1, j))) return fail(LDGMG_ENOTCONV, "GMRES breakdown (non-finite Arnoldi vector)");
      if (Hij(j + 1, j) > 0.0) CK(vec_div(n, Hij(j + 1, j), w, w, st));
      for (int i = 0; i < j; ++i) {      // previous rotations
        const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double den = std::hypot(Hij(j, j), Hij(j + 1, j));
      cs[j] = Hij(j, j) / den;
      sn[j] = Hij(j + 1, j) / den;
      Hij(j, j) = den;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++k;
      jd = j + 1;
      h->hhist.push_back(g[j + 1] * g[j + 1]);
      h->hist_len[0] = int(h->hhist.size());
      if (std::fabs(g[j + 1]) <= tol * beta0) break;
    }
    // y = R^{-1} g (upper triangular), x += Q y (left) or Z y (flexible)
    for (int i = jd - 1; i >= 0; --i) {
      double t = g[i];
      for (int c = i + 1; c < jd; ++c) t -= Hij(i, c) * y[c];
      y[i] = t / Hij(i, i);
    }
    CK(cudaMemcpyAsync(h->gs, y.data(), size_t(jd) * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(vec_combine(n, jd, flexible ? h->gz : Q, n, h->gs, x, st));
    const bool estimate_met = std::fabs(g[jd]) <= tol * beta0;
    if (estimate_met && !flexible && exact_V) {
      converged = true;
      break;
    }
    // restart from the recomputed (preconditioned) residual.  Where the
    // Arnoldi relation holds only to a rounding level above tol (a
    // reduced-precision V in left GMRES; the rounding of A Z = Q H in the
    // flexible form) a met estimate is confirmed here, and the iteration
    // continues from this residual if it is not.
    CK(bsr_apply_strided(h->op->A, M_RES, x, b, nullptr, h->r, 1.0, 1, L0.b, 0, st));
    if (flexible) CK(cudaMemcpyAsync(q(0), h->r, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else CKS(apply_V(h, h->r, q(0), 1, st));
    CKS(norm2(q(0), &beta));
    if (beta <= tol * beta0) {
      converged = true;
      break;
    }
    if (!(beta > 0.0)) {
      converged = beta == 0.0;
      break;
    }
  }
  if (iters) *iters = k;
  return converged ? LDGMG_OK : fail(LDGMG_ENOTCONV, "max_iter reached");
}

// q = A p with the operator apply of the outer CG (Sec. 2.2), FP64 vectors of R
// right-hand sides laid out [element][rhs][mode].  Batched hierarchies apply A
// once per block row for all right-hand sides, in double-FP32 (use_df) or
// FP64.  The arithmetic of each right-hand side does not depend on R, so a
// right-hand side solved alone matches the batch.  Multi-RHS hierarchies use
// the same outer apply for every R (so each right-hand side is bitwise the
// same alone and batched): the block-reuse kernels for b = 16 / 64, else the
// CUDA-core kernel.
// r = b - A x in FP64 on R right-hand sides ([element][rhs][mode]): the CG's
// true residual.  Multi-RHS hierarchies with b = 16 / 64 use the FP64
// block-reuse kernel (A read once for all right-hand sides, and a right-hand
// side's residual the same alone and batched), the others the CUDA-core kernel.
static ldgmg_status true_residual(ldgmg_hier* h, const double* x, const double* b, double* r, int R, cudaStream_t s) {
  const int bsz = h->op->host.b;
  const bool multi = (h->batched || h->Rmax > 1) && R <= 64 && tc_block_size_supported(bsz);
  if (multi) CK(bsr_apply_multi64(h->op->A, M_RES, x, b, r, R, s));
  else CK(bsr_apply_strided(h->op->A, M_RES, x, b, nullptr, r, 1.0, R, int64_t(R) * bsz, bsz, s));
  return LDGMG_OK;
}

static ldgmg_status krylov_apply(ldgmg_hier* h, const double* p, double* q, int R, cudaStream_t s) {
  const int bsz = h->op->host.b;
  const bool multi = (h->batched || h->Rmax > 1) && R <= 64 && tc_block_size_supported(bsz);
  if (multi && h->use_df) CK(bsr_apply_df(h->op->A, h->op->A_pairs, M_Y, p, nullptr, q, R, s));
  else if (multi) CK(bsr_apply_multi64(h->op->A, M_Y, p, nullptr, q, R, s));
  else if (h->use_df && R == 1) CK(bsr_apply_df1(h->op->A, h->op->A_pairs, M_Y, p, nullptr, q, s));
  else CK(bsr_apply_strided(h->op->A, M_Y, p, nullptr, nullptr, q, 1.0, R, int64_t(R) * bsz, bsz, s));
  return LDGMG_OK;
}

ldgmg_status ldgmg_krylov_apply(ldgmg_hier* h, int nrhs, const double* x, double* y, void* stream) {
  g_err.clear();
  if (!h || !x || !y) return fail(LDGMG_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > h->Rmax) return fail(LDGMG_EINVAL, "nrhs must be in 1..max_rhs of the setup");
  if (h->gmres) return fail(LDGMG_EUNSUPPORTED, "GMRES hierarchies apply A in FP64 (ldgmg_apply)");
  return krylov_apply(h, x, y, nrhs, (cudaStream_t)stream);
}

ldgmg_status ldgmg_solve(ldgmg_hier* h, const double* rhs, double tol, double* x, int nrhs, int* iters,
                         double* relres, void* stream) {
  NvtxRange nvtx_("ldgmg_solve");
  g_err.clear();
  if (!h || !rhs || !x) return fail(LDGMG_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > h->Rmax) return fail(LDGMG_EINVAL, "nrhs must be in 1..max_rhs of the setup");
  if (!(tol > 0.0)) return fail(LDGMG_EINVAL, "tol must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  const HostLevel& L0 = h->op->host;
  const int R = nrhs;
  const int64_t N = L0.N, bsz = L0.b;
  const int64_t n = N * bsz * R;
  const size_t nb = size_t(n) * sizeof(double);
  const bool host_rhs = is_host_ptr(rhs), host_x = is_host_ptr(x);
  // right-hand sides in the [element][rhs][mode] layout (the stacked layout when R = 1)
  const double* src = rhs;
  if (host_rhs) {
    CK(cudaMemcpyAsync(h->stage_rhs, rhs, nb, cudaMemcpyHostToDevice, st));
    src = h->stage_rhs;
  }
  const double* b = src;
  if (R > 1) {
    CK(stack_to_batch(N, R, int(bsz), src, h->bvec, st));
    b = h->bvec;
  }
  if (h->gmres) {
    double* xd = host_x ? h->stage_x : x;
    if (R != 1) return fail(LDGMG_EUNSUPPORTED, "GMRES solves take one right-hand side per call");
    int it = 0;
    double bn = 0.0;
    CK(dot(n, b, b, h->partials, h->scal + S_BB, st));
    CK(cudaMemcpyAsync(h->hscal, h->scal + S_BB, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bn = h->hscal[0];
    ldgmg_status result = gmres_solve(h, b, xd, tol, &it, st);
    if (result != LDGMG_OK && result != LDGMG_ENOTCONV) return result;
    const std::string msg = g_err;
    CK(bsr_apply_strided(h->op->A, M_RES, xd, b, nullptr, h->r, 1.0, 1, bsz, 0, st));
    CK(dot(n, h->r, h->r, h->partials, h->scal + S_TMP, st));
    CK(cudaMemcpyAsync(h->hscal + S_TMP, h->scal + S_TMP, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (host_x) CK(cudaMemcpyAsync(x, xd, nb, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (iters) iters[0] = it;
    if (relres) relres[0] = bn > 0.0 ? std::sqrt(h->hscal[S_TMP] / bn) : 0.0;
    if (result != LDGMG_OK) g_err = msg;
    return result;
  }
  // CG.  The iterate lives in h->xvec (a fixed address, so chunks of
  // iterations can be replayed as CUDA graphs) and is copied out at the end.
  double* xg = h->xvec;
  const bool flexible = h->prec != P_FP64;
  double* S = h->scal;
  auto slot = [&](int s) { return S + size_t(s) * R; };
  auto hslot = [&](int s) { return h->hscal + size_t(s) * R; };
  CK(dot_batched(N, R, int(bsz), b, nullptr, h->partials, slot(S_BB), st));
  CKS(read_slot(h, S_BB, R, st));
  std::vector<double> bb(hslot(S_BB), hslot(S_BB) + R);
  for (double v : bb)
    if (!std::isfinite(v)) return fail(LDGMG_EINVAL, "rhs contains NaN or Inf");
  // device state: active[R], it[R], flag[R] (one D2H copy per chunk)
  int* dact = h->active;
  int* dit = h->active + R;
  int* dflag = h->active + 2 * R;
  int nact = 0;
  for (int r = 0; r < R; ++r) {
    h->hactive[r] = bb[r] > 0.0;
    h->hactive[R + r] = 0;
    h->hactive[2 * R + r] = 0;
    nact += h->hactive[r];
  }
  // Inner tolerance.  With the double-FP32 outer apply and a coefficient jump
  // (cancellation costs it accuracy) CG runs to a relative 1e-8 of the residual
  // it starts from, and the FP64 confirmation below restarts it from the true
  // residual until tol is met: iterative refinement with a cheap inner apply.
  const double inner = (h->use_df && h->op->mu_contrast > 10.0) ? 1e-8 : 0.0;
  auto set_tol = [&](const double* start_rr) -> ldgmg_status {
    for (int r = 0; r < R; ++r) {
      const double t2 = tol * tol, i2 = inner * inner * (start_rr[r] / (bb[r] > 0.0 ? bb[r] : 1.0));
      h->hscal[S_TOL2 * R + r] = std::max(t2, i2);
    }
    CK(cudaMemcpyAsync(slot(S_TOL2), hslot(S_TOL2), R * sizeof(double), cudaMemcpyHostToDevice, st));
    return LDGMG_OK;
  };
  CK(cudaMemcpyAsync(h->active, h->hactive, 3 * R * sizeof(int), cudaMemcpyHostToDevice, st));
  CKS(set_tol(bb.data()));
  CK(cudaMemsetAsync(xg, 0, nb, st));
  ldgmg_status result = LDGMG_OK;
  std::vector<int> it(R, 0);
  int k = 0;
  bool true_res_fresh = false;
  if (nact > 0) {
    CK(cudaMemcpyAsync(h->r, b, nb, cudaMemcpyDeviceToDevice, st));
    CKS(apply_V(h, h->r, h->z, R, st));
    CK(cudaMemcpyAsync(h->p, h->z, nb, cudaMemcpyDeviceToDevice, st));
    CK(dot_batched(N, R, int(bsz), h->r, h->z, h->partials, slot(S_RZ), st));
    // Batched hierarchies apply A once per block row for all right-hand sides,
    // in double-FP32 (use_df) or FP64.  The arithmetic of each right-hand side
    // does not depend on R, so a right-hand side solved alone matches the batch.
    // Multi-RHS hierarchies use the same outer apply for every R (so each
    // right-hand side is bitwise the same alone and batched): the block-reuse
    // kernels for b = 16 / 64, else the CUDA-core kernel.
    // One CG iteration (Sec. 2.2).  The stopping test runs on the device right
    // after the residual norms (cg_check_b), so a converged right-hand side is
    // frozen (alpha = beta = 0) at the same iteration as with a host test, and
    // several iterations can run between host reads; work after the last
    // right-hand side converged changes nothing.
    // part 1: q = A p, alpha, x and r updates, residual norms, stopping test
    auto step = [&](cudaStream_t s) -> ldgmg_status {
      CKS(krylov_apply(h, h->p, h->q, R, s));
      CK(dot_batched(N, R, int(bsz), h->p, h->q, h->partials, slot(S_PQ), s));
      CK(cg_alpha_b(R, S, dact, s));
      CK(cg_update_xr_b(N, R, int(bsz), xg, h->r, h->p, h->q, S, s));
      CK(dot_batched(N, R, int(bsz), h->r, nullptr, h->partials, slot(S_RR), s));
      CK(cg_check_b(R, S, dact, dit, dflag, h->hist, h->o.max_iter + 1, s));
      return LDGMG_OK;
    };
    // part 2: z = V r, beta, new direction p
    auto precondition = [&](cudaStream_t s) -> ldgmg_status {
      if (flexible) CK(dot_batched(N, R, int(bsz), h->r, h->z, h->partials, slot(S_RZOLD), s));
      CKS(apply_V(h, h->r, h->z, R, s, false));
      CK(dot_batched(N, R, int(bsz), h->r, h->z, h->partials, slot(S_RZNEW), s));
      CK(cg_beta_b(R, S, dact, flexible ? 1 : 0, s));
      CK(cg_update_p_b(N, R, int(bsz), h->p, h->z, S, s));
      return LDGMG_OK;
    };
    auto body = [&](cudaStream_t s) -> ldgmg_status {
      CKS(step(s));
      return precondition(s);
    };
    // Chunk length: large solves read the stopping state after every
    // iteration's residual norms (as a host test would) and run the V-cycle
    // part only while something is active: two graphs per iteration.  Small
    // solves (launch and synchronisation bound) run four whole iterations per
    // read; the work after the last right-hand side converged changes nothing.
    const int chunk = n >= (int64_t(1) << 19) ? 1 : 4;
    auto read_state = [&]() -> ldgmg_status {
      CK(cudaMemcpyAsync(h->hactive, h->active, 3 * R * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      nact = 0;
      for (int r = 0; r < R; ++r) {
        nact += h->hactive[r];
        it[r] = h->hactive[R + r];
        if (h->hactive[2 * R + r] && result == LDGMG_OK)
          result = fail(LDGMG_ENOTCONV, "CG breakdown (non-finite residual)");
      }
      return LDGMG_OK;
    };
    for (int round = 0;; ++round) {
      while (nact > 0 && k < h->o.max_iter) {
        if (chunk == 1) {
          CKS(run_graphed(h, graph_key(G_CG, R, 0), st, step));
          ++k;
          CKS(read_state());
          if (nact > 0 && k < h->o.max_iter) CKS(run_graphed(h, graph_key(G_CG, R, 8), st, precondition));
          continue;
        }
        const int c = std::min(chunk, h->o.max_iter - k);
        CKS(run_graphed(h, graph_key(G_CG, R, c), st, [&](cudaStream_t s) -> ldgmg_status {
          for (int i = 0; i < c; ++i) CKS(body(s));
          return LDGMG_OK;
        }));
        k += c;
        CKS(read_state());
      }
      // With a reduced-precision V-cycle the recurrence residual can drift from
      // the true one (flexible CG, large coefficient jumps): confirm every
      // right-hand side on its FP64 residual b - A x and restart the ones that
      // miss tol from it (r = b - A x, z = V r, p = z).  Restarting touches
      // r, z, p of every right-hand side, which frozen ones no longer read.
      if (!flexible || nact > 0 || k >= h->o.max_iter || result != LDGMG_OK || round >= 16) break;
      CKS(true_residual(h, xg, b, h->r, R, st));
      CK(dot_batched(N, R, int(bsz), h->r, nullptr, h->partials, slot(S_TMP), st));
      CKS(read_slot(h, S_TMP, R, st));
      true_res_fresh = true;
      int again = 0;
      for (int r = 0; r < R; ++r) {
        const bool miss = bb[r] > 0.0 && !(hslot(S_TMP)[r] <= tol * tol * bb[r]);
        h->hactive[r] = miss;
        again += miss;
      }
      if (again == 0) break;
      true_res_fresh = false;
      nact = again;
      CKS(set_tol(hslot(S_TMP)));
      CK(cudaMemcpyAsync(h->active, h->hactive, R * sizeof(int), cudaMemcpyHostToDevice, st));
      CKS(apply_V(h, h->r, h->z, R, st));
      CK(cudaMemcpyAsync(h->p, h->z, nb, cudaMemcpyDeviceToDevice, st));
      CK(dot_batched(N, R, int(bsz), h->r, h->z, h->partials, slot(S_RZ), st));
    }
    if (nact > 0 && result == LDGMG_OK) result = fail(LDGMG_ENOTCONV, "max_iter reached");
  }
  // residual history of this solve (host copy for ldgmg_solve_history)
  {
    const int kmax = std::min(k, h->o.max_iter);
    h->hist_R = R;
    h->hhist.assign(size_t(kmax + 1) * R, 0.0);
    if (kmax > 0)
      CK(cudaMemcpyAsync(h->hhist.data() + R, h->hist + R, size_t(kmax) * R * sizeof(double),
                         cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    h->hist_len.assign(R, 1);
    h->hist_b2 = bb;
    for (int r = 0; r < R; ++r) {
      h->hhist[r] = bb[r];
      h->hist_len[r] = std::min(it[r], kmax) + 1;
    }
  }
  double* xd = xg;
  // true residual of the returned iterates (already in S_TMP when the
  // flexible confirmation just computed it for this x)
  if (!true_res_fresh) {
    CKS(true_residual(h, xd, b, h->r, R, st));
    CK(dot_batched(N, R, int(bsz), h->r, nullptr, h->partials, slot(S_TMP), st));
    CKS(read_slot(h, S_TMP, R, st));
  }
  if (R > 1) {
    double* dst = host_x ? h->stage_x : x;
    CK(batch_to_stack(N, R, int(bsz), xd, dst, st));
    if (host_x) CK(cudaMemcpyAsync(x, h->stage_x, nb, cudaMemcpyDeviceToHost, st));
  } else {
    CK(cudaMemcpyAsync(x, xd, nb, host_x ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  }
  CK(cudaStreamSynchronize(st));
  for (int r = 0; r < R; ++r) {
    if (iters) iters[r] = it[r];
    if (relres) relres[r] = bb[r] > 0.0 ? std::sqrt(hslot(S_TMP)[r] / bb[r]) : 0.0;
  }
  if (h->batched) {
    ldgmg_status e = check_err_flag(h, st);
    if (e != LDGMG_OK) return e;
  }
  return result;
}

// ---------------------------------------------------------------------------
// grouped solves (group.cu): many small problems, one launch per cluster size
// ---------------------------------------------------------------------------

}  // extern "C"

struct ldgmg_group {
  char* dev = nullptr;       // descriptors, staged vectors, per-problem work space
  size_t dev_cap = 0;
  char* host = nullptr;      // pinned mirror of the descriptor and staging regions
  size_t host_cap = 0;
  // the launches of the second to fourth cluster size run beside the first,
  // on side streams ordered after the copy-in (ev[0]) and joined back (ev[1..3])
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

static std::string group_ineligible(const ldgmg_hier* h) {
  if (h->batched) return "a tensor-core (batched) hierarchy";
  if (h->gmres) return "a GMRES (Stokes) hierarchy";
  if (h->op->host.nf != 1) return "a multi-field operator";
  if (h->lv.size() > size_t(kGroupMaxLevels)) return "more than 12 levels";
  return "";
}

// A grouped solve is latency bound (each step is a few L2 round trips per
// thread, then a barrier): about two unknowns per thread, i.e. 1024 per
// 512-thread CTA of the cluster, up to 8 CTAs.
static int group_cluster_of(const ldgmg_hier* h) {
  const int64_t n0 = h->op->host.N * h->op->host.b;
  int c = 1;
  while (c < 8 && n0 > int64_t(c) * 1024) c *= 2;
  return c;
}

static GroupMat group_mat(const DevMat& M) {
  GroupMat g;
  g.row_ptr = M.row_ptr;
  g.col = M.col;
  g.vals = M.vals;
  g.prec = M.prec;
  g.cs = M.cs;
  g.inv_scale = 1.0 / M.scale;
  return g;
}

// descriptor of hierarchy h; colour pointers of Gauss-Seidel levels are
// appended to cptr (their device copy will start at cptr_dev + cptr.size()
// at entry); returns the level-vector entries one problem needs
static int64_t group_problem(const ldgmg_hier* h, GroupProblem& P, std::vector<int>& cptr, const int* cptr_dev) {
  std::memset(&P, 0, sizeof P);
  const HostLevel& L0 = h->op->host;
  P.dim = L0.dim;
  P.q = L0.p + 1;
  P.nl = int(h->lv.size());
  P.smoother = h->o.smoother == LDGMG_SAI ? G_SAI : (h->o.smoother == LDGMG_JACOBI ? G_JACOBI : G_GS);
  P.pre_bt = h->o.pre_form == LDGMG_FORM_BT;
  P.post_bt = h->o.post_form == LDGMG_FORM_BT;
  P.nu1 = h->o.nu1;
  P.nu2 = h->o.nu2;
  P.vprec = h->vprec;
  P.flexible = h->prec != P_FP64;
  P.max_iter = h->o.max_iter;
  P.omega = h->o.omega;
  P.P = h->P1d;
  P.pinv = h->pinv;
  P.nbot = h->nbot;
  P.A0 = group_mat(h->op->A);
  P.n0 = L0.N * L0.b;
  int64_t off = 0;
  for (int l = 0; l < P.nl; ++l) {
    const DevLevel& D = h->lv[l];
    GroupLevel& G = P.lv[l];
    G.N = D.N;
    G.n = D.n;
    G.b = D.b;
    G.A = group_mat(D.A);
    G.S = group_mat(D.S);
    G.ST = group_mat(D.ST);
    if (P.smoother == G_GS && l + 1 < P.nl) {
      G.crows = D.crows;
      G.ncolours = int(D.cptr.size()) - 1;
      G.cptr = cptr_dev + cptr.size();
      for (int64_t v : D.cptr) cptr.push_back(int(v));
    }
    G.voff = off;
    off += 3 * D.N * D.b;
  }
  return off;
}

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

extern "C" {

ldgmg_status ldgmg_group_create(ldgmg_group** out) {
  g_err.clear();
  if (!out) return fail(LDGMG_EINVAL, "null argument");
  *out = new (std::nothrow) ldgmg_group();
  return *out ? LDGMG_OK : fail(LDGMG_ENOMEM, "host allocation");
}

void ldgmg_group_free(ldgmg_group* g) {
  if (!g) return;
  for (cudaStream_t& x : g->side)
    if (x) cudaStreamDestroy(x);
  for (cudaEvent_t& e : g->ev)
    if (e) cudaEventDestroy(e);
  cudaFree(g->dev);
  cudaFreeHost(g->host);
  delete g;
}

ldgmg_status ldgmg_group_cluster(const ldgmg_hier* h, int* cluster) {
  g_err.clear();
  if (!h || !cluster) return fail(LDGMG_EINVAL, "null argument");
  *cluster = group_ineligible(h).empty() ? group_cluster_of(h) : 0;
  return LDGMG_OK;
}

ldgmg_status ldgmg_solve_group(ldgmg_group* g, int count, ldgmg_hier* const* hs, const double* const* rhs,
                               double* const* x, const double* tol, int* iters, double* relres,
                               ldgmg_status* status, void* stream) {
  NvtxRange nvtx_("ldgmg_solve_group");
  g_err.clear();
  if (!g) return fail(LDGMG_EINVAL, "null group");
  if (count < 0 || count > (1 << 20)) return fail(LDGMG_EINVAL, "count must be in 0..2^20");
  if (count == 0) return LDGMG_OK;
  if (!hs || !rhs || !x || !tol) return fail(LDGMG_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  // distinct hierarchies, eligibility, cluster sizes
  std::map<const ldgmg_hier*, int> pid;
  std::vector<const ldgmg_hier*> uniq;
  std::vector<int> item_prob(count), item_c(count);
  std::vector<char> hb(count), hx(count);
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !rhs[i] || !x[i]) return fail(LDGMG_EINVAL, "null hierarchy or vector of problem " + std::to_string(i));
    if (!(tol[i] > 0.0)) return fail(LDGMG_EINVAL, "tol must be positive");
    auto it = pid.find(hs[i]);
    if (it == pid.end()) {
      const std::string why = group_ineligible(hs[i]);
      if (!why.empty()) return fail(LDGMG_EUNSUPPORTED, "grouped solves do not take " + why);
      it = pid.emplace(hs[i], int(uniq.size())).first;
      uniq.push_back(hs[i]);
    }
    item_prob[i] = it->second;
    item_c[i] = group_cluster_of(hs[i]);
    hb[i] = is_host_ptr(rhs[i]);
    hx[i] = is_host_ptr(x[i]);
  }
  const int np = int(uniq.size());
  // launch order: by cluster size
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return item_c[a] < item_c[b]; });
  // descriptors (the cptr device address is fixed once the layout is known, so
  // take the sizes in a first pass)
  std::vector<GroupProblem> probs(static_cast<size_t>(np));
  std::vector<int> cptr;
  std::vector<int64_t> lvec(np), n0(np);
  std::vector<int> vsz(np);
  for (int k = 0; k < np; ++k) {
    lvec[k] = group_problem(uniq[k], probs[k], cptr, nullptr);
    n0[k] = probs[k].n0;
    vsz[k] = probs[k].vprec == 0 ? 8 : 4;
  }
  // layout: region H2D [probs | items | cptr | staged rhs], region D2H [outs | staged x],
  // then per-problem work space (level vectors, CG vectors)
  size_t off = 0;
  const size_t o_probs = off;
  off = align256(off + sizeof(GroupProblem) * np);
  const size_t o_items = off;
  off = align256(off + sizeof(GroupItem) * count);
  const size_t o_cptr = off;
  off = align256(off + sizeof(int) * cptr.size());
  std::vector<size_t> o_b(count, 0), o_x(count, 0), o_lv(count), o_cg(count);
  for (int i = 0; i < count; ++i)
    if (hb[i]) {
      o_b[i] = off;
      off = align256(off + size_t(n0[item_prob[i]]) * 8);
    }
  const size_t h2d_end = off;
  const size_t o_outs = off;
  off = align256(off + sizeof(GroupOut) * count);
  for (int i = 0; i < count; ++i)
    if (hx[i]) {
      o_x[i] = off;
      off = align256(off + size_t(n0[item_prob[i]]) * 8);
    }
  const size_t d2h_end = off;
  for (int i = 0; i < count; ++i) {
    const int k = item_prob[i];
    o_lv[i] = off;
    off = align256(off + size_t(lvec[k]) * vsz[k]);
    o_cg[i] = off;
    off = align256(off + size_t(n0[k]) * 4 * 8);
  }
  const size_t total = off;
  if (total > g->dev_cap) {
    CK(cudaStreamSynchronize(st));
    cudaFree(g->dev);
    g->dev = nullptr;
    g->dev_cap = 0;
    const size_t want = total + total / 4;
    CK(cudaMalloc(&g->dev, want));
    g->dev_cap = want;
  }
  if (d2h_end > g->host_cap) {
    cudaFreeHost(g->host);
    g->host = nullptr;
    g->host_cap = 0;
    const size_t want = d2h_end + d2h_end / 4;
    CK(cudaMallocHost(&g->host, want));
    g->host_cap = want;
  }
  char* D = g->dev;
  char* H = g->host;
  // descriptors with their device addresses
  cptr.clear();
  for (int k = 0; k < np; ++k) group_problem(uniq[k], probs[k], cptr, reinterpret_cast<const int*>(D + o_cptr));
  std::memcpy(H + o_probs, probs.data(), sizeof(GroupProblem) * np);
  if (!cptr.empty()) std::memcpy(H + o_cptr, cptr.data(), sizeof(int) * cptr.size());
  GroupItem* items = reinterpret_cast<GroupItem*>(H + o_items);
  for (int j = 0; j < count; ++j) {
    const int i = order[j];
    const int k = item_prob[i];
    GroupItem& I = items[j];
    std::memset(&I, 0, sizeof I);
    I.prob = k;
    I.b = hb[i] ? reinterpret_cast<const double*>(D + o_b[i]) : rhs[i];
    I.x = hx[i] ? reinterpret_cast<double*>(D + o_x[i]) : x[i];
    I.tol = tol[i];
    I.lvec = D + o_lv[i];
    I.cg = reinterpret_cast<double*>(D + o_cg[i]);
    I.out = reinterpret_cast<GroupOut*>(D + o_outs) + j;
    if (hb[i]) std::memcpy(H + o_b[i], rhs[i], size_t(n0[k]) * 8);
  }
  CK(cudaMemcpyAsync(D, H, h2d_end, cudaMemcpyHostToDevice, st));
  const GroupProblem* dprobs = reinterpret_cast<const GroupProblem*>(D + o_probs);
  const GroupItem* ditems = reinterpret_cast<const GroupItem*>(D + o_items);
  std::vector<std::pair<int, int>> ranges;     // items of one cluster size
  for (int j0 = 0; j0 < count;) {
    int j1 = j0;
    while (j1 < count && item_c[order[j1]] == item_c[order[j0]]) ++j1;
    ranges.emplace_back(j0, j1);
    j0 = j1;
  }
  if (ranges.size() > 1) {
    for (size_t k = 0; k < ranges.size(); ++k) {
      if (!g->ev[k]) CK(cudaEventCreateWithFlags(&g->ev[k], cudaEventDisableTiming));
      if (k > 0 && !g->side[k - 1]) CK(cudaStreamCreateWithFlags(&g->side[k - 1], cudaStreamNonBlocking));
    }
    CK(cudaEventRecord(g->ev[0], st));
  }
  for (size_t k = 0; k < ranges.size(); ++k) {
    cudaStream_t sk = k == 0 ? st : g->side[k - 1];
    if (k > 0) CK(cudaStreamWaitEvent(sk, g->ev[0], 0));
    const int j0 = ranges[k].first, j1 = ranges[k].second;
    CK(group_solve(dprobs, ditems + j0, j1 - j0, item_c[order[j0]], sk));
    if (k > 0) CK(cudaEventRecord(g->ev[k], sk));
  }
  for (size_t k = 1; k < ranges.size(); ++k) CK(cudaStreamWaitEvent(st, g->ev[k], 0));
  CK(cudaMemcpyAsync(H + o_outs, D + o_outs, d2h_end - o_outs, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const GroupOut* outs = reinterpret_cast<const GroupOut*>(H + o_outs);
  int first_bad = count;          // lowest failing problem index
  int first_code = 0;
  for (int j = 0; j < count; ++j) {
    const int i = order[j];
    const GroupOut& o = outs[j];
    const ldgmg_status si = o.status == 0 ? LDGMG_OK : (o.status == 3 ? LDGMG_EINVAL : LDGMG_ENOTCONV);
    if (iters) iters[i] = o.iters;
    if (relres) relres[i] = o.relres;
    if (status) status[i] = si;
    if (hx[i]) std::memcpy(x[i], H + o_x[i], size_t(n0[item_prob[i]]) * 8);
    if (si != LDGMG_OK && i < first_bad) {
      first_bad = i;
      first_code = o.status;
    }
  }
  if (first_bad < count) {
    const ldgmg_status r = first_code == 3 ? LDGMG_EINVAL : LDGMG_ENOTCONV;
    return fail(r, "problem " + std::to_string(first_bad) +
                       (first_code == 3 ? ": rhs contains NaN or Inf"
                                        : (first_code == 2 ? ": CG breakdown (non-finite residual)"
                                                           : ": max_iter reached")));
  }
  return LDGMG_OK;
}

// ---------------------------------------------------------------------------
// per-level entry points
// ---------------------------------------------------------------------------

static ldgmg_status check_level(ldgmg_hier* h, int l, bool need_smoother) {
  if (!h) return fail(LDGMG_EINVAL, "null hierarchy");
  if (l < 0 || l >= int(h->lv.size())) return fail(LDGMG_EINVAL, "level out of range");
  if (need_smoother && l == int(h->lv.size()) - 1) return fail(LDGMG_EINVAL, "bottom level has no smoother");
  return LDGMG_OK;
}

static const DevMat* level_mat(ldgmg_hier* h, int l, int which) {
  const DevLevel& D = h->lv[l];
  if (which == LDGMG_MAT_A) return &D.A;
  if (which == LDGMG_MAT_D && (h->o.smoother == LDGMG_JACOBI || h->o.smoother == LDGMG_GS)) return &D.S;
  if (which == LDGMG_MAT_B && h->o.smoother == LDGMG_SAI) return &D.S;
  if (which == LDGMG_MAT_BT && h->o.smoother == LDGMG_SAI) return &D.ST;
  return nullptr;
}

ldgmg_status ldgmg_level_apply(ldgmg_hier* h, int l, int which, const void* x, void* y, void* stream) {
  CKS(check_level(h, l, which != LDGMG_MAT_A));
  if (!x || !y) return fail(LDGMG_EINVAL, "null vector");
  const DevMat* M = level_mat(h, l, which);
  if (!M) return fail(LDGMG_EINVAL, "matrix not present for this smoother");
  return apply_mat(h, *M, M_Y, x, nullptr, nullptr, y, 1.0, 1, (cudaStream_t)stream);
}

ldgmg_status ldgmg_level_apply_batched(ldgmg_hier* h, int l, int which, int nrhs, const float* x, float* y,
                                       void* stream) {
  CKS(check_level(h, l, which != LDGMG_MAT_A));
  if (!x || !y) return fail(LDGMG_EINVAL, "null vector");
  if (nrhs < 1 || nrhs > 128) return fail(LDGMG_EINVAL, "nrhs must be in 1..128");
  if (h->vprec != 1) return fail(LDGMG_EUNSUPPORTED, "batched level apply needs an FP32 or BF16 hierarchy");
  const DevMat* M = level_mat(h, l, which);
  if (!M) return fail(LDGMG_EINVAL, "matrix not present for this smoother");
  return apply_mat(h, *M, M_Y, x, nullptr, nullptr, y, 1.0, nrhs, (cudaStream_t)stream);
}

ldgmg_status ldgmg_level_smooth(ldgmg_hier* h, int l, int form, const void* rhs, const void* xin, void* xout,
                                int x_is_zero, void* stream) {
  CKS(check_level(h, l, true));
  if (!rhs || !xout || (!x_is_zero && !xin)) return fail(LDGMG_EINVAL, "null vector");
  if (form != LDGMG_FORM_B1 && form != LDGMG_FORM_BT) return fail(LDGMG_EINVAL, "form");
  return smooth(h, l, form, rhs, xin, xout, x_is_zero != 0, 1, (cudaStream_t)stream);
}

ldgmg_status ldgmg_level_restrict(ldgmg_hier* h, int l, const void* rhs, const void* x, void* rc,
                                  void* stream) {
  CKS(check_level(h, l, true));
  if (!rhs || !x || !rc) return fail(LDGMG_EINVAL, "null vector");
  return restrict_residual(h, l, rhs, x, false, rc, 1, (cudaStream_t)stream);
}

ldgmg_status ldgmg_level_prolong(ldgmg_hier* h, int l, const void* xc, void* x, void* stream) {
  CKS(check_level(h, l, true));
  if (!xc || !x) return fail(LDGMG_EINVAL, "null vector");
  CK(prolong_apply(h->op->host.dim, h->op->host.p + 1, h->lv[l].n, h->P1d, xc, x, h->vprec, h->op->host.nf,
                   (cudaStream_t)stream));
  return LDGMG_OK;
}

ldgmg_status ldgmg_bottom_solve(ldgmg_hier* h, const void* rhs, void* x, void* stream) {
  if (!h || !rhs || !x) return fail(LDGMG_EINVAL, "null argument");
  CK(dense_gemv(h->nbot, h->lv.back().b, h->pinv, rhs, x, h->vprec, 1, (cudaStream_t)stream));
  return LDGMG_OK;
}

static double fp16_to_double(uint16_t v) {
  const int sign = v >> 15, ex = (v >> 10) & 0x1F, man = v & 0x3FF;
  double mag;
  if (ex == 0) mag = std::ldexp(double(man), -24);                 // subnormal
  else if (ex == 31) mag = man ? NAN : INFINITY;
  else mag = std::ldexp(double(man | 0x400), ex - 25);
  return sign ? -mag : mag;
}

static float bf16_to_float(uint16_t v) {
  uint32_t u = uint32_t(v) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

ldgmg_status ldgmg_export_level(ldgmg_hier* h, int l, int which, int64_t* row_ptr, int32_t* col, double* vals) {
  CKS(check_level(h, l, which != LDGMG_MAT_A));
  const DevMat* M = level_mat(h, l, which);
  if (!M) return fail(LDGMG_EINVAL, "matrix not present for this smoother");
  CK(cudaDeviceSynchronize());
  if (row_ptr) {
    std::vector<int> rp(M->nrows + 1);
    CK(cudaMemcpy(rp.data(), M->row_ptr, rp.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < rp.size(); ++i) row_ptr[i] = rp[i];
  }
  if (col && M->nnzb) CK(cudaMemcpy(col, M->col, M->nnzb * sizeof(int), cudaMemcpyDeviceToHost));
  if (vals && M->nnzb) {
    const int b = M->b, cs = M->cs;
    const size_t cnt = size_t(M->nnzb) * b * cs;      // stored entries (padding included)
    std::vector<char> raw(cnt * esize(M->prec));
    CK(cudaMemcpy(raw.data(), M->vals, raw.size(), cudaMemcpyDeviceToHost));
    if (M->tc_image) {
      // operand images: BF16 hi (+ lo for FP32 storage); the stored value is hi + lo
      const size_t img = size_t(b) * b * 2, per = M->prec == P_FP32 ? 2 * img : img;
      for (size_t nz = 0; nz < size_t(M->nnzb); ++nz)
        for (int r = 0; r < b; ++r)
          for (int c = 0; c < b; ++c) {
            const char* blk = raw.data() + nz * per;
            const uint32_t off = tc_image_offset(b, r, c);
            uint16_t u;
            std::memcpy(&u, blk + off, 2);
            double v = bf16_to_float(u);
            if (M->prec == P_FP32) {
              std::memcpy(&u, blk + img + off, 2);
              v = double(float(v) + bf16_to_float(u));
            }
            vals[nz * b * b + r * b + c] = v / M->scale;
          }
      return LDGMG_OK;
    }
    for (size_t t = 0; t < cnt; ++t) {
      const size_t nz = t / (size_t(b) * cs), e = t % (size_t(b) * cs);
      const size_t c = e / cs, r = e % cs;
      if (r >= size_t(b)) continue;
      double v;
      if (M->prec == P_FP64) v = reinterpret_cast<const double*>(raw.data())[t];
      else if (M->prec == P_FP32) v = reinterpret_cast<const float*>(raw.data())[t];
      else if (M->prec == P_BF16) v = bf16_to_float(reinterpret_cast<const uint16_t*>(raw.data())[t]);
      else v = fp16_to_double(reinterpret_cast<const uint16_t*>(raw.data())[t]);
      vals[nz * b * b + r * b + c] = v / M->scale;
    }
  }
  return LDGMG_OK;
}

}  // extern "C"
