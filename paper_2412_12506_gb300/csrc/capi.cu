// C ABI of the LDG multigrid library (declared in include/ldgmg.h).
//
// Setup (assembly, operator coarsening, smoother construction) runs in host
// C++ on pooled block storage (host.cpp), then every level matrix is
// expanded on the device into explicit block-CSR in the requested precision.
// The bottom pseudo-inverse comes from a cuSOLVER FP64 eigendecomposition on
// the device.  Everything the V-cycle and CG touch afterwards is device
// resident; the host only enqueues kernels and reads one scalar per CG
// iteration for the stopping test.
#include "ldgmg.h"

#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "host.h"
#include "kernels.h"

using namespace ldgmg;

static thread_local std::string g_err;

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

template <class T>
static ldgmg_status dalloc(T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return LDGMG_OK;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(LDGMG_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
  }
  return LDGMG_OK;
}

static void free_mat(DevMat& M) {
  cudaFree(M.row_ptr);
  cudaFree(M.col);
  cudaFree(M.vals);
  M = DevMat();
}

// Expand a pooled host matrix into an explicit device block-CSR of precision prec.
static ldgmg_status upload(const PBSR& H, int b, int prec, DevMat& M, cudaStream_t st) {
  if (H.nnzb() >= (int64_t(1) << 31)) return fail(LDGMG_EUNSUPPORTED, "more than 2^31 blocks");
  M.nrows = H.nrows;
  M.nnzb = H.nnzb();
  M.b = b;
  M.prec = prec;
  std::vector<int> rp(H.row_ptr.begin(), H.row_ptr.end());
  CKS(dalloc(&M.row_ptr, rp.size() * sizeof(int)));
  CKS(dalloc(&M.col, H.col.size() * sizeof(int)));
  CKS(dalloc((char**)&M.vals, size_t(M.nnzb) * b * b * esize(prec)));
  CK(cudaMemcpyAsync(M.row_ptr, rp.data(), rp.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (M.nnzb) CK(cudaMemcpyAsync(M.col, H.col.data(), H.col.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  uint32_t* d_ids = nullptr;
  double* d_pool = nullptr;
  CKS(dalloc(&d_ids, H.id.size() * sizeof(uint32_t)));
  CKS(dalloc(&d_pool, H.pool.data.size() * sizeof(double)));
  if (M.nnzb) {
    CK(cudaMemcpyAsync(d_ids, H.id.data(), H.id.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_pool, H.pool.data.data(), H.pool.data.size() * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    CK(expand_blocks(M.nnzb, b, d_ids, d_pool, M.vals, prec, st));
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
  DevMat A;              // FP64 finest-level operator
  double tau0 = 1.0;
  double* partials = nullptr;
  double* scal = nullptr;
};

struct DevLevel {
  int n = 0;
  int64_t N = 0;
  int b = 0;
  DevMat A, S, ST;       // A_l; smoother matrix (B_l or D_l); B_l^T (SAI only)
  bool own_A = true;
  void* rhs = nullptr;
  void* x = nullptr;
  void* r = nullptr;
};

struct ldgmg_hier {
  ldgmg_op* op = nullptr;
  ldgmg_setup_opts o;
  int prec = P_FP64;
  int vprec = 0;         // 0: double level vectors, 1: float
  size_t vsz = 8;
  std::vector<HostLevel> host;   // host[0] is unused (the op holds the finest level)
  std::vector<DevLevel> lv;
  double* P1d = nullptr;         // 2 * q * q injection matrices
  double* pinv = nullptr;        // bottom pseudo-inverse, nbot x nbot
  int64_t nbot = 0;
  // CG work space (FP64)
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *xk = nullptr;
  double *scal = nullptr, *partials = nullptr;
  double *stage_rhs = nullptr, *stage_x = nullptr;
  double* hscal = nullptr;       // pinned host mirror of the CG scalars
};

static const HostLevel& host_level(const ldgmg_hier* h, int l) {
  return l == 0 ? h->op->host : h->host[l];
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
}

void ldgmg_op_free(ldgmg_op* op) {
  if (!op) return;
  free_mat(op->A);
  cudaFree(op->partials);
  cudaFree(op->scal);
  delete op;
}

ldgmg_status ldgmg_assemble(const ldgmg_mesh* mesh, int p, const double* mu_host, double tau0,
                            ldgmg_op** out) {
  g_err.clear();
  if (!mesh || !out) return fail(LDGMG_EINVAL, "null argument");
  *out = nullptr;
  if (!mesh->periodic) return fail(LDGMG_EUNSUPPORTED, "only periodic meshes are supported");
  if (mesh->dim != 2 && mesh->dim != 3) return fail(LDGMG_EINVAL, "dim must be 2 or 3");
  if (mesh->n < 1 || mesh->n > 4096) return fail(LDGMG_EINVAL, "n out of range");
  int b = 1;
  for (int t = 0; t < mesh->dim; ++t) b *= (p + 1);
  if (p < 1 || !block_size_supported(b)) return fail(LDGMG_EUNSUPPORTED, "unsupported block size");
  ldgmg_op* op = new (std::nothrow) ldgmg_op();
  if (!op) return fail(LDGMG_ENOMEM, "host allocation");
  std::string err = assemble_fine(op->host, mesh->dim, mesh->n, p, mu_host, tau0);
  if (!err.empty()) {
    delete op;
    return fail(LDGMG_EINVAL, err);
  }
  op->tau0 = tau0;
  ldgmg_status s = upload(op->host.A, b, P_FP64, op->A, 0);
  if (s == LDGMG_OK) s = dalloc(&op->partials, kDotBlocks * sizeof(double));
  if (s == LDGMG_OK) s = dalloc(&op->scal, kCgSlots * sizeof(double));
  if (s != LDGMG_OK) {
    ldgmg_op_free(op);
    return s;
  }
  *out = op;
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
  if (nrhs != 1) return fail(LDGMG_EUNSUPPORTED, "nrhs must be 1");
  CK(bsr_apply(op->A, M_Y, x, nullptr, nullptr, y, 1.0, (cudaStream_t)stream));
  return LDGMG_OK;
}

ldgmg_status ldgmg_project_kernel(ldgmg_op* op, double* v, int nrhs, void* stream) {
  if (!op || !v) return fail(LDGMG_EINVAL, "null argument");
  if (nrhs != 1) return fail(LDGMG_EUNSUPPORTED, "nrhs must be 1");
  cudaStream_t st = (cudaStream_t)stream;
  // c has equal mode-0 entries and zeros elsewhere, so the projection
  // subtracts the mean of the mode-0 coefficients from each of them.
  CK(strided_sum(op->host.N, op->host.b, v, op->partials, op->scal, st));
  CK(strided_sub_mean(op->host.N, op->host.b, v, op->scal, st));
  return LDGMG_OK;
}

void ldgmg_hier_free(ldgmg_hier* h) {
  if (!h) return;
  for (auto& L : h->lv) {
    if (L.own_A) free_mat(L.A);
    free_mat(L.S);
    free_mat(L.ST);
    cudaFree(L.rhs);
    cudaFree(L.x);
    cudaFree(L.r);
  }
  cudaFree(h->P1d);
  cudaFree(h->pinv);
  for (double* v : {h->r, h->z, h->p, h->q, h->xk, h->scal, h->partials, h->stage_rhs, h->stage_x}) cudaFree(v);
  if (h->hscal) cudaFreeHost(h->hscal);
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
  // symmetrise against rounding
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      const double m = 0.5 * (dense[i * n + j] + dense[j * n + i]);
      dense[i * n + j] = dense[j * n + i] = m;
    }
  h->nbot = n;
  double *dA = nullptr, *dW = nullptr, *dWork = nullptr, *dU2 = nullptr, *dInv = nullptr;
  int* dInfo = nullptr;
  CKS(dalloc(&dA, size_t(n) * n * sizeof(double)));
  CKS(dalloc(&dU2, size_t(n) * n * sizeof(double)));
  CKS(dalloc(&dW, n * sizeof(double)));
  CKS(dalloc(&dInv, n * sizeof(double)));
  CKS(dalloc(&dInfo, sizeof(int)));
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
  if ((status = dalloc(&dWork, size_t(lwork) * sizeof(double))) != LDGMG_OK) goto done;
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

ldgmg_status ldgmg_setup(ldgmg_op* op, const ldgmg_setup_opts* o, void* stream, ldgmg_hier** out) {
  g_err.clear();
  if (!op || !o || !out) return fail(LDGMG_EINVAL, "null argument");
  *out = nullptr;
  if (o->smoother != LDGMG_JACOBI && o->smoother != LDGMG_SAI) return fail(LDGMG_EINVAL, "smoother");
  if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 > 64 || o->nu2 > 64) return fail(LDGMG_EINVAL, "nu1/nu2");
  if (o->vcycle_precision < 0 || o->vcycle_precision > 2) return fail(LDGMG_EINVAL, "precision");
  if (o->max_iter < 1) return fail(LDGMG_EINVAL, "max_iter");
  if (o->smoother == LDGMG_JACOBI && !(o->omega > 0.0 && o->omega < 2.0)) return fail(LDGMG_EINVAL, "omega");
  cudaStream_t st = (cudaStream_t)stream;
  ldgmg_hier* h = new (std::nothrow) ldgmg_hier();
  if (!h) return fail(LDGMG_ENOMEM, "host allocation");
  h->op = op;
  h->o = *o;
  h->prec = o->vcycle_precision;
  h->vprec = h->prec == P_FP64 ? 0 : 1;
  h->vsz = h->vprec ? 4 : 8;
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
      s = upload(L.A, L.b, h->prec, D.A, st);
    }
    if (s == LDGMG_OK && l + 1 < nl) {
      if (o->smoother == LDGMG_SAI) {
        s = upload(L.B, L.b, h->prec, D.S, st);
        if (s == LDGMG_OK) s = upload(L.BT, L.b, h->prec, D.ST, st);
      } else {
        s = upload(jacobi_pbsr(L), L.b, h->prec, D.S, st);
      }
    }
    const size_t vb = size_t(L.N) * L.b * h->vsz;
    if (s == LDGMG_OK) s = dalloc((char**)&D.rhs, vb);
    if (s == LDGMG_OK) s = dalloc((char**)&D.x, vb);
    if (s == LDGMG_OK) s = dalloc((char**)&D.r, vb);
    if (s != LDGMG_OK) return bail(s);
  }
  {
    ldgmg_status s = bottom_pinv(h, host_level(h, nl - 1), st);
    if (s != LDGMG_OK) return bail(s);
  }
  const size_t n0 = size_t(L0.N) * L0.b * sizeof(double);
  for (double** v : {&h->r, &h->z, &h->p, &h->q, &h->xk, &h->stage_rhs, &h->stage_x}) {
    ldgmg_status s = dalloc(v, n0);
    if (s != LDGMG_OK) return bail(s);
  }
  if (dalloc(&h->scal, kCgSlots * sizeof(double)) != LDGMG_OK ||
      dalloc(&h->partials, kDotBlocks * sizeof(double)) != LDGMG_OK)
    return bail(LDGMG_ENOMEM);
  if (cudaMallocHost((void**)&h->hscal, kCgSlots * sizeof(double)) != cudaSuccess)
    return bail(fail(LDGMG_ENOMEM, "cudaMallocHost"));
  if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(LDGMG_ECUDA, "setup sync"));
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
// V-cycle steps
// ---------------------------------------------------------------------------

static ldgmg_status smooth(ldgmg_hier* h, int l, int form, const void* rhs, const void* xin, void* xout,
                           bool x_zero, cudaStream_t st) {
  DevLevel& D = h->lv[l];
  if (h->o.smoother == LDGMG_JACOBI) {
    // Eq. Jsmooth written as x + omega D^{-1} (b - A x)
    if (x_zero) {
      CK(bsr_apply(D.S, M_SCALE, rhs, nullptr, nullptr, xout, h->o.omega, st));
    } else {
      CK(bsr_apply(D.A, M_RES, xin, rhs, nullptr, D.r, 1.0, st));
      CK(bsr_apply(D.S, M_AXPY, D.r, nullptr, xin, xout, h->o.omega, st));
    }
    return LDGMG_OK;
  }
  // Eq. B1: x - B (A x - b) = x + B (b - A x); Eq. BT with B^T
  const DevMat& M = form == LDGMG_FORM_BT ? D.ST : D.S;
  if (x_zero) {
    CK(bsr_apply(M, M_Y, rhs, nullptr, nullptr, xout, 1.0, st));
  } else {
    CK(bsr_apply(D.A, M_RES, xin, rhs, nullptr, D.r, 1.0, st));
    CK(bsr_apply(M, M_AXPY, D.r, nullptr, xin, xout, 1.0, st));
  }
  return LDGMG_OK;
}

static ldgmg_status restrict_residual(ldgmg_hier* h, int l, const void* rhs, const void* x, bool x_zero,
                                      void* rc, cudaStream_t st) {
  DevLevel& D = h->lv[l];
  const void* r = rhs;
  if (!x_zero) {
    CK(bsr_apply(D.A, M_RES, x, rhs, nullptr, D.r, 1.0, st));
    r = D.r;
  }
  CK(restrict_apply(h->op->host.dim, h->op->host.p + 1, D.n, h->P1d, r, rc, h->vprec, st));
  return LDGMG_OK;
}

// Algorithm 1 on level l with x_l = 0 initially; rhs in lv[l].rhs, result in lv[l].x
static ldgmg_status vcycle_level(ldgmg_hier* h, int l, cudaStream_t st) {
  DevLevel& D = h->lv[l];
  const int nl = int(h->lv.size());
  if (l == nl - 1) {
    CK(dense_gemv(h->nbot, h->pinv, D.rhs, D.x, h->vprec, st));
    return LDGMG_OK;
  }
  bool xz = true;
  for (int s = 0; s < h->o.nu1; ++s) {
    CKS(smooth(h, l, h->o.pre_form, D.rhs, D.x, D.x, xz, st));
    xz = false;
  }
  CKS(restrict_residual(h, l, D.rhs, D.x, xz, h->lv[l + 1].rhs, st));
  CKS(vcycle_level(h, l + 1, st));
  if (xz) CK(cudaMemsetAsync(D.x, 0, size_t(D.N) * D.b * h->vsz, st));
  CK(prolong_apply(h->op->host.dim, h->op->host.p + 1, D.n, h->P1d, h->lv[l + 1].x, D.x, h->vprec, st));
  for (int s = 0; s < h->o.nu2; ++s) CKS(smooth(h, l, h->o.post_form, D.rhs, D.x, D.x, false, st));
  return LDGMG_OK;
}

// x = V b, FP64 device vectors
static ldgmg_status apply_V(ldgmg_hier* h, const double* b, double* x, cudaStream_t st) {
  DevLevel& D = h->lv[0];
  const int64_t n = D.N * D.b;
  if (h->vprec == 0) CK(cudaMemcpyAsync(D.rhs, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else CK(cast_d2f(n, b, (float*)D.rhs, st));
  CKS(vcycle_level(h, 0, st));
  if (h->vprec == 0) CK(cudaMemcpyAsync(x, D.x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else CK(cast_f2d(n, (const float*)D.x, x, st));
  return LDGMG_OK;
}

ldgmg_status ldgmg_vcycle(ldgmg_hier* h, const double* b, double* x, int nrhs, void* stream) {
  if (!h || !b || !x) return fail(LDGMG_EINVAL, "null argument");
  if (nrhs != 1) return fail(LDGMG_EUNSUPPORTED, "nrhs must be 1");
  return apply_V(h, b, x, (cudaStream_t)stream);
}

static bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

static ldgmg_status read_scalar(ldgmg_hier* h, int slot, double* v, cudaStream_t st) {
  CK(cudaMemcpyAsync(h->hscal + slot, h->scal + slot, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *v = h->hscal[slot];
  return LDGMG_OK;
}

ldgmg_status ldgmg_solve(ldgmg_hier* h, const double* rhs, double tol, double* x, int nrhs, int* iters,
                         double* relres, void* stream) {
  g_err.clear();
  if (!h || !rhs || !x) return fail(LDGMG_EINVAL, "null argument");
  if (nrhs != 1) return fail(LDGMG_EUNSUPPORTED, "nrhs must be 1");
  if (!(tol > 0.0)) return fail(LDGMG_EINVAL, "tol must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  const HostLevel& L0 = h->op->host;
  const int64_t n = L0.N * L0.b;
  const size_t nb = size_t(n) * sizeof(double);
  const bool host_rhs = is_host_ptr(rhs), host_x = is_host_ptr(x);
  const double* b = rhs;
  if (host_rhs) {
    CK(cudaMemcpyAsync(h->stage_rhs, rhs, nb, cudaMemcpyHostToDevice, st));
    b = h->stage_rhs;
  }
  double* xd = host_x ? h->stage_x : x;
  const bool flexible = h->prec != P_FP64;
  double bb = 0.0, rr = 0.0;
  CK(dot(n, b, b, h->partials, h->scal + S_BB, st));
  CKS(read_scalar(h, S_BB, &bb, st));
  if (!std::isfinite(bb)) return fail(LDGMG_EINVAL, "rhs contains NaN or Inf");
  CK(cudaMemsetAsync(xd, 0, nb, st));
  int k = 0;
  ldgmg_status result = LDGMG_OK;
  if (bb > 0.0) {
    const double stop2 = tol * tol * bb;
    CK(cudaMemcpyAsync(h->r, b, nb, cudaMemcpyDeviceToDevice, st));
    CKS(apply_V(h, h->r, h->z, st));
    CK(cudaMemcpyAsync(h->p, h->z, nb, cudaMemcpyDeviceToDevice, st));
    CK(dot(n, h->r, h->z, h->partials, h->scal + S_RZ, st));
    bool conv = false;
    while (k < h->o.max_iter) {
      CK(bsr_apply(h->op->A, M_Y, h->p, nullptr, nullptr, h->q, 1.0, st));
      CK(dot(n, h->p, h->q, h->partials, h->scal + S_PQ, st));
      CK(cg_alpha(h->scal, st));
      CK(cg_update_xr(n, xd, h->r, h->p, h->q, h->scal, st));
      CK(dot(n, h->r, h->r, h->partials, h->scal + S_RR, st));
      ++k;
      CKS(read_scalar(h, S_RR, &rr, st));
      if (!std::isfinite(rr)) {
        result = fail(LDGMG_ENOTCONV, "CG breakdown (non-finite residual)");
        break;
      }
      if (rr <= stop2) {
        conv = true;
        break;
      }
      if (flexible) CK(dot(n, h->r, h->z, h->partials, h->scal + S_RZOLD, st));
      CKS(apply_V(h, h->r, h->z, st));
      CK(dot(n, h->r, h->z, h->partials, h->scal + S_RZNEW, st));
      CK(cg_beta(h->scal, flexible ? 1 : 0, st));
      CK(cg_update_p(n, h->p, h->z, h->scal, st));
    }
    if (!conv && result == LDGMG_OK) result = fail(LDGMG_ENOTCONV, "max_iter reached");
  }
  // true residual of the returned iterate
  double rel = 0.0;
  if (bb > 0.0) {
    CK(bsr_apply(h->op->A, M_RES, xd, b, nullptr, h->r, 1.0, st));
    CK(dot(n, h->r, h->r, h->partials, h->scal + S_TMP, st));
    double t = 0.0;
    CKS(read_scalar(h, S_TMP, &t, st));
    rel = std::sqrt(t / bb);
  }
  if (host_x) CK(cudaMemcpyAsync(x, xd, nb, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (iters) iters[0] = k;
  if (relres) relres[0] = rel;
  return result;
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

ldgmg_status ldgmg_level_apply(ldgmg_hier* h, int l, int which, const void* x, void* y, void* stream) {
  CKS(check_level(h, l, which != LDGMG_MAT_A));
  if (!x || !y) return fail(LDGMG_EINVAL, "null vector");
  const DevLevel& D = h->lv[l];
  const DevMat* M = nullptr;
  if (which == LDGMG_MAT_A) M = &D.A;
  else if (which == LDGMG_MAT_D && h->o.smoother == LDGMG_JACOBI) M = &D.S;
  else if (which == LDGMG_MAT_B && h->o.smoother == LDGMG_SAI) M = &D.S;
  else if (which == LDGMG_MAT_BT && h->o.smoother == LDGMG_SAI) M = &D.ST;
  if (!M) return fail(LDGMG_EINVAL, "matrix not present for this smoother");
  CK(bsr_apply(*M, M_Y, x, nullptr, nullptr, y, 1.0, (cudaStream_t)stream));
  return LDGMG_OK;
}

ldgmg_status ldgmg_level_smooth(ldgmg_hier* h, int l, int form, const void* rhs, const void* xin, void* xout,
                                int x_is_zero, void* stream) {
  CKS(check_level(h, l, true));
  if (!rhs || !xout || (!x_is_zero && !xin)) return fail(LDGMG_EINVAL, "null vector");
  if (form != LDGMG_FORM_B1 && form != LDGMG_FORM_BT) return fail(LDGMG_EINVAL, "form");
  return smooth(h, l, form, rhs, xin, xout, x_is_zero != 0, (cudaStream_t)stream);
}

ldgmg_status ldgmg_level_restrict(ldgmg_hier* h, int l, const void* rhs, const void* x, void* rc,
                                  void* stream) {
  CKS(check_level(h, l, true));
  if (!rhs || !x || !rc) return fail(LDGMG_EINVAL, "null vector");
  return restrict_residual(h, l, rhs, x, false, rc, (cudaStream_t)stream);
}

ldgmg_status ldgmg_level_prolong(ldgmg_hier* h, int l, const void* xc, void* x, void* stream) {
  CKS(check_level(h, l, true));
  if (!xc || !x) return fail(LDGMG_EINVAL, "null vector");
  CK(prolong_apply(h->op->host.dim, h->op->host.p + 1, h->lv[l].n, h->P1d, xc, x, h->vprec,
                   (cudaStream_t)stream));
  return LDGMG_OK;
}

ldgmg_status ldgmg_bottom_solve(ldgmg_hier* h, const void* rhs, void* x, void* stream) {
  if (!h || !rhs || !x) return fail(LDGMG_EINVAL, "null argument");
  CK(dense_gemv(h->nbot, h->pinv, rhs, x, h->vprec, (cudaStream_t)stream));
  return LDGMG_OK;
}

static float bf16_to_float(uint16_t v) {
  uint32_t u = uint32_t(v) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

ldgmg_status ldgmg_export_level(ldgmg_hier* h, int l, int which, int64_t* row_ptr, int32_t* col, double* vals) {
  CKS(check_level(h, l, which != LDGMG_MAT_A));
  const DevLevel& D = h->lv[l];
  const DevMat* M = nullptr;
  if (which == LDGMG_MAT_A) M = &D.A;
  else if (which == LDGMG_MAT_D && h->o.smoother == LDGMG_JACOBI) M = &D.S;
  else if (which == LDGMG_MAT_B && h->o.smoother == LDGMG_SAI) M = &D.S;
  else if (which == LDGMG_MAT_BT && h->o.smoother == LDGMG_SAI) M = &D.ST;
  if (!M) return fail(LDGMG_EINVAL, "matrix not present for this smoother");
  CK(cudaDeviceSynchronize());
  if (row_ptr) {
    std::vector<int> rp(M->nrows + 1);
    CK(cudaMemcpy(rp.data(), M->row_ptr, rp.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < rp.size(); ++i) row_ptr[i] = rp[i];
  }
  if (col && M->nnzb) CK(cudaMemcpy(col, M->col, M->nnzb * sizeof(int), cudaMemcpyDeviceToHost));
  if (vals && M->nnzb) {
    const int b = M->b;
    const size_t cnt = size_t(M->nnzb) * b * b;
    std::vector<char> raw(cnt * esize(M->prec));
    CK(cudaMemcpy(raw.data(), M->vals, raw.size(), cudaMemcpyDeviceToHost));
    for (size_t t = 0; t < cnt; ++t) {
      const size_t nz = t / (size_t(b) * b), e = t % (size_t(b) * b);
      const size_t c = e / b, r = e % b;   // device storage is column-major
      double v;
      if (M->prec == P_FP64) v = reinterpret_cast<const double*>(raw.data())[t];
      else if (M->prec == P_FP32) v = reinterpret_cast<const float*>(raw.data())[t];
      else v = bf16_to_float(reinterpret_cast<const uint16_t*>(raw.data())[t]);
      vals[nz * b * b + r * b + c] = v;
    }
  }
  return LDGMG_OK;
}

}  // extern "C"
