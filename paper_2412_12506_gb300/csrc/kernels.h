// Device kernels of the LDG multigrid hot path (launchers callable from host code).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

namespace ldgmg {

enum Prec { P_FP64 = 0, P_FP32 = 1, P_BF16 = 2, P_FP16 = 3 };

// Block-CSR matrix resident on the device.  Block nz of row i is the dense
// b x b block M_{i, col[nz]}, stored column-major with column stride
// cs = col_stride(b) (b rounded up to a multiple of 4; rows b..cs-1 are zero)
// so every column starts on a 16-byte boundary: element (r, c) at
// vals[nz*b*cs + c*cs + r], in the storage precision `prec`.  Blocks of the
// tensor-core path (b = 16 or 64, tc_image = 1) have cs = b and are stored as
// the BF16 operand images the tensor cores read (tc_image_offset below).
inline int col_stride(int b) { return (b + 3) / 4 * 4; }
// Schedule of the cached tensor-core apply (tc_cached.cu) of one matrix: the
// processing order as 32-byte step records, the CTA ranges and the x loads,
// all device arrays owned by the DevMat that holds it.
struct TcSched {
  int G = 0;                // CTAs (two per SM): CTA c takes steps [seg[c], seg[c + 1])
  int S = 0;                // x slots per CTA
  int L = 0;                // strip width (element columns)
  int kmax = 0;             // most blocks in a row
  int rcap = 0;             // most right-hand sides per call
  int64_t nloads = 0;       // x_j loads per apply (all CTAs)
  void* rec = nullptr;      // nrows step records
  int* seg = nullptr;       // G + 1
  int* ld_elem = nullptr;   // nloads + 32
};
struct DevMat {
  int64_t nrows = 0, nnzb = 0;
  int b = 0, cs = 0, prec = P_FP64;
  int tc_image = 0;         // 1: blocks stored as tensor-core operand images (batched path)
  double scale = 1.0;       // stored value = scale * entry (a power of two; FP16 storage only)
  int* row_ptr = nullptr;   // nrows + 1
  int* col = nullptr;       // nnzb
  void* vals = nullptr;     // nnzb * b * b elements
  TcSched sched;            // tensor-core images, 2D b = 16: cached apply schedule (rec == null: none)
};

// Epilogue of a block-row apply, acc_i = sum_j M_ij x_j:
enum BsrMode {
  M_Y = 0,      // y_i = acc_i
  M_RES = 1,    // y_i = rhs_i - acc_i
  M_AXPY = 2,   // y_i = xin_i + s * acc_i   (xin may alias y)
  M_SCALE = 3   // y_i = s * acc_i
};

bool block_size_supported(int b);

// kernels enqueued by this library so far
unsigned long long launches();

// vector type: double when prec == P_FP64, float otherwise
cudaError_t bsr_apply(const DevMat& M, int mode, const void* x, const void* rhs, const void* xin,
                      void* y, double s, cudaStream_t st);
// Same on R right-hand sides (CUDA cores, column-major blocks): entry (element e,
// rhs r, mode c) of every vector lives at e*es + r*rs + c.  Each right-hand side
// is computed exactly as the single-RHS apply would compute it.
cudaError_t bsr_apply_strided(const DevMat& M, int mode, const void* x, const void* rhs, const void* xin,
                              void* y, double s, int R, int64_t es, int64_t rs, cudaStream_t st);

// Same on the `count` block rows listed in `rows` (device int32; e.g. one
// colour class of multi-coloured Gauss-Seidel); other rows of y are untouched.
cudaError_t bsr_apply_rows(const DevMat& M, const int* rows, int64_t count, int mode, const void* x, const void* rhs,
                           const void* xin, void* y, double s, int R, int64_t es, int64_t rs, cudaStream_t st);

// Batched apply on tensor cores (tc_apply.cu): BF16 row-major blocks, FP32 vectors.
struct BatchArgs {
  int64_t nrows;
  const int* row_ptr;
  const int* col;
  const void* vals;       // block operand images (BF16, or BF16 hi + lo for FP32 storage)
  const void* ximg;       // operand images of x, written by split_x_images for this R
  const float* x;
  const float* rhs;
  const float* xin;
  float* y;
  double s;
  int mode;
  int R;                  // right-hand sides, 1..128
  int64_t es, rs;         // element and right-hand-side strides of the vectors (floats)
  int* err;               // set to 1 if a bounded wait gave up (may be null)
  int ctas_per_sm = 0;    // resident CTAs per SM to launch (0: as many as fit); the
                          // result does not depend on it (a block row is one CTA's work)
};
bool tc_block_size_supported(int b);
// one bounded wait on an mbarrier that never completes; sets *err = 1 when it gives up
cudaError_t bounded_wait_probe(int* err, cudaStream_t st);
// most CTAs of the tensor-core kernel that fit on one SM for (b, prec, R)
int tc_max_ctas_per_sm(int b, int prec, int R);
// prec: P_BF16 (2 MMAs per K step) or P_FP32 (3 MMAs: A_hi x_hi + A_hi x_lo + A_lo x_hi).
// a.ximg must hold split_x_images(a.x) for the same R (a.x itself is not read).
cudaError_t bsr_apply_tc(const BatchArgs& a, int b, int prec, cudaStream_t st);

// Cached tensor-core apply (tc_cached.cu; 2D, b = 16, R <= 64, vectors
// [element][rhs][mode] with es = R b, rs = b): the products of bsr_apply_tc
// (plus x_lo A_lo) without x images; a.ximg and a.ctas_per_sm are not used.
// tc_sched_plan builds the host schedule for strip width L on G SMs (two
// CTAs each), or returns why it cannot; the caller uploads it into a TcSched.
struct TcSchedHost {
  int G = 0, S = 0, L = 0, kmax = 0, rcap = 0;
  int64_t nloads = 0;
  std::vector<uint8_t> rec;
  std::vector<int> seg, ld_elem;
};
std::string tc_sched_plan(int dim, int n, int64_t nrows, const int64_t* row_ptr, const int32_t* col, int rcap,
                          int prec, int G, int L, TcSchedHost* out);
cudaError_t bsr_apply_tc_cached(const BatchArgs& a, const TcSched& s, int prec, cudaStream_t st);

// Operand images of a batched vector x ([element][rhs][mode], R right-hand
// sides, b = 16 or 64) for the tensor-core apply: per element j the image of
// hi = bf16(x_j^T) and then that of lo = bf16(x_j^T - hi), each R_8 x b BF16
// (R_8 = R rounded up to 8; rows R..R_8-1 zero) in the K-major core-matrix
// layout of tc_image_offset (rows = right-hand sides, K = modes).
size_t x_image_bytes(int64_t N, int R, int b);
cudaError_t split_x_images(const float* x, int64_t N, int R, int b, void* ximg, cudaStream_t st);

// vals[nz] = scale * pool[ids[nz]] converted to `prec`, stored column-major
// with column stride cs (tc_image = 0; padding rows written as zero) or as
// tensor-core operand images (tc_image = 1, cs = b, prec P_BF16 or P_FP32);
// pool blocks are row-major FP64
cudaError_t expand_blocks(int64_t nnzb, int b, int cs, const uint32_t* ids, const double* pool, void* vals,
                          int prec, int tc_image, double scale, cudaStream_t st);

// Tensor-core operand image of a b x b block (b = 16 or 64): entry (r, c) --
// output mode r, input mode c -- in the K-major, no-swizzle core-matrix
// layout (8 rows x 16 bytes per core matrix, b/8 core matrices along K),
// BF16.  P_BF16 storage holds one image (2 b^2 bytes); P_FP32 storage holds
// the image of hi = bf16(a) followed by that of lo = bf16(a - hi), a the FP32
// entry (4 b^2 bytes, the same as FP32).  Byte offset within one image:
__host__ __device__ inline uint32_t tc_image_offset(int b, int r, int c) {
  return uint32_t(((r >> 3) * (b >> 3) + (c >> 3)) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// P: device array of the 1D child-injection matrices P[s][i][j] (2*q*q doubles,
// q = p + 1 <= 8).  Level vectors are double (vprec 0) or float (vprec 1).
// Vectors of R right-hand sides use the layout [element][rhs][mode] (R = 1:
// plain [element][mode]).
// rc_C = sum_children P_c^T rf_c
cudaError_t restrict_apply(int d, int q, int n_fine, const double* P, const void* rf, void* rc,
                           int vprec, int R, cudaStream_t st);
// xf_c += P_c xc_C
cudaError_t prolong_apply(int d, int q, int n_fine, const double* P, const void* xc, void* xf,
                          int vprec, int R, cudaStream_t st);

// y = Pinv v, Pinv dense n x n FP64 row-major (n = N*b), per right-hand side
cudaError_t dense_gemv(int64_t n, int b, const double* Pinv, const void* v, void* y, int vprec, int R,
                       cudaStream_t st);

// layout changes between R stacked vectors [rhs][element][mode] and [element][rhs][mode]
cudaError_t stack_to_batch(int64_t N, int R, int b, const double* src, double* dst, cudaStream_t st);
cudaError_t batch_to_stack(int64_t N, int R, int b, const double* src, double* dst, cudaStream_t st);

// conversions and BLAS-1 (FP64 unless stated)
cudaError_t cast_d2f(int64_t n, const double* a, float* b, cudaStream_t st);
cudaError_t cast_f2d(int64_t n, const float* a, double* b, cudaStream_t st);

// deterministic dot: out[0] = sum_i a_i b_i (two-stage, fixed order).  partials
// holds at least kDotBlocks doubles.
constexpr int kDotBlocks = 1024;
cudaError_t dot(int64_t n, const double* a, const double* b, double* partials, double* out,
                cudaStream_t st);
// out[0] = sum_e v[e*stride]  (sum of mode-0 coefficients)
cudaError_t strided_sum(int64_t count, int64_t stride, const double* v, double* partials,
                        double* out, cudaStream_t st);
// v[e*stride] -= (*sum) / count
cudaError_t strided_sub_mean(int64_t count, int64_t stride, double* v, const double* sum,
                             cudaStream_t st);

// GMRES steps: y += sgn * coef[0] * x (coef on the device); y = x / s;
// x += sum_{i<k} y[i] * Q[i*ldq ...] (y on the device, fixed summation order)
cudaError_t axpy_dev(int64_t n, const double* coef, double sgn, const double* x, double* y, cudaStream_t st);
cudaError_t vec_div(int64_t n, double s, const double* x, double* y, cudaStream_t st);
cudaError_t vec_combine(int64_t n, int k, const double* Q, int64_t ldq, const double* y, double* x,
                        cudaStream_t st);

// per right-hand-side dots on [element][rhs][mode] vectors: out[r] = sum u_r v_r
// (v may be null: sum of squares of u).  partials: kBatchDotBlocks * R doubles.
constexpr int kBatchDotBlocks = 256;
cudaError_t dot_batched(int64_t N, int R, int b, const double* u, const double* v, double* partials,
                        double* out, cudaStream_t st);

// CG scalar slots
enum CgSlot { S_RZ = 0, S_PQ = 1, S_RR = 2, S_RZNEW = 3, S_RZOLD = 4, S_ALPHA = 5, S_BETA = 6,
              S_BB = 7, S_TMP = 8, S_TOL2 = 9, kCgSlots = 16 };
cudaError_t cg_alpha(double* scal, cudaStream_t st);                    // alpha = rz / pq
cudaError_t cg_update_xr(int64_t n, double* x, double* r, const double* p, const double* q,
                         const double* scal, cudaStream_t st);          // x += a p ; r -= a q
cudaError_t cg_beta(double* scal, int flexible, cudaStream_t st);       // beta, rz <- rz_new
cudaError_t cg_update_p(int64_t n, double* p, const double* z, const double* scal,
                        cudaStream_t st);                              // p = z + beta p
// Batched CG: scalars scal[slot * R + r]; active[r] = 0 freezes right-hand side r
cudaError_t cg_alpha_b(int R, double* scal, const int* active, cudaStream_t st);
cudaError_t cg_update_xr_b(int64_t N, int R, int b, double* x, double* r, const double* p, const double* q,
                           const double* scal, cudaStream_t st);
cudaError_t cg_beta_b(int R, double* scal, const int* active, int flexible, cudaStream_t st);
cudaError_t cg_update_p_b(int64_t N, int R, int b, double* p, const double* z, const double* scal,
                          cudaStream_t st);
// Device-side stopping test after the residual norms: for each active r,
// it[r] += 1 and hist[it[r] * R + r] = ||r||^2 (while it[r] < hist_cap; hist may
// be null), then r stops when scal[S_RR] <= scal[S_TOL2] * scal[S_BB]
// (flag[r] = 0) or when the norm is not finite (flag[r] = 1).
cudaError_t cg_check_b(int R, const double* scal, int* active, int* it, int* flag, double* hist, int hist_cap,
                       cudaStream_t st);
// Double-FP32 operator apply (df_apply.cu): `pairs` holds A's FP64 entries as
// (hi, lo) FP32 pairs in the layout of M (column-major blocks, b = 16 or 64);
// x, rhs, y are FP64 [element][rhs][mode] with R <= 64 right-hand sides.
// mode: M_Y or M_RES.  Accuracy ~2^-44 of sum |a x|.
cudaError_t split_to_float_pairs(int64_t n, const double* src, void* dst, cudaStream_t st);
cudaError_t bsr_apply_df(const DevMat& M, const void* pairs, int mode, const double* x, const double* rhs, double* y,
                         int R, cudaStream_t st);

// single right-hand side version of the double-FP32 apply (b = 16, 64)
cudaError_t bsr_apply_df1(const DevMat& M, const void* pairs, int mode, const double* x, const double* rhs,
                          double* y, cudaStream_t st);
// FP64 apply with the same block reuse over R <= 64 right-hand sides (b = 16, 64)
cudaError_t bsr_apply_multi64(const DevMat& M, int mode, const double* x, const double* rhs, double* y, int R,
                              cudaStream_t st);

// Batched FP64 least squares of the SAI setup on the device (sai_ls.cu): fills
// X and ok of every problem (host.h LsProblem); "" or an error message.
struct LsProblem;
std::string sai_ls_device(std::vector<LsProblem>& batch, cudaStream_t st);

// Grouped solve (group.cu): many independent single-right-hand-side scalar
// problems, of any mix of classes, in one launch.  Each problem is a whole
// preconditioned CG solve (Sec. 2.2; the V-cycle of Algorithm 1 as the
// preconditioner, FP64 outer operator) run by one thread-block cluster of
// `cluster` CTAs, which synchronise with cluster barriers between steps; no
// host round trip inside a solve.  Descriptors live in device memory.
constexpr int kGroupMaxLevels = 12;
enum { G_SAI = 0, G_JACOBI = 1, G_GS = 2 };
struct GroupMat {
  const int* row_ptr;
  const int* col;
  const void* vals;     // column-major blocks, column stride cs, storage precision prec
  int prec;
  int cs;
  double inv_scale;     // 1 / storage scale
};
struct GroupLevel {
  int64_t N;            // elements
  int n, b, ncolours, pad;
  GroupMat A, S, ST;    // operator; smoother (B or D^-1); B^T (SAI)
  const int* crows;     // Gauss-Seidel: element rows grouped by colour
  const int* cptr;      // device, ncolours + 1
  int64_t voff;         // rhs, x, r of this level at voff, voff + N b, voff + 2 N b (vector entries)
};
struct GroupProblem {
  int dim, q, nl, smoother, pre_bt, post_bt, nu1, nu2;
  int vprec;            // level vectors: 0 double (FP64 storage), 1 float
  int flexible;         // flexible CG (reduced-precision V-cycle)
  int max_iter, pad;
  double omega;
  const double* P;      // 2 q^2 one-dimensional injection matrices
  const double* pinv;   // bottom pseudo-inverse, nbot x nbot row-major
  int64_t nbot;
  GroupMat A0;          // FP64 finest operator of the outer CG
  int64_t n0;           // unknowns N_0 b
  GroupLevel lv[kGroupMaxLevels];
};
struct GroupOut {
  int iters;
  int status;           // 0 converged, 1 max_iter reached, 2 non-finite residual, 3 non-finite rhs
  double relres;        // true ||b - A x|| / ||b||
};
struct GroupItem {
  int prob, pad;
  const double* b;      // device FP64 right-hand side, [element][mode]
  double* x;            // device FP64 solution
  double tol;
  void* lvec;           // level vectors of this item (double or float)
  double* cg;           // r, z, p, q: 4 n0 doubles
  GroupOut* out;
};
// items[0 .. count) all run with clusters of `cluster` CTAs (1, 2, 4 or 8)
cudaError_t group_solve(const GroupProblem* probs, const GroupItem* items, int count, int cluster, cudaStream_t st);

// launch-count bookkeeping for kernels defined in other translation units
cudaError_t launched(int count = 1);

}  // namespace ldgmg
