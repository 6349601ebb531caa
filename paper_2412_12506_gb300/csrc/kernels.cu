// Device kernels of the LDG multigrid hot path, written for sm_103a (GB300).
//
// Block-row apply (Sec. 2.3: sum_j A_ij x_j over the element-block pattern;
// the same kernel applies A, B, B^T and the Jacobi inverse blocks): the
// matrix is streamed exactly once from HBM.  A "team" of threads owns one
// block row (a warp for b <= 32, the whole 256-thread CTA for b > 32).  Each
// team splits the block's columns into G groups; inside a group, LPC threads
// cover the b rows of one column with 16-byte vector loads, so every load
// step of the team reads G consecutive columns = one contiguous run of the
// column-major block.  The neighbour vector x_j is staged in shared memory
// and broadcast.  Partial sums of the G groups are reduced in shared memory
// in a fixed order (results are deterministic), then a fused epilogue writes
// y = acc, rhs - acc (residual), xin + s*acc (smoother update) or s*acc.
#include "kernels.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

namespace ldgmg {

typedef __nv_bfloat16 bf16;
typedef __half f16;

// number of kernels this library has enqueued (all streams, all devices)
static std::atomic<unsigned long long> g_launches{0};
unsigned long long launches() { return g_launches.load(); }
cudaError_t launched(int count) {
  g_launches.fetch_add(count);
  return cudaGetLastError();
}

__device__ __forceinline__ float to_f(bf16 v) { return __bfloat162float(v); }
template <class T> __device__ __forceinline__ T from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return float(v); }
template <> __device__ __forceinline__ bf16 from_d<bf16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ f16 from_d<f16>(double v) { return __double2half(v); }

template <class TACC, class TA> __device__ __forceinline__ TACC cvt(TA v) { return TACC(v); }
template <> __device__ __forceinline__ float cvt<float, bf16>(bf16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double cvt<double, bf16>(bf16 v) {
  return double(__bfloat162float(v));
}
template <> __device__ __forceinline__ float cvt<float, f16>(f16 v) { return __half2float(v); }

template <class T, int N> struct alignas(sizeof(T) * N) VecT { T v[N]; };

// largest power-of-two element count <= 16 bytes that divides B
template <class TA> constexpr int vec_for(int B) {
  int v = 16 / int(sizeof(TA));
  while (v > 1 && (B % v) != 0) v /= 2;
  return v;
}

template <class TA> struct AccOf { typedef float type; };
template <> struct AccOf<double> { typedef double type; };

template <class TA, class TV> struct BsrArgs {
  int64_t nrows;
  const int* __restrict__ row_ptr;
  const int* __restrict__ col;
  const TA* __restrict__ vals;
  const TV* __restrict__ x;
  const TV* rhs;
  const TV* xin;
  TV* y;
  double s;
  int mode;
  int64_t es, rs;   // vector entry (element e, rhs r, mode c) at e*es + r*rs + c; rhs = blockIdx.y
  int R;            // right-hand sides (grid y dimension)
  double inv_scale; // 1 / storage scale of the matrix (exact power of two)
};

template <int TEAM> __device__ __forceinline__ void team_sync() {
  if (TEAM == 32) __syncwarp(); else __syncthreads();
}

template <int B, class TA, class TV>
__global__ void __launch_bounds__(256) bsr_kernel(BsrArgs<TA, TV> a) {
  typedef typename AccOf<TA>::type TACC;
  constexpr int VEC = vec_for<TA>(B);
  constexpr int TEAM = (B > 32) ? 256 : 32;
  constexpr int LPC = B / VEC;             // threads per column
  constexpr int G = TEAM / LPC;            // column groups per team
  constexpr int TEAMS = 256 / TEAM;        // block rows per CTA
  constexpr int STEPS = (B + G - 1) / G;   // load steps per block
  static_assert(G >= 1, "team too small");
  constexpr int KMAX = 16;                 // blocks whose x_j are staged at once
  __shared__ TACC xs[TEAMS][KMAX][B];
  __shared__ TACC red[TEAMS][G][B];

  const int team = threadIdx.x / TEAM, lt = threadIdx.x % TEAM;
  const int g = lt / LPC, rl = lt % LPC;
  const bool active = g < G;
  const int64_t row = int64_t(blockIdx.x) * TEAMS + team;
  const int64_t roff = int64_t(blockIdx.y) * a.rs;
  if (TEAM == 32 && row >= a.nrows) return;   // whole warp leaves together
  TACC acc[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc[v] = TACC(0);

  if (row < a.nrows) {
    const int z0 = a.row_ptr[row], z1 = a.row_ptr[row + 1];
    // stage the neighbour vectors of up to KMAX blocks, then stream those
    // blocks with no barrier in between (many loads in flight per thread)
    for (int zb = z0; zb < z1; zb += KMAX) {
      const int nb = min(KMAX, z1 - zb);
      team_sync<TEAM>();
      for (int t = lt; t < nb * B; t += TEAM) {
        const int kk = t / B, c = t % B;
        xs[team][kk][c] = TACC(a.x[int64_t(a.col[zb + kk]) * a.es + roff + c]);
      }
      team_sync<TEAM>();
      if (active) {
        for (int kk = 0; kk < nb; ++kk) {
          const TA* blk = a.vals + int64_t(zb + kk) * (B * B) + rl * VEC;
#pragma unroll 4
          for (int st = 0; st < STEPS; ++st) {
            const int c = st * G + g;
            if (c < B) {
              const VecT<TA, VEC> w = *reinterpret_cast<const VecT<TA, VEC>*>(blk + c * B);
              const TACC xc = xs[team][kk][c];
#pragma unroll
              for (int v = 0; v < VEC; ++v) acc[v] += cvt<TACC>(w.v[v]) * xc;
            }
          }
        }
      }
    }
  }
  if (active) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) red[team][g][rl * VEC + v] = acc[v];
  }
  team_sync<TEAM>();
  if (row < a.nrows && lt < B) {
    TACC sum = TACC(0);
#pragma unroll
    for (int gg = 0; gg < G; ++gg) sum += red[team][gg][lt];
    sum *= TACC(a.inv_scale);
    const int64_t o = row * a.es + roff + lt;
    switch (a.mode) {
      case M_Y: a.y[o] = TV(sum); break;
      case M_RES: a.y[o] = TV(TACC(a.rhs[o]) - sum); break;
      case M_AXPY: a.y[o] = TV(TACC(a.xin[o]) + TACC(a.s) * sum); break;
      default: a.y[o] = TV(TACC(a.s) * sum); break;
    }
  }
}

bool block_size_supported(int b) {
  switch (b) {
    case 4: case 8: case 9: case 16: case 25: case 27: case 36: case 64: return true;
    default: return false;
  }
}

template <int B, class TA, class TV>
static cudaError_t launch_bsr_b(const DevMat& M, const BsrArgs<TA, TV>& a, cudaStream_t st) {
  constexpr int TEAMS = (B > 32) ? 1 : 8;
  if (M.nrows == 0) return cudaSuccess;
  const int64_t grid = (M.nrows + TEAMS - 1) / TEAMS;
  bsr_kernel<B, TA, TV><<<dim3(unsigned(grid), unsigned(a.R)), 256, 0, st>>>(a);
  return launched();
}

template <class TA, class TV>
static cudaError_t launch_bsr_t(const DevMat& M, int mode, const void* x, const void* rhs,
                                const void* xin, void* y, double s, int R, int64_t es, int64_t rs,
                                cudaStream_t st) {
  BsrArgs<TA, TV> a;
  a.nrows = M.nrows;
  a.row_ptr = M.row_ptr;
  a.col = M.col;
  a.vals = static_cast<const TA*>(M.vals);
  a.x = static_cast<const TV*>(x);
  a.rhs = static_cast<const TV*>(rhs);
  a.xin = static_cast<const TV*>(xin);
  a.y = static_cast<TV*>(y);
  a.s = s;
  a.mode = mode;
  a.es = es;
  a.rs = rs;
  a.R = R;
  a.inv_scale = 1.0 / M.scale;
  switch (M.b) {
    case 4: return launch_bsr_b<4>(M, a, st);
    case 8: return launch_bsr_b<8>(M, a, st);
    case 9: return launch_bsr_b<9>(M, a, st);
    case 16: return launch_bsr_b<16>(M, a, st);
    case 25: return launch_bsr_b<25>(M, a, st);
    case 27: return launch_bsr_b<27>(M, a, st);
    case 36: return launch_bsr_b<36>(M, a, st);
    case 64: return launch_bsr_b<64>(M, a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t bsr_apply_strided(const DevMat& M, int mode, const void* x, const void* rhs, const void* xin,
                              void* y, double s, int R, int64_t es, int64_t rs, cudaStream_t st) {
  if (M.row_major || R < 1) return cudaErrorInvalidValue;
  switch (M.prec) {
    case P_FP64: return launch_bsr_t<double, double>(M, mode, x, rhs, xin, y, s, R, es, rs, st);
    case P_FP32: return launch_bsr_t<float, float>(M, mode, x, rhs, xin, y, s, R, es, rs, st);
    case P_BF16: return launch_bsr_t<bf16, float>(M, mode, x, rhs, xin, y, s, R, es, rs, st);
    case P_FP16: return launch_bsr_t<f16, float>(M, mode, x, rhs, xin, y, s, R, es, rs, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t bsr_apply(const DevMat& M, int mode, const void* x, const void* rhs, const void* xin,
                      void* y, double s, cudaStream_t st) {
  return bsr_apply_strided(M, mode, x, rhs, xin, y, s, 1, M.b, 0, st);
}

// --------------------------------------------------------------------------
// pool expansion (setup): vals[nz] = transpose(pool[ids[nz]]) in precision T
// --------------------------------------------------------------------------

template <class T>
__global__ void expand_kernel(int64_t total, int b, const uint32_t* __restrict__ ids,
                              const double* __restrict__ pool, T* __restrict__ vals, int row_major, double scale) {
  const int64_t bb = int64_t(b) * b;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t nz = t / bb, e = t % bb;
    int r, c;
    if (row_major) { r = int(e / b); c = int(e % b); }
    else { c = int(e / b); r = int(e % b); }
    vals[t] = from_d<T>(scale * pool[int64_t(ids[nz]) * bb + int64_t(r) * b + c]);
  }
}

cudaError_t expand_blocks(int64_t nnzb, int b, const uint32_t* ids, const double* pool, void* vals,
                          int prec, int row_major, double scale, cudaStream_t st) {
  const int64_t total = nnzb * b * b;
  if (total == 0) return cudaSuccess;
  const int grid = int(std::min<int64_t>((total + 255) / 256, 152 * 64));
  switch (prec) {
    case P_FP64: expand_kernel<double><<<grid, 256, 0, st>>>(total, b, ids, pool, (double*)vals, row_major, scale); break;
    case P_FP32: expand_kernel<float><<<grid, 256, 0, st>>>(total, b, ids, pool, (float*)vals, row_major, scale); break;
    case P_BF16: expand_kernel<bf16><<<grid, 256, 0, st>>>(total, b, ids, pool, (bf16*)vals, row_major, scale); break;
    case P_FP16: expand_kernel<f16><<<grid, 256, 0, st>>>(total, b, ids, pool, (f16*)vals, row_major, scale); break;
    default: return cudaErrorInvalidValue;
  }
  return launched();
}

// --------------------------------------------------------------------------
// Restriction and prolongation (Algorithm 1, lines 5 and 7).  The injection
// block of child s is the Kronecker product of 1D matrices P[s_a] (Sec. 2.2,
// polynomial injection); it is applied by sum factorisation, one axis at a
// time, in shared memory.  One CTA per coarse element.
// --------------------------------------------------------------------------

// One CTA per coarse element handles all R right-hand sides: the R*b entries
// of an element are contiguous in the [element][rhs][mode] layout.  Each
// thread owns outputs o = rr*b + t (right-hand side rr, mode t); the 1D
// transforms along the d axes run in shared memory with a barrier per axis.
// The arithmetic of every output is independent of R.
constexpr int kXferThreads = 256;
constexpr int kXferMaxOut = 16;        // outputs per thread: R*b <= 4096

__device__ __forceinline__ void load_P(double (*Ps)[8][8], const double* P, int q) {
  for (int i = threadIdx.x; i < 2 * q * q; i += blockDim.x) {
    const int s = i / (q * q), r = (i / q) % q, c = i % q;
    Ps[s][r][c] = P[i];
  }
}

// in -> out along all d axes for child offsets sidx; TRANSPOSE applies P_s^T.
// Returns the buffer that holds the result.
template <bool TRANSPOSE>
__device__ __forceinline__ double* child_transform(const double (*Ps)[8][8], double* in, double* out, int d, int q,
                                                   int b, int nout, int sidx) {
  int stride = 1;
  for (int a = 0; a < d; ++a) {
    const int s = (sidx >> a) & 1;
    for (int o = threadIdx.x; o < nout; o += kXferThreads) {
      const int rr = o / b, t = o % b;
      const int ka = (t / stride) % q;
      const int base = rr * b + t - ka * stride;
      double v = 0.0;
      for (int k = 0; k < q; ++k) v += (TRANSPOSE ? Ps[s][k][ka] : Ps[s][ka][k]) * in[base + k * stride];
      out[o] = v;
    }
    __syncthreads();
    double* tmp = in;
    in = out;
    out = tmp;
    stride *= q;
  }
  return in;
}

template <class TV>
__global__ void __launch_bounds__(kXferThreads) restrict_kernel(int d, int q, int nf, const double* __restrict__ P,
                                                                const TV* __restrict__ rf, TV* __restrict__ rc, int R) {
  extern __shared__ double xbuf[];
  __shared__ double Ps[2][8][8];
  load_P(Ps, P, q);
  const int b = (d == 2) ? q * q : q * q * q;
  const int nout = R * b;
  double* buf0 = xbuf;
  double* buf1 = xbuf + nout;
  const int64_t nc = nf / 2;
  const int64_t C = blockIdx.x;
  int cc[3] = {int(C % nc), int((C / nc) % nc), int(C / (nc * nc))};
  double acc[kXferMaxOut];
#pragma unroll
  for (int k = 0; k < kXferMaxOut; ++k) acc[k] = 0.0;
  for (int s = 0; s < (1 << d); ++s) {
    int64_t f = 0;
    for (int a = d - 1; a >= 0; --a) f = f * nf + (2 * cc[a] + ((s >> a) & 1));
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += kXferThreads) buf0[o] = double(rf[f * nout + o]);
    __syncthreads();
    const double* res = child_transform<true>(Ps, buf0, buf1, d, q, b, nout, s);
#pragma unroll
    for (int k = 0; k < kXferMaxOut; ++k) {
      const int o = threadIdx.x + k * kXferThreads;
      if (o < nout) acc[k] += res[o];
    }
  }
#pragma unroll
  for (int k = 0; k < kXferMaxOut; ++k) {
    const int o = threadIdx.x + k * kXferThreads;
    if (o < nout) rc[C * nout + o] = TV(acc[k]);
  }
}

template <class TV>
__global__ void __launch_bounds__(kXferThreads) prolong_kernel(int d, int q, int nf, const double* __restrict__ P,
                                                               const TV* __restrict__ xc, TV* __restrict__ xf, int R) {
  extern __shared__ double xbuf[];
  __shared__ double Ps[2][8][8];
  load_P(Ps, P, q);
  const int b = (d == 2) ? q * q : q * q * q;
  const int nout = R * b;
  double* buf0 = xbuf;
  double* buf1 = xbuf + nout;
  const int64_t nc = nf / 2;
  const int64_t C = blockIdx.x;
  int cc[3] = {int(C % nc), int((C / nc) % nc), int(C / (nc * nc))};
  for (int s = 0; s < (1 << d); ++s) {
    int64_t f = 0;
    for (int a = d - 1; a >= 0; --a) f = f * nf + (2 * cc[a] + ((s >> a) & 1));
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += kXferThreads) buf0[o] = double(xc[C * nout + o]);
    __syncthreads();
    const double* res = child_transform<false>(Ps, buf0, buf1, d, q, b, nout, s);
    for (int o = threadIdx.x; o < nout; o += kXferThreads) xf[f * nout + o] = TV(double(xf[f * nout + o]) + res[o]);
  }
}

static int64_t coarse_count(int d, int nf) {
  int64_t nc = nf / 2, r = 1;
  for (int a = 0; a < d; ++a) r *= nc;
  return r;
}

static cudaError_t xfer_config(int smem) {
  static int configured = 0;
  if (smem > 48 * 1024 && configured < smem) {
    cudaError_t e = cudaFuncSetAttribute(restrict_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(restrict_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(prolong_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(prolong_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  return cudaSuccess;
}

cudaError_t restrict_apply(int d, int q, int n_fine, const double* P, const void* rf, void* rc,
                           int vprec, int R, cudaStream_t st) {
  const int b = (d == 2) ? q * q : q * q * q;
  if (R * b > kXferThreads * kXferMaxOut) return cudaErrorInvalidValue;
  const int smem = 2 * R * b * int(sizeof(double));
  cudaError_t e = xfer_config(smem);
  if (e != cudaSuccess) return e;
  const int64_t Nc = coarse_count(d, n_fine);
  if (vprec == 0) restrict_kernel<double><<<unsigned(Nc), kXferThreads, smem, st>>>(d, q, n_fine, P, (const double*)rf, (double*)rc, R);
  else restrict_kernel<float><<<unsigned(Nc), kXferThreads, smem, st>>>(d, q, n_fine, P, (const float*)rf, (float*)rc, R);
  return launched();
}

cudaError_t prolong_apply(int d, int q, int n_fine, const double* P, const void* xc, void* xf,
                          int vprec, int R, cudaStream_t st) {
  const int b = (d == 2) ? q * q : q * q * q;
  if (R * b > kXferThreads * kXferMaxOut) return cudaErrorInvalidValue;
  const int smem = 2 * R * b * int(sizeof(double));
  cudaError_t e = xfer_config(smem);
  if (e != cudaSuccess) return e;
  const int64_t Nc = coarse_count(d, n_fine);
  if (vprec == 0) prolong_kernel<double><<<unsigned(Nc), kXferThreads, smem, st>>>(d, q, n_fine, P, (const double*)xc, (double*)xf, R);
  else prolong_kernel<float><<<unsigned(Nc), kXferThreads, smem, st>>>(d, q, n_fine, P, (const float*)xc, (float*)xf, R);
  return launched();
}

// --------------------------------------------------------------------------
// bottom solve: dense FP64 pseudo-inverse times vector, one warp per row
// --------------------------------------------------------------------------

// dof i = e*b + c of right-hand side r lives at (e*R + r)*b + c
template <class TV>
__global__ void gemv_kernel(int64_t n, int b, const double* __restrict__ P, const TV* __restrict__ v,
                            TV* __restrict__ y) {
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32;
  const int R = gridDim.y, rr = blockIdx.y;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  const double* pr = P + row * n;
  for (int64_t j = lane; j < n; j += 32) s += pr[j] * double(v[((j / b) * R + rr) * b + j % b]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[((row / b) * R + rr) * b + row % b] = TV(s);
}

cudaError_t dense_gemv(int64_t n, int b, const double* Pinv, const void* v, void* y, int vprec, int R,
                       cudaStream_t st) {
  const dim3 grid{unsigned((n * 32 + 255) / 256), unsigned(R), 1u};
  if (vprec == 0) gemv_kernel<double><<<grid, 256, 0, st>>>(n, b, Pinv, (const double*)v, (double*)y);
  else gemv_kernel<float><<<grid, 256, 0, st>>>(n, b, Pinv, (const float*)v, (float*)y);
  return launched();
}

// --------------------------------------------------------------------------
// BLAS-1 and CG helpers (FP64).  Reductions are two-stage with a fixed grid
// and a fixed combination order, so results are bitwise reproducible.
// --------------------------------------------------------------------------

__global__ void cast_d2f_kernel(int64_t n, const double* a, float* b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = float(a[i]);
}
__global__ void cast_f2d_kernel(int64_t n, const float* a, double* b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = double(a[i]);
}

static int grid_for(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16))); }

cudaError_t cast_d2f(int64_t n, const double* a, float* b, cudaStream_t st) {
  cast_d2f_kernel<<<grid_for(n), 256, 0, st>>>(n, a, b);
  return launched();
}
cudaError_t cast_f2d(int64_t n, const float* a, double* b, cudaStream_t st) {
  cast_f2d_kernel<<<grid_for(n), 256, 0, st>>>(n, a, b);
  return launched();
}

__device__ __forceinline__ double block_reduce(double v) {
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < int(blockDim.x / 32)) ? ws[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

__global__ void dot_partial(int64_t n, int64_t stride_a, const double* a, const double* b,
                            double* partials) {
  double s = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    s += a[i * stride_a] * (b ? b[i] : 1.0);
  s = block_reduce(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void sum_final(int count, const double* partials, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += partials[i];
  s = block_reduce(s);
  if (threadIdx.x == 0) out[0] = s;
}

cudaError_t dot(int64_t n, const double* a, const double* b, double* partials, double* out,
                cudaStream_t st) {
  dot_partial<<<kDotBlocks, 256, 0, st>>>(n, 1, a, b, partials);
  sum_final<<<1, 1024, 0, st>>>(kDotBlocks, partials, out);
  return launched(2);
}

cudaError_t strided_sum(int64_t count, int64_t stride, const double* v, double* partials,
                        double* out, cudaStream_t st) {
  dot_partial<<<kDotBlocks, 256, 0, st>>>(count, stride, v, nullptr, partials);
  sum_final<<<1, 1024, 0, st>>>(kDotBlocks, partials, out);
  return launched(2);
}

__global__ void sub_mean_kernel(int64_t count, int64_t stride, double* v, const double* sum) {
  const double m = sum[0] / double(count);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    v[i * stride] -= m;
}

cudaError_t strided_sub_mean(int64_t count, int64_t stride, double* v, const double* sum,
                             cudaStream_t st) {
  sub_mean_kernel<<<grid_for(count), 256, 0, st>>>(count, stride, v, sum);
  return launched();
}

__global__ void cg_alpha_kernel(double* s) { s[S_ALPHA] = s[S_RZ] / s[S_PQ]; }
__global__ void cg_beta_kernel(double* s, int flexible) {
  const double num = flexible ? (s[S_RZNEW] - s[S_RZOLD]) : s[S_RZNEW];
  s[S_BETA] = num / s[S_RZ];
  s[S_RZ] = s[S_RZNEW];
}
__global__ void cg_update_xr_kernel(int64_t n, double* x, double* r, const double* p, const double* q,
                                    const double* s) {
  const double al = s[S_ALPHA];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    x[i] += al * p[i];
    r[i] -= al * q[i];
  }
}
__global__ void cg_update_p_kernel(int64_t n, double* p, const double* z, const double* s) {
  const double be = s[S_BETA];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = z[i] + be * p[i];
}

cudaError_t cg_alpha(double* scal, cudaStream_t st) {
  cg_alpha_kernel<<<1, 1, 0, st>>>(scal);
  return launched();
}
cudaError_t cg_beta(double* scal, int flexible, cudaStream_t st) {
  cg_beta_kernel<<<1, 1, 0, st>>>(scal, flexible);
  return launched();
}
cudaError_t cg_update_xr(int64_t n, double* x, double* r, const double* p, const double* q,
                         const double* scal, cudaStream_t st) {
  cg_update_xr_kernel<<<grid_for(n), 256, 0, st>>>(n, x, r, p, q, scal);
  return launched();
}
cudaError_t cg_update_p(int64_t n, double* p, const double* z, const double* scal, cudaStream_t st) {
  cg_update_p_kernel<<<grid_for(n), 256, 0, st>>>(n, p, z, scal);
  return launched();
}

// --------------------------------------------------------------------------
// batched right-hand sides: layout changes, per-RHS dots and CG updates
// --------------------------------------------------------------------------

__global__ void relayout_kernel(int64_t N, int R, int b, const double* __restrict__ src,
                                double* __restrict__ dst, int to_batch) {
  const int64_t total = N * R * b;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    // t indexes the batched layout [e][r][c]
    const int64_t e = t / (int64_t(R) * b), r = (t / b) % R, c = t % b;
    const int64_t stacked = (r * N + e) * b + c;
    if (to_batch) dst[t] = src[stacked];
    else dst[stacked] = src[t];
  }
}

cudaError_t stack_to_batch(int64_t N, int R, int b, const double* src, double* dst, cudaStream_t st) {
  relayout_kernel<<<grid_for(N * R * b), 256, 0, st>>>(N, R, b, src, dst, 1);
  return launched();
}
cudaError_t batch_to_stack(int64_t N, int R, int b, const double* src, double* dst, cudaStream_t st) {
  relayout_kernel<<<grid_for(N * R * b), 256, 0, st>>>(N, R, b, src, dst, 0);
  return launched();
}

// block (p, r) sums entries of right-hand side r over a fixed slice of the element range
__global__ void dot_batched_partial(int64_t N, int b, const double* __restrict__ u, const double* __restrict__ v,
                                    double* __restrict__ partials) {
  const int R = gridDim.y, rr = blockIdx.y;
  const int64_t n = N * b;
  double s = 0.0;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t o = ((t / b) * R + rr) * b + t % b;
    const double a = u[o];
    s += a * (v ? v[o] : a);
  }
  s = block_reduce(s);
  if (threadIdx.x == 0) partials[int64_t(rr) * gridDim.x + blockIdx.x] = s;
}

__global__ void dot_batched_final(int P, const double* __restrict__ partials, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < P; i += blockDim.x) s += partials[int64_t(blockIdx.x) * P + i];
  s = block_reduce(s);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

cudaError_t dot_batched(int64_t N, int R, int b, const double* u, const double* v, double* partials,
                        double* out, cudaStream_t st) {
  dot_batched_partial<<<dim3(kBatchDotBlocks, unsigned(R)), 256, 0, st>>>(N, b, u, v, partials);
  dot_batched_final<<<unsigned(R), 256, 0, st>>>(kBatchDotBlocks, partials, out);
  return launched(2);
}

__global__ void cg_alpha_b_kernel(int R, double* s, const int* active) {
  const int r = threadIdx.x + blockIdx.x * blockDim.x;
  if (r < R) s[S_ALPHA * R + r] = active[r] ? s[S_RZ * R + r] / s[S_PQ * R + r] : 0.0;
}
__global__ void cg_beta_b_kernel(int R, double* s, const int* active, int flexible) {
  const int r = threadIdx.x + blockIdx.x * blockDim.x;
  if (r >= R) return;
  const double num = flexible ? (s[S_RZNEW * R + r] - s[S_RZOLD * R + r]) : s[S_RZNEW * R + r];
  s[S_BETA * R + r] = active[r] ? num / s[S_RZ * R + r] : 0.0;
  if (active[r]) s[S_RZ * R + r] = s[S_RZNEW * R + r];
}
__global__ void cg_update_xr_b_kernel(int64_t n, int R, int b, double* x, double* r, const double* p,
                                      const double* q, const double* s) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double al = s[S_ALPHA * R + (i / b) % R];
    x[i] += al * p[i];
    r[i] -= al * q[i];
  }
}
__global__ void cg_update_p_b_kernel(int64_t n, int R, int b, double* p, const double* z, const double* s) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = z[i] + s[S_BETA * R + (i / b) % R] * p[i];
}

cudaError_t cg_alpha_b(int R, double* scal, const int* active, cudaStream_t st) {
  cg_alpha_b_kernel<<<(R + 127) / 128, 128, 0, st>>>(R, scal, active);
  return launched();
}
cudaError_t cg_beta_b(int R, double* scal, const int* active, int flexible, cudaStream_t st) {
  cg_beta_b_kernel<<<(R + 127) / 128, 128, 0, st>>>(R, scal, active, flexible);
  return launched();
}
cudaError_t cg_update_xr_b(int64_t N, int R, int b, double* x, double* r, const double* p, const double* q,
                           const double* scal, cudaStream_t st) {
  cg_update_xr_b_kernel<<<grid_for(N * R * b), 256, 0, st>>>(N * R * b, R, b, x, r, p, q, scal);
  return launched();
}
cudaError_t cg_update_p_b(int64_t N, int R, int b, double* p, const double* z, const double* scal,
                          cudaStream_t st) {
  cg_update_p_b_kernel<<<grid_for(N * R * b), 256, 0, st>>>(N * R * b, R, b, p, z, scal);
  return launched();
}

}  // namespace ldgmg
