// Device kernels of the LDG multigrid hot path other than the operator
// applies: pool expansion, restriction/prolongation, bottom solve, FP64
// vector and CG kernels, batched layouts.  Written for sm_103a (GB300).
#include "kernels.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>

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

template <class T> __device__ __forceinline__ T from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return float(v); }
template <> __device__ __forceinline__ bf16 from_d<bf16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ f16 from_d<f16>(double v) { return __double2half(v); }

// --------------------------------------------------------------------------
// pool expansion (setup): vals[nz] = transpose(pool[ids[nz]]) in precision T
// --------------------------------------------------------------------------

template <class T>
__global__ void expand_kernel(int64_t total, int b, int cs, const uint32_t* __restrict__ ids,
                              const double* __restrict__ pool, T* __restrict__ vals, double scale) {
  const int64_t bb = int64_t(b) * b, bs = int64_t(b) * cs;   // pool block, stored block
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t nz = t / bs, e = t % bs;
    const int c = int(e / cs), r = int(e % cs);
    vals[t] = r >= b ? from_d<T>(0.0) : from_d<T>(scale * pool[int64_t(ids[nz]) * bb + int64_t(r) * b + c]);
  }
}

// tensor-core operand images: one thread per block entry (r, c)
template <bool SPLIT>
__global__ void expand_tc_kernel(int64_t total, int b, const uint32_t* __restrict__ ids,
                                 const double* __restrict__ pool, unsigned char* __restrict__ vals, double scale) {
  const int64_t bb = int64_t(b) * b;
  const int64_t img = bb * 2;                          // bytes of one BF16 image
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t nz = t / bb, e = t % bb;
    const int r = int(e / b), c = int(e % b);
    const double v = scale * pool[int64_t(ids[nz]) * bb + e];
    unsigned char* blk = vals + nz * img * (SPLIT ? 2 : 1);
    const uint32_t off = tc_image_offset(b, r, c);
    if (SPLIT) {
      const float a = float(v);
      const bf16 hi = __float2bfloat16_rn(a);
      const bf16 lo = __float2bfloat16_rn(a - __bfloat162float(hi));
      *reinterpret_cast<bf16*>(blk + off) = hi;
      *reinterpret_cast<bf16*>(blk + img + off) = lo;
    } else {
      *reinterpret_cast<bf16*>(blk + off) = __double2bfloat16(v);
    }
  }
}

cudaError_t expand_blocks(int64_t nnzb, int b, int cs, const uint32_t* ids, const double* pool, void* vals,
                          int prec, int tc_image, double scale, cudaStream_t st) {
  if (tc_image) {
    if (cs != b || (b != 16 && b != 64) || (prec != P_BF16 && prec != P_FP32)) return cudaErrorInvalidValue;
    const int64_t total = nnzb * b * b;
    if (total == 0) return cudaSuccess;
    const int grid = int(std::min<int64_t>((total + 255) / 256, 152 * 64));
    if (prec == P_FP32) expand_tc_kernel<true><<<grid, 256, 0, st>>>(total, b, ids, pool, (unsigned char*)vals, scale);
    else expand_tc_kernel<false><<<grid, 256, 0, st>>>(total, b, ids, pool, (unsigned char*)vals, scale);
    return launched();
  }
  const int64_t total = nnzb * b * cs;
  if (total == 0) return cudaSuccess;
  const int grid = int(std::min<int64_t>((total + 255) / 256, 152 * 64));
  switch (prec) {
    case P_FP64: expand_kernel<double><<<grid, 256, 0, st>>>(total, b, cs, ids, pool, (double*)vals, scale); break;
    case P_FP32: expand_kernel<float><<<grid, 256, 0, st>>>(total, b, cs, ids, pool, (float*)vals, scale); break;
    case P_BF16: expand_kernel<bf16><<<grid, 256, 0, st>>>(total, b, cs, ids, pool, (bf16*)vals, scale); break;
    case P_FP16: expand_kernel<f16><<<grid, 256, 0, st>>>(total, b, cs, ids, pool, (f16*)vals, scale); break;
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
// of an element are contiguous in the [element][rhs][mode] layout.  The
// right-hand sides are taken in chunks of Rc; within a chunk the 2^d children
// are transformed together, so a chunk costs d + 2 barriers whatever d and R.
// Work item i = (child s, rhs rr, mode t) with i = (s*Rc + rr)*b + t.  The 1D
// transform along axis a uses the child's own factor P[s_a]; the arithmetic
// of every output (the order of the k-sums and of the sum over children) is
// independent of R and of Rc.  The arithmetic runs in the vector precision:
// FP64 for FP64 vectors, FP32 for the reduced-precision V-cycle (GB300's FP64
// pipe would otherwise bound these kernels well below HBM speed).
constexpr int kXferCap = 2048;          // work items per chunk (2 buffers of TV)
constexpr int kXferMaxThreads = 256;

template <class TV>
__device__ __forceinline__ void load_P(TV (*Ps)[8][8], const double* P, int q) {
  for (int i = threadIdx.x; i < 2 * q * q; i += blockDim.x) {
    const int s = i / (q * q), r = (i / q) % q, c = i % q;
    Ps[s][r][c] = TV(P[i]);
  }
}

static int xfer_chunk(int d, int b, int R) {
  const int per = (1 << d) * b;
  return std::max(1, std::min(R, kXferCap / per));
}

template <bool RESTRICT, class TV>
__global__ void __launch_bounds__(kXferMaxThreads) xfer_kernel(int d, int q, int nf, const double* __restrict__ P,
                                                               const TV* __restrict__ src, TV* __restrict__ dst,
                                                               int R, int Rc) {
  extern __shared__ __align__(16) unsigned char xraw[];
  TV* xbuf = reinterpret_cast<TV*>(xraw);
  __shared__ TV Ps[2][8][8];
  load_P(Ps, P, q);
  const int b = (d == 2) ? q * q : q * q * q;
  const int nch = 1 << d;
  const int64_t nc = nf / 2;
  const int64_t C = blockIdx.x;
  // fine element of child s: fbase + (s_0) + (s_1) nf + (s_2) nf^2
  const int64_t c0 = C % nc, c1 = (C / nc) % nc, c2 = C / (nc * nc);
  const int64_t nf2 = int64_t(nf) * nf;
  const int64_t fbase = 2 * c0 + 2 * c1 * nf + (d == 3 ? 2 * c2 * nf2 : 0);
  auto fidx = [&](int s) -> int64_t { return fbase + (s & 1) + ((s >> 1) & 1) * nf + ((s >> 2) & 1) * nf2; };
  const int64_t row = int64_t(R) * b;            // entries per element
  TV* buf0 = xbuf;
  TV* buf1 = xbuf + nch * Rc * b;
  for (int r0 = 0; r0 < R; r0 += Rc) {
    const int seg = min(Rc, R - r0) * b;          // entries per child in this chunk
    const int tot = nch * seg;
    __syncthreads();                               // previous chunk done with the buffers
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int s = i / seg, o = i - s * seg;
      buf0[i] = RESTRICT ? src[fidx(s) * row + int64_t(r0) * b + o] : src[C * row + int64_t(r0) * b + o];
    }
    __syncthreads();
    TV* in = buf0;
    TV* out = buf1;
    int stride = 1;
    for (int a = 0; a < d; ++a) {
      for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        const int s = i / seg, o = i - s * seg;
        const int t = o % b;
        const int ka = (t / stride) % q;
        const int base = i - ka * stride;
        const int sa = (s >> a) & 1;
        TV v = TV(0);
        for (int k = 0; k < q; ++k) v += (RESTRICT ? Ps[sa][k][ka] : Ps[sa][ka][k]) * in[base + k * stride];
        out[i] = v;
      }
      __syncthreads();
      TV* tmp = in;
      in = out;
      out = tmp;
      stride *= q;
    }
    if (RESTRICT) {
      for (int o = threadIdx.x; o < seg; o += blockDim.x) {
        TV acc = TV(0);
        for (int s = 0; s < nch; ++s) acc += in[s * seg + o];
        dst[C * row + int64_t(r0) * b + o] = acc;
      }
    } else {
      for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        const int s = i / seg, o = i - s * seg;
        TV* y = dst + fidx(s) * row + int64_t(r0) * b + o;
        *y = *y + in[i];
      }
    }
  }
}

static int64_t coarse_count(int d, int nf) {
  int64_t nc = nf / 2, r = 1;
  for (int a = 0; a < d; ++a) r *= nc;
  return r;
}

// The largest chunk needs 2 * max(kXferCap, 8 * 8^3) doubles = 64 KB of dynamic
// shared memory; the opt-in is set once for every instance (thread safe).
static cudaError_t xfer_config() {
  static std::once_flag once;
  static cudaError_t cfg = cudaSuccess;
  std::call_once(once, [] {
    const int smem = 2 * 4096 * int(sizeof(double));
    cfg = cudaFuncSetAttribute(xfer_kernel<true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cfg == cudaSuccess) cfg = cudaFuncSetAttribute(xfer_kernel<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cfg == cudaSuccess) cfg = cudaFuncSetAttribute(xfer_kernel<false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cfg == cudaSuccess) cfg = cudaFuncSetAttribute(xfer_kernel<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  return cfg;
}

template <bool RESTRICT>
static cudaError_t xfer_apply(int d, int q, int n_fine, const double* P, const void* src, void* dst,
                              int vprec, int R, cudaStream_t st) {
  if (q < 1 || q > 8 || (d != 2 && d != 3) || R < 1 || n_fine < 2) return cudaErrorInvalidValue;
  const int b = (d == 2) ? q * q : q * q * q;
  const int Rc = xfer_chunk(d, b, R);
  const int tot = (1 << d) * Rc * b;
  const int smem = 2 * tot * (vprec == 0 ? 8 : 4);
  if (smem > 48 * 1024) {
    cudaError_t e = xfer_config();
    if (e != cudaSuccess) return e;
  }
  const int threads = std::min(kXferMaxThreads, (tot + 31) / 32 * 32);
  const int64_t Nc = coarse_count(d, n_fine);
  if (vprec == 0)
    xfer_kernel<RESTRICT, double><<<unsigned(Nc), threads, smem, st>>>(d, q, n_fine, P, (const double*)src, (double*)dst, R, Rc);
  else
    xfer_kernel<RESTRICT, float><<<unsigned(Nc), threads, smem, st>>>(d, q, n_fine, P, (const float*)src, (float*)dst, R, Rc);
  return launched();
}

cudaError_t restrict_apply(int d, int q, int n_fine, const double* P, const void* rf, void* rc,
                           int vprec, int R, cudaStream_t st) {
  return xfer_apply<true>(d, q, n_fine, P, rf, rc, vprec, R, st);
}

cudaError_t prolong_apply(int d, int q, int n_fine, const double* P, const void* xc, void* xf,
                          int vprec, int R, cudaStream_t st) {
  return xfer_apply<false>(d, q, n_fine, P, xc, xf, vprec, R, st);
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

// GMRES vector steps (FP64): y += sgn * coef[0] * x with the coefficient read on
// the device (a Hessenberg entry), y = x / s, and x += sum_i y_i Q_i.
__global__ void axpy_dev_kernel(int64_t n, const double* __restrict__ coef, double sgn, const double* __restrict__ x,
                                double* __restrict__ y) {
  const double a = sgn * coef[0];
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x)
    y[t] += a * x[t];
}

__global__ void div_kernel(int64_t n, double s, const double* x, double* y) {   // x may alias y
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x)
    y[t] = x[t] / s;
}

__global__ void combine_kernel(int64_t n, int k, const double* __restrict__ Q, int64_t ldq,
                               const double* __restrict__ y, double* __restrict__ x) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += y[i] * Q[int64_t(i) * ldq + t];
    x[t] += acc;
  }
}

cudaError_t axpy_dev(int64_t n, const double* coef, double sgn, const double* x, double* y, cudaStream_t st) {
  axpy_dev_kernel<<<grid_for(n), 256, 0, st>>>(n, coef, sgn, x, y);
  return launched();
}

cudaError_t vec_div(int64_t n, double s, const double* x, double* y, cudaStream_t st) {
  div_kernel<<<grid_for(n), 256, 0, st>>>(n, s, x, y);
  return launched();
}

cudaError_t vec_combine(int64_t n, int k, const double* Q, int64_t ldq, const double* y, double* x,
                        cudaStream_t st) {
  combine_kernel<<<grid_for(n), 256, 0, st>>>(n, k, Q, ldq, y, x);
  return launched();
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

__global__ void cg_check_b_kernel(int R, const double* s, int* active, int* it, int* flag, double* hist,
                                  int hist_cap) {
  const int r = threadIdx.x + blockIdx.x * blockDim.x;
  if (r >= R || !active[r]) return;
  it[r] += 1;
  const double rr = s[S_RR * R + r];
  if (hist && it[r] < hist_cap) hist[int64_t(it[r]) * R + r] = rr;
  if (!isfinite(rr)) {
    flag[r] = 1;
    active[r] = 0;
  } else if (rr <= s[S_TOL2 * R + r] * s[S_BB * R + r]) {
    active[r] = 0;
  }
}

cudaError_t cg_check_b(int R, const double* scal, int* active, int* it, int* flag, double* hist, int hist_cap,
                       cudaStream_t st) {
  cg_check_b_kernel<<<(R + 127) / 128, 128, 0, st>>>(R, scal, active, it, flag, hist, hist_cap);
  return launched();
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
