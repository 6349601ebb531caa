// Batched operator apply in double-FP32 ("double-float") arithmetic.
//
// The outer CG of a batched solve needs y = A x to FP64-level accuracy for R
// right-hand sides at once.  GB300's FP64 rate is ~1/64 of its FP32 rate, so
// this kernel keeps the FP64 accuracy without FP64 multiply-adds:
//   * A is stored as pairs (a_hi, a_lo) of FP32 with a = a_hi + a_lo exactly to
//     ~2^-48 (same 8 bytes per entry as FP64), column-major per block;
//   * x_j is split the same way when it is staged (one FP64 subtraction per
//     entry of x, not per multiply-add);
//   * each product a*x is a_hi*x_hi taken exactly with an FMA (TwoProd) plus
//     the cross terms a_hi*x_lo + a_lo*x_hi, accumulated in an FP32 pair with
//     TwoSum (Knuth), about 12 FP32 operations per multiply-add.
// The rounding error is ~2^-44 of sum |a_ij x_j| (FP64's is 2^-53), far below
// what CG needs to reach a 1e-10 residual.  Each block is read once per row
// and applied to all R right-hand sides (one CTA per block row), so the
// matrix streams once regardless of R.
#include "kernels.h"

#include <mutex>

#include <algorithm>
#include <cstdint>

namespace ldgmg {

namespace {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

template <int B>
__global__ void __launch_bounds__(256, 2) bsr_df_kernel(int64_t nrows, const int* __restrict__ row_ptr,
                                                     const int* __restrict__ col, const float2* __restrict__ vals,
                                                     const double* __restrict__ x, const double* __restrict__ rhs,
                                                     double* __restrict__ y, int R, int mode) {
  extern __shared__ __align__(16) float2 sm[];
  float2* As = sm;              // B*B pairs, column-major
  float2* Xs = sm + B * B;      // R*B pairs, [rhs][c]
  constexpr int MAXO = (64 * B + 255) / 256;    // outputs per thread for R <= 64
  const int tid = threadIdx.x;
  const int nout = R * B;
  const int64_t row = blockIdx.x;
  float hi[MAXO], lo[MAXO];
#pragma unroll
  for (int k = 0; k < MAXO; ++k) hi[k] = lo[k] = 0.0f;
  const int z0 = row_ptr[row], z1 = row_ptr[row + 1];
  for (int nz = z0; nz < z1; ++nz) {
    const int64_t j = col[nz];
    __syncthreads();
    const float2* blk = vals + int64_t(nz) * (B * B);
    for (int t = tid; t < B * B; t += 256) As[t] = blk[t];
    const double* xj = x + j * int64_t(R) * B;
    for (int t = tid; t < nout; t += 256) {
      const double v = xj[t];
      const float vh = float(v);
      Xs[t] = make_float2(vh, float(v - double(vh)));
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < MAXO; ++k) {
      const int o = tid + k * 256;
      if (o < nout) {
        const int rr = o / B, r = o % B;
        const float2* xr = Xs + rr * B;
        float s = hi[k], e = lo[k];
#pragma unroll 4
        for (int c = 0; c < B; ++c) {
          const float2 a = As[c * B + r];
          const float2 xv = xr[c];
          const float p = a.x * xv.x;
          const float pe = fmaf(a.x, xv.x, -p);                 // exact error of a_hi * x_hi
          const float cross = fmaf(a.x, xv.y, a.y * xv.x);     // a_hi x_lo + a_lo x_hi
          float t, te;
          two_sum(s, p, t, te);
          s = t;
          e += te + pe + cross;
        }
        hi[k] = s;
        lo[k] = e;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < MAXO; ++k) {
    const int o = tid + k * 256;
    if (o < nout) {
      const double acc = double(hi[k]) + double(lo[k]);
      const int64_t off = row * int64_t(R) * B + o;
      y[off] = (mode == M_RES) ? rhs[off] - acc : acc;
    }
  }
}

// The same block-reuse structure in plain FP64 (one CTA per block row, every
// block applied to all R right-hand sides; FP64 multiply-adds).
template <int B>
__global__ void __launch_bounds__(256, 2) bsr_multi64_kernel(int64_t nrows, const int* __restrict__ row_ptr,
                                                             const int* __restrict__ col,
                                                             const double* __restrict__ vals,
                                                             const double* __restrict__ x,
                                                             const double* __restrict__ rhs,
                                                             double* __restrict__ y, int R, int mode) {
  extern __shared__ __align__(16) double smd[];
  double* As = smd;             // B*B, column-major
  double* Xs = smd + B * B;     // R*B, [rhs][c]
  constexpr int MAXO = (64 * B + 255) / 256;
  const int tid = threadIdx.x;
  const int nout = R * B;
  const int64_t row = blockIdx.x;
  double acc[MAXO];
#pragma unroll
  for (int k = 0; k < MAXO; ++k) acc[k] = 0.0;
  const int z0 = row_ptr[row], z1 = row_ptr[row + 1];
  for (int nz = z0; nz < z1; ++nz) {
    const int64_t j = col[nz];
    __syncthreads();
    const double* blk = vals + int64_t(nz) * (B * B);
    for (int t = tid; t < B * B; t += 256) As[t] = blk[t];
    const double* xj = x + j * int64_t(R) * B;
    for (int t = tid; t < nout; t += 256) Xs[t] = xj[t];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < MAXO; ++k) {
      const int o = tid + k * 256;
      if (o < nout) {
        const int rr = o / B, r = o % B;
        const double* xr = Xs + rr * B;
        double s = acc[k];
#pragma unroll 4
        for (int c = 0; c < B; ++c) s = fma(As[c * B + r], xr[c], s);
        acc[k] = s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < MAXO; ++k) {
    const int o = tid + k * 256;
    if (o < nout) {
      const int64_t off = row * int64_t(R) * B + o;
      y[off] = (mode == M_RES) ? rhs[off] - acc[k] : acc[k];
    }
  }
}

// Single right-hand side: the team layout of the CUDA-core block-row kernel
// (a warp per row for b = 16, the CTA for b = 64; column groups of threads
// read 16-byte runs = 2 pairs of one column), with the same double-FP32
// arithmetic and a fixed-order TwoSum reduction of the group partials.
template <int B>
__global__ void __launch_bounds__(256) bsr_df1_kernel(int64_t nrows, const int* __restrict__ row_ptr,
                                                      const int* __restrict__ col, const float2* __restrict__ vals,
                                                      const double* __restrict__ x, const double* __restrict__ rhs,
                                                      double* __restrict__ y, int mode) {
  constexpr int VEC = 2;                    // pairs per 16-byte load
  constexpr int TEAM = (B > 32) ? 256 : 32;
  constexpr int LPC = B / VEC;
  constexpr int G = TEAM / LPC;
  constexpr int TEAMS = 256 / TEAM;
  constexpr int STEPS = B / G;
  constexpr int KMAX = 16;
  __shared__ float2 xs[TEAMS][KMAX][B];
  __shared__ float red_hi[TEAMS][G][B], red_lo[TEAMS][G][B];
  const int team = threadIdx.x / TEAM, lt = threadIdx.x % TEAM;
  const int g = lt / LPC, rl = lt % LPC;
  const int64_t row = int64_t(blockIdx.x) * TEAMS + team;
  if (TEAM == 32 && row >= nrows) return;
  float hi[VEC] = {0.0f, 0.0f}, lo[VEC] = {0.0f, 0.0f};
  if (row < nrows) {
    const int z0 = row_ptr[row], z1 = row_ptr[row + 1];
    for (int zb = z0; zb < z1; zb += KMAX) {
      const int nb = min(KMAX, z1 - zb);
      if (TEAM == 32) __syncwarp(); else __syncthreads();
      for (int t = lt; t < nb * B; t += TEAM) {
        const int kk = t / B, c = t % B;
        const double v = x[int64_t(col[zb + kk]) * B + c];
        const float h = float(v);
        xs[team][kk][c] = make_float2(h, float(v - double(h)));
      }
      if (TEAM == 32) __syncwarp(); else __syncthreads();
      for (int kk = 0; kk < nb; ++kk) {
        const float4* blk = reinterpret_cast<const float4*>(vals + int64_t(zb + kk) * (B * B) + rl * VEC);
#pragma unroll 4
        for (int st = 0; st < STEPS; ++st) {
          const int c = st * G + g;
          const float4 w = blk[c * (B / 2)];          // pairs (r, c), (r+1, c): a_hi, a_lo, a_hi', a_lo'
          const float2 xv = xs[team][kk][c];
          const float a[2][2] = {{w.x, w.y}, {w.z, w.w}};
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const float p = a[v][0] * xv.x;
            const float pe = fmaf(a[v][0], xv.x, -p);
            const float cross = fmaf(a[v][0], xv.y, a[v][1] * xv.x);
            float t, te;
            two_sum(hi[v], p, t, te);
            hi[v] = t;
            lo[v] += te + pe + cross;
          }
        }
      }
    }
  }
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    red_hi[team][g][rl * VEC + v] = hi[v];
    red_lo[team][g][rl * VEC + v] = lo[v];
  }
  if (TEAM == 32) __syncwarp(); else __syncthreads();
  if (row < nrows && lt < B) {
    float S = 0.0f, E = 0.0f;
    for (int gg = 0; gg < G; ++gg) {
      float t, te;
      two_sum(S, red_hi[team][gg][lt], t, te);
      S = t;
      E += te + red_lo[team][gg][lt];
    }
    const double acc = double(S) + double(E);
    const int64_t o = row * B + lt;
    y[o] = (mode == M_RES) ? rhs[o] - acc : acc;
  }
}

__global__ void split_kernel(int64_t n, const double* __restrict__ src, float2* __restrict__ dst) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
    const double v = src[t];
    const float h = float(v);
    dst[t] = make_float2(h, float(v - double(h)));
  }
}

}  // namespace

cudaError_t split_to_float_pairs(int64_t n, const double* src, void* dst, cudaStream_t st) {
  const int grid = int(std::min<int64_t>((n + 255) / 256, 152 * 32));
  if (n <= 0) return cudaSuccess;
  split_kernel<<<grid, 256, 0, st>>>(n, src, static_cast<float2*>(dst));
  return launched();
}

cudaError_t bsr_apply_df(const DevMat& M, const void* pairs, int mode, const double* x, const double* rhs, double* y,
                         int R, cudaStream_t st) {
  if (R < 1 || R > 64 || M.nrows == 0) return M.nrows == 0 ? cudaSuccess : cudaErrorInvalidValue;
  if (mode != M_Y && mode != M_RES) return cudaErrorInvalidValue;
  const float2* v = static_cast<const float2*>(pairs);
  switch (M.b) {
#define LDGMG_DF_CASE(BB)                                                                                  \
  case BB: {                                                                                               \
    const size_t smem = size_t(BB * BB + R * BB) * sizeof(float2);                                         \
    static std::once_flag once;                                                                            \
    static cudaError_t cfg = cudaSuccess;                                                                  \
    std::call_once(once, [] {                                                                              \
      cfg = cudaFuncSetAttribute(bsr_df_kernel<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                 int(size_t(BB * BB + 64 * BB) * sizeof(float2)));                         \
    });                                                                                                    \
    if (cfg != cudaSuccess) return cfg;                                                                    \
    bsr_df_kernel<BB><<<unsigned(M.nrows), 256, smem, st>>>(M.nrows, M.row_ptr, M.col, v, x, rhs, y, R,    \
                                                            mode);                                         \
    return launched();                                                                                     \
  }
    LDGMG_DF_CASE(16)
    LDGMG_DF_CASE(64)
#undef LDGMG_DF_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t bsr_apply_df1(const DevMat& M, const void* pairs, int mode, const double* x, const double* rhs,
                          double* y, cudaStream_t st) {
  if (M.nrows == 0) return cudaSuccess;
  if (mode != M_Y && mode != M_RES) return cudaErrorInvalidValue;
  const float2* v = static_cast<const float2*>(pairs);
  switch (M.b) {
    case 16:
      bsr_df1_kernel<16><<<unsigned((M.nrows + 7) / 8), 256, 0, st>>>(M.nrows, M.row_ptr, M.col, v, x, rhs, y, mode);
      return launched();
    case 64:
      bsr_df1_kernel<64><<<unsigned(M.nrows), 256, 0, st>>>(M.nrows, M.row_ptr, M.col, v, x, rhs, y, mode);
      return launched();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t bsr_apply_multi64(const DevMat& M, int mode, const double* x, const double* rhs, double* y, int R,
                              cudaStream_t st) {
  if (R < 1 || R > 64 || M.nrows == 0) return M.nrows == 0 ? cudaSuccess : cudaErrorInvalidValue;
  if (mode != M_Y && mode != M_RES) return cudaErrorInvalidValue;
  const double* v = static_cast<const double*>(M.vals);
  switch (M.b) {
#define LDGMG_M64_CASE(BB)                                                                                      \
  case BB: {                                                                                                    \
    const size_t smem = size_t(BB * BB + R * BB) * sizeof(double);                                              \
    static std::once_flag once;                                                                                 \
    static cudaError_t cfg = cudaSuccess;                                                                       \
    std::call_once(once, [] {                                                                                   \
      cfg = cudaFuncSetAttribute(bsr_multi64_kernel<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                 int(size_t(BB * BB + 64 * BB) * sizeof(double)));                              \
    });                                                                                                         \
    if (cfg != cudaSuccess) return cfg;                                                                         \
    bsr_multi64_kernel<BB><<<unsigned(M.nrows), 256, smem, st>>>(M.nrows, M.row_ptr, M.col, v, x, rhs, y, R,     \
                                                                 mode);                                         \
    return launched();                                                                                          \
  }
    LDGMG_M64_CASE(16)
    LDGMG_M64_CASE(64)
#undef LDGMG_M64_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ldgmg
