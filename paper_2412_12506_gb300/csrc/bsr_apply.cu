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
#include <cstdint>

namespace ldgmg {

typedef __nv_bfloat16 bf16;
typedef __half f16;

__device__ __forceinline__ float to_f(bf16 v) { return __bfloat162float(v); }

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
  const int* rows;  // null: block rows 0..nrows-1; else the nrows block rows listed
};

template <int TEAM> __device__ __forceinline__ void team_sync() {
  if (TEAM == 32) __syncwarp(); else __syncthreads();
}

template <int B, class TA, class TV>
__global__ void __launch_bounds__(256) bsr_kernel(BsrArgs<TA, TV> a) {
  typedef typename AccOf<TA>::type TACC;
  constexpr int CS = (B + 3) / 4 * 4;      // column stride of the stored block (padding rows are zero)
  constexpr int VEC = vec_for<TA>(CS);
  constexpr int TEAM = (B > 32) ? 256 : 32;
  constexpr int LPC = CS / VEC;            // threads per column
  constexpr int G = TEAM / LPC;            // column groups per team
  constexpr int TEAMS = 256 / TEAM;        // block rows per CTA
  constexpr int STEPS = (B + G - 1) / G;   // load steps per block
  static_assert(G >= 1, "team too small");
  constexpr int KMAX = 16;                 // blocks whose x_j are staged at once
  __shared__ TACC xs[TEAMS][KMAX][B];
  __shared__ TACC red[TEAMS][G][CS];

  const int team = threadIdx.x / TEAM, lt = threadIdx.x % TEAM;
  const int g = lt / LPC, rl = lt % LPC;
  const bool active = g < G;
  const int64_t t = int64_t(blockIdx.x) * TEAMS + team;     // team's position in the row range / list
  const bool live = t < a.nrows;
  const int64_t row = (a.rows && live) ? int64_t(a.rows[t]) : t;
  const int64_t roff = int64_t(blockIdx.y) * a.rs;
  if (TEAM == 32 && !live) return;            // whole warp leaves together
  TACC acc[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc[v] = TACC(0);

  if (live) {
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
          const TA* blk = a.vals + int64_t(zb + kk) * (B * CS) + rl * VEC;
#pragma unroll 4
          for (int st = 0; st < STEPS; ++st) {
            const int c = st * G + g;
            if (c < B) {
              const VecT<TA, VEC> w = *reinterpret_cast<const VecT<TA, VEC>*>(blk + c * CS);
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
  if (live && lt < B) {
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
    case 4: case 8: case 9: case 12: case 16: case 25: case 27: case 32: case 36: case 48: case 64: return true;
    default: return false;
  }
}

template <int B, class TA, class TV>
static cudaError_t launch_bsr_b(const DevMat& M, const BsrArgs<TA, TV>& a, cudaStream_t st) {
  constexpr int TEAMS = (B > 32) ? 1 : 8;
  (void)M;
  if (a.nrows == 0) return cudaSuccess;
  const int64_t grid = (a.nrows + TEAMS - 1) / TEAMS;
  bsr_kernel<B, TA, TV><<<dim3(unsigned(grid), unsigned(a.R)), 256, 0, st>>>(a);
  return launched();
}

template <class TA, class TV>
static cudaError_t launch_bsr_t(const DevMat& M, const int* rows, int64_t count, int mode, const void* x,
                                const void* rhs, const void* xin, void* y, double s, int R, int64_t es,
                                int64_t rs, cudaStream_t st) {
  BsrArgs<TA, TV> a;
  a.nrows = rows ? count : M.nrows;
  a.rows = rows;
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
    case 12: return launch_bsr_b<12>(M, a, st);
    case 16: return launch_bsr_b<16>(M, a, st);
    case 25: return launch_bsr_b<25>(M, a, st);
    case 27: return launch_bsr_b<27>(M, a, st);
    case 32: return launch_bsr_b<32>(M, a, st);
    case 36: return launch_bsr_b<36>(M, a, st);
    case 48: return launch_bsr_b<48>(M, a, st);
    case 64: return launch_bsr_b<64>(M, a, st);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t bsr_dispatch(const DevMat& M, const int* rows, int64_t count, int mode, const void* x,
                                const void* rhs, const void* xin, void* y, double s, int R, int64_t es, int64_t rs,
                                cudaStream_t st) {
  if (M.tc_image || R < 1 || count < 0) return cudaErrorInvalidValue;
  switch (M.prec) {
    case P_FP64: return launch_bsr_t<double, double>(M, rows, count, mode, x, rhs, xin, y, s, R, es, rs, st);
    case P_FP32: return launch_bsr_t<float, float>(M, rows, count, mode, x, rhs, xin, y, s, R, es, rs, st);
    case P_BF16: return launch_bsr_t<bf16, float>(M, rows, count, mode, x, rhs, xin, y, s, R, es, rs, st);
    case P_FP16: return launch_bsr_t<f16, float>(M, rows, count, mode, x, rhs, xin, y, s, R, es, rs, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t bsr_apply_strided(const DevMat& M, int mode, const void* x, const void* rhs, const void* xin,
                              void* y, double s, int R, int64_t es, int64_t rs, cudaStream_t st) {
  return bsr_dispatch(M, nullptr, M.nrows, mode, x, rhs, xin, y, s, R, es, rs, st);
}

cudaError_t bsr_apply_rows(const DevMat& M, const int* rows, int64_t count, int mode, const void* x, const void* rhs,
                           const void* xin, void* y, double s, int R, int64_t es, int64_t rs, cudaStream_t st) {
  if (!rows) return cudaErrorInvalidValue;
  return bsr_dispatch(M, rows, count, mode, x, rhs, xin, y, s, R, es, rs, st);
}

cudaError_t bsr_apply(const DevMat& M, int mode, const void* x, const void* rhs, const void* xin,
                      void* y, double s, cudaStream_t st) {
  return bsr_apply_strided(M, mode, x, rhs, xin, y, s, 1, M.b, 0, st);
}

}  // namespace ldgmg
