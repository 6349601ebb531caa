// Batched-RHS block-row apply on the 5th-generation tensor cores (tcgen05).
//
// For R right-hand sides the element-block apply of Sec. 2.3 becomes, per
// block row i,  Y_i^T (R x b) = sum_j X_j^T (R x b) * A_ij^T (b x b),  a
// chain of dense contractions.  Each is issued as tcgen05.mma kind::f16 with
//   M = 128 (right-hand sides; rows >= R are zero),  N = b,  K = 16 per step,
// BF16 operands and an FP32 accumulator in tensor memory.  The FP32 vectors
// are split into hi + lo BF16 parts (hi = bf16(x), lo = bf16(x - hi)) and both
// are multiplied, so the product carries ~16 bits of x -- the same accuracy
// as the CUDA-core path that multiplies BF16-stored blocks by FP32 vectors.
// With FP32-stored blocks the matrix is split the same way while it is staged
// and three products are accumulated (A_hi x_hi + A_hi x_lo + A_lo x_hi;
// A_lo x_lo is below 2^-16 of the result), which gives FP32-like accuracy on
// the BF16 tensor cores.
//
// Operands are staged into shared memory in the canonical K-major,
// no-swizzle layout: 8-row x 16-byte core matrices, rows 16 B apart, core
// matrices adjacent in K 128 B apart (LBO) and adjacent in M/N
// (b/8)*128 B apart (SBO).  Matrix blocks are stored row-major in HBM for
// this path, so a block row of 8 BF16 values is one 16-byte copy.
//
// One CTA of 128 threads (4 warps) owns one block row at a time; thread 0
// issues the MMAs and commits them to an mbarrier; all threads wait on it
// with a bounded spin, then warp w reads TMEM lanes 32w..32w+31 (one right-
// hand side per lane) and applies the fused epilogue.  Several CTAs share an
// SM (TMEM 32 or 64 columns each), which overlaps staging with MMAs.
#include "kernels.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

namespace ldgmg {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;
constexpr unsigned kSpinLimit = 1u << 20;   // bounded waits: error flag instead of a hang

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version of the sm_100 family; base offset 0, no swizzle
  return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 16 columns of 32-bit TMEM words: this thread's lane, 16 columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// byte offset of element (row, k) in a K-major no-swizzle operand with KQ = b/8 core matrices along K
__device__ __forceinline__ uint32_t core_off(int row, int kq, int KQ) {
  return uint32_t(((row >> 3) * KQ + kq) * 128 + (row & 7) * 16);
}

template <int B, bool SPLIT>
struct TcSmem {
  static constexpr int KQ = B / 8;
  static constexpr int A_BYTES = kTcM * B * 2;   // one BF16 operand part (hi or lo)
  static constexpr int B_BYTES = B * B * 2;
  static constexpr int TOTAL = 2 * A_BYTES + (SPLIT ? 2 : 1) * B_BYTES + 128;
};

template <int B, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads) bsr_tc_kernel(BatchArgs a) {
  static_assert(B == 16 || B == 64, "tensor-core path supports b = 16 and b = 64");
  constexpr int KQ = B / 8;
  constexpr int KSTEPS = B / 16;
  constexpr uint32_t NCOLS = B < 32 ? 32 : B;
  constexpr uint32_t IDESC = make_idesc(kTcM, B);
  extern __shared__ __align__(1024) unsigned char smem[];
  typedef TcSmem<B, SPLIT> L;
  unsigned char* a_hi = smem;
  unsigned char* a_lo = smem + L::A_BYTES;
  unsigned char* b_op = smem + 2 * L::A_BYTES;
  unsigned char* b_lo = b_op + L::B_BYTES;       // used only when SPLIT
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::TOTAL - 128);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = a.R;
  // zero the A-operand rows of absent right-hand sides once (staging never writes them)
  for (int t = tid; t < kTcM * KQ; t += kTcThreads) {
    const int m = t / KQ, kq = t % KQ;
    if (m >= R) {
      *reinterpret_cast<uint4*>(a_hi + core_off(m, kq, KQ)) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(a_lo + core_off(m, kq, KQ)) = make_uint4(0, 0, 0, 0);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sa_hi = smem_u32(a_hi), sa_lo = smem_u32(a_lo), sb = smem_u32(b_op), sb_lo = smem_u32(b_lo);
  constexpr uint32_t SBO = KQ * 128;
  uint32_t phase = 0;
  bool timed_out = false;

  for (int64_t row = blockIdx.x; row < a.nrows && !timed_out; row += gridDim.x) {
    const int z0 = a.row_ptr[row], z1 = a.row_ptr[row + 1];
    for (int nz = z0; nz < z1; ++nz) {
      const int64_t j = a.col[nz];
      // stage A_ij (row-major): chunk (r, kq) = 8 consecutive columns of row r
      if (!SPLIT) {
        const uint4* blk = reinterpret_cast<const uint4*>(a.vals) + int64_t(nz) * (B * B / 8);
        for (int t = tid; t < B * KQ; t += kTcThreads) {
          const int r = t / KQ, kq = t % KQ;
          *reinterpret_cast<uint4*>(b_op + core_off(r, kq, KQ)) = __ldg(blk + t);
        }
      } else {
        const float4* blk = reinterpret_cast<const float4*>(a.vals) + int64_t(nz) * (B * B / 4);
        for (int t = tid; t < B * KQ; t += kTcThreads) {
          const int r = t / KQ, kq = t % KQ;
          const float4 v0 = __ldg(blk + 2 * t), v1 = __ldg(blk + 2 * t + 1);
          const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
            const float2 hf = __bfloat1622float2(h);
            hi[e] = *reinterpret_cast<const uint32_t*>(&h);
            lo[e] = pack_bf16(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
          }
          *reinterpret_cast<uint4*>(b_op + core_off(r, kq, KQ)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(b_lo + core_off(r, kq, KQ)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
      // stage X_j^T as hi/lo BF16: chunk (m, kq) = modes 8kq..8kq+7 of right-hand side m
      const float* xj = a.x + j * a.es;
      for (int t = tid; t < R * KQ; t += kTcThreads) {
        const int m = t / KQ, kq = t % KQ;
        const float4* src = reinterpret_cast<const float4*>(xj + int64_t(m) * a.rs + kq * 8);
        const float4 v0 = __ldg(src), v1 = __ldg(src + 1);
        const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
          const float2 hf = __bfloat1622float2(h);
          hi[e] = *reinterpret_cast<const uint32_t*>(&h);
          lo[e] = pack_bf16(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
        }
        *reinterpret_cast<uint4*>(a_hi + core_off(m, kq, KQ)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(a_lo + core_off(m, kq, KQ)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int s = 0; s < KSTEPS; ++s) {
          const uint64_t bd = make_sdesc(sb + 256u * s, 128u, SBO);
          const uint64_t ah = make_sdesc(sa_hi + 256u * s, 128u, SBO);
          mma_bf16(tmem, ah, bd, IDESC, (nz > z0 || s > 0) ? 1u : 0u);
          mma_bf16(tmem, make_sdesc(sa_lo + 256u * s, 128u, SBO), bd, IDESC, 1u);
          if (SPLIT) mma_bf16(tmem, ah, make_sdesc(sb_lo + 256u * s, 128u, SBO), IDESC, 1u);
        }
        mma_commit(bar);
      }
      // wait for the MMAs (they read the staged operands) before restaging;
      // the give-up decision is made together so no thread is left at a barrier
      bool gave_up = false;
      unsigned spins = 0;
      while (!mbar_try_wait(bar, phase)) {
        if (++spins > kSpinLimit) {
          gave_up = true;
          break;
        }
      }
      if (__syncthreads_or(gave_up)) {
        timed_out = true;
        break;
      }
      phase ^= 1u;
    }
    if (timed_out) break;
    tc_fence_after();
    // epilogue: warp w holds right-hand sides 32w..32w+31, one per lane
    const int m = warp * 32 + lane;
    const bool empty = (z1 == z0);
#pragma unroll
    for (int c0 = 0; c0 < B; c0 += 16) {
      float acc[16];
      tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), acc);
      if (m < R) {
        const int64_t o = row * a.es + int64_t(m) * a.rs + c0;
#pragma unroll
        for (int q = 0; q < 16; q += 4) {
          float4 y;
          float* yy = reinterpret_cast<float*>(&y);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float s = empty ? 0.0f : acc[q + e];
            float out;
            switch (a.mode) {
              case M_Y: out = s; break;
              case M_RES: out = a.rhs[o + q + e] - s; break;
              case M_AXPY: out = a.xin[o + q + e] + float(a.s) * s; break;
              default: out = float(a.s) * s; break;
            }
            yy[e] = out;
          }
          *reinterpret_cast<float4*>(a.y + o + q) = y;
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (timed_out) {
    if (tid == 0 && a.err) atomicExch(a.err, 1);
    // give the outstanding MMAs a second bounded chance to finish before TMEM is released
    unsigned spins = 0;
    while (!mbar_try_wait(bar, phase) && ++spins < kSpinLimit) {
    }
  }
  // every thread is past its last MMA wait (or gave up); release TMEM
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

}  // namespace

bool tc_block_size_supported(int b) { return b == 16 || b == 64; }

template <int B, bool SPLIT>
static cudaError_t launch_tc(const BatchArgs& a, cudaStream_t st) {
  const int smem = TcSmem<B, SPLIT>::TOTAL;
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(bsr_tc_kernel<B, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  // at most 8 CTAs per SM (TMEM: 8 x 64 columns = 512), persistent over rows
  const int64_t grid = std::min<int64_t>(a.nrows, 152 * 8);
  if (grid <= 0) return cudaSuccess;
  bsr_tc_kernel<B, SPLIT><<<unsigned(grid), kTcThreads, smem, st>>>(a);
  return launched();
}

cudaError_t bsr_apply_tc(const BatchArgs& a, int b, int prec, cudaStream_t st) {
  if (a.R < 1 || a.R > kTcM) return cudaErrorInvalidValue;
  const bool split = prec == P_FP32;
  if (!split && prec != P_BF16) return cudaErrorInvalidValue;
  switch (b) {
    case 16: return split ? launch_tc<16, true>(a, st) : launch_tc<16, false>(a, st);
    case 64: return split ? launch_tc<64, true>(a, st) : launch_tc<64, false>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ldgmg
