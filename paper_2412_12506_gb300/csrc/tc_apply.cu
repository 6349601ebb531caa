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
// A_lo x_lo is below 2^-16 of the result): both factors then carry about 17
// significant bits (|x - x_hi - x_lo| <= 2^-18 |x|), between BF16 (8) and
// FP32 (24), with FP32 accumulation.
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
#include <mutex>

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

// One potentially blocking test of an mbarrier phase; the suspend-time hint
// caps each call at about 1 us, so kSpinLimit calls bound a wait to ~1 s.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
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

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 1D bulk copy global -> shared, completion counted on `bar` (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// bounded wait on an mbarrier phase; returns false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity))
    if (++spins > kSpinLimit) return false;
  return true;
}

__host__ __device__ __forceinline__ uint32_t round128(uint32_t x) { return (x + 127u) & ~127u; }

// Shared-memory plan of one CTA for b = B, R right-hand sides.
template <int B, bool SPLIT>
struct TcPlan {
  static constexpr int KQ = B / 8;
  static constexpr uint32_t A_BYTES = kTcM * B * 2;             // one BF16 part of X^T
  static constexpr uint32_t B_BYTES = B * B * 2;                // one BF16 part of A_ij
  static constexpr uint32_t OP_BYTES = 2 * A_BYTES + (SPLIT ? 2 : 1) * B_BYTES;
  static constexpr uint32_t RAWA_BYTES = B * B * (SPLIT ? 4 : 2);
  __host__ __device__ static uint32_t rawx_bytes(int R) { return round128(uint32_t(R) * B * 4); }
  __host__ __device__ static uint32_t total(int R) {
    return 2 * OP_BYTES + 2 * RAWA_BYTES + 2 * rawx_bytes(R) + 128;
  }
};

// Software pipeline over the flattened sequence of (block row, block) items of
// this CTA: thread 0 keeps the raw X_j slab and matrix block of the next two
// items in flight with bulk copies (raw buffers 0/1), all threads convert the
// current item into BF16 core-matrix operands (operand buffers 0/1) while the
// tensor cores still work on the previous item, and thread 0 issues the MMAs.
template <int B, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads) bsr_tc_kernel(BatchArgs a) {
  static_assert(B == 16 || B == 64, "tensor-core path supports b = 16 and b = 64");
  typedef TcPlan<B, SPLIT> P;
  constexpr int KQ = P::KQ;
  constexpr int KSTEPS = B / 16;
  constexpr uint32_t NCOLS = B < 32 ? 32 : B;
  constexpr uint32_t IDESC = make_idesc(kTcM, B);
  constexpr uint32_t SBO = KQ * 128;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int R = a.R;
  const uint32_t rawx_bytes = P::rawx_bytes(R);
  // operand buffer bf at smem + bf*OP_BYTES; raw buffers after them
  auto op = [&](int bf) { return smem + bf * P::OP_BYTES; };
  auto rawa = [&](int bf) { return smem + 2 * P::OP_BYTES + bf * P::RAWA_BYTES; };
  auto rawx = [&](int bf) { return smem + 2 * P::OP_BYTES + 2 * P::RAWA_BYTES + bf * rawx_bytes; };
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P::total(R) - 128);   // full[0..1], mma[2..3]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // rows of absent right-hand sides stay zero in both operand buffers
  for (int t = tid; t < kTcM * KQ; t += kTcThreads) {
    const int m = t / KQ, kq = t % KQ;
    if (m >= R)
      for (int bf = 0; bf < 2; ++bf) {
        *reinterpret_cast<uint4*>(op(bf) + core_off(m, kq, KQ)) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(op(bf) + P::A_BYTES + core_off(m, kq, KQ)) = make_uint4(0, 0, 0, 0);
      }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(bars + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // lookahead iterator over items (only thread 0 advances it)
  int64_t la_row = blockIdx.x;
  int la_nz = 0, la_z1 = 0;
  if (la_row < a.nrows) { la_nz = a.row_ptr[la_row]; la_z1 = a.row_ptr[la_row + 1]; }
  auto la_skip_empty = [&]() {
    while (la_row < a.nrows && la_nz >= la_z1) {
      la_row += gridDim.x;
      if (la_row < a.nrows) { la_nz = a.row_ptr[la_row]; la_z1 = a.row_ptr[la_row + 1]; }
    }
  };
  const uint32_t item_bytes = uint32_t(R) * B * 4 + P::RAWA_BYTES;
  auto issue = [&](int bf) {     // thread 0: copies of the lookahead item into raw buffer bf
    la_skip_empty();
    if (la_row >= a.nrows) return false;
    const int64_t j = a.col[la_nz];
    mbar_arrive_expect_tx(bars + bf, item_bytes);
    bulk_g2s(rawx(bf), a.x + j * a.es, uint32_t(R) * B * 4, bars + bf);
    bulk_g2s(rawa(bf), static_cast<const unsigned char*>(a.vals) + int64_t(la_nz) * P::RAWA_BYTES, P::RAWA_BYTES,
             bars + bf);
    ++la_nz;
    return true;
  };
  int issued = 0;                // items whose copies were issued (thread 0's count)
  if (tid == 0) {
    if (issue(0)) ++issued;
    if (issue(1)) ++issued;
  }

  // per buffer: bit bf of fph / mph = phase parity to wait for; bit bf of pend = MMA outstanding
  uint32_t fph = 0, mph = 0, pend = 0;
  int consumed = 0;              // items converted so far
  bool timed_out = false;

  for (int64_t row = blockIdx.x; row < a.nrows && !timed_out; row += gridDim.x) {
    const int z0 = a.row_ptr[row], z1 = a.row_ptr[row + 1];
    for (int nz = z0; nz < z1; ++nz) {
      const int bf = consumed & 1;
      bool ok = mbar_wait_bounded(bars + bf, (fph >> bf) & 1u);                        // raw data of this item
      if (ok && ((pend >> bf) & 1u)) ok = mbar_wait_bounded(bars + 2 + bf, (mph >> bf) & 1u);   // operands free
      if (__syncthreads_or(!ok)) { timed_out = true; break; }
      fph ^= 1u << bf;
      if ((pend >> bf) & 1u) { mph ^= 1u << bf; pend &= ~(1u << bf); }
      // convert: X_j^T -> hi/lo BF16 (A operand), A_ij -> BF16 (hi [, lo]) (B operand)
      unsigned char* o = op(bf);
      const float* xr = reinterpret_cast<const float*>(rawx(bf));
      // one float4 (4 modes of one right-hand side) per thread: consecutive
      // 16-byte reads, 8-byte stores that tile the core matrices without conflicts
      for (int t = tid; t < R * (B / 4); t += kTcThreads) {
        const int m = t / (B / 4), q4 = t % (B / 4);
        const float4 v = *reinterpret_cast<const float4*>(xr + m * B + q4 * 4);
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
        const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
        const uint32_t off = core_off(m, q4 >> 1, KQ) + (q4 & 1) * 8;
        *reinterpret_cast<uint2*>(o + off) =
            make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
        *reinterpret_cast<uint2*>(o + P::A_BYTES + off) =
            make_uint2(pack_bf16(v.x - f0.x, v.y - f0.y), pack_bf16(v.z - f1.x, v.w - f1.y));
      }
      unsigned char* bo = o + 2 * P::A_BYTES;
      if (!SPLIT) {
        const uint4* ra = reinterpret_cast<const uint4*>(rawa(bf));
        for (int t = tid; t < B * KQ; t += kTcThreads) {
          const int r = t / KQ, kq = t % KQ;
          *reinterpret_cast<uint4*>(bo + core_off(r, kq, KQ)) = ra[t];
        }
      } else {
        const float4* ra = reinterpret_cast<const float4*>(rawa(bf));
        for (int t = tid; t < B * (B / 4); t += kTcThreads) {
          const int r = t / (B / 4), q4 = t % (B / 4);
          const float4 v = ra[t];
          const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
          const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
          const uint32_t off = core_off(r, q4 >> 1, KQ) + (q4 & 1) * 8;
          *reinterpret_cast<uint2*>(bo + off) =
              make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
          *reinterpret_cast<uint2*>(bo + P::B_BYTES + off) =
              make_uint2(pack_bf16(v.x - f0.x, v.y - f0.y), pack_bf16(v.z - f1.x, v.w - f1.y));
        }
      }
      fence_proxy_async();     // operands visible to the tensor cores; raw reads ordered before new copies
      __syncthreads();
      if (tid == 0) {
        if (issue(bf)) ++issued;                         // raw buffer bf is free again
        tc_fence_after();
        const uint32_t sa = smem_u32(o), sbh = smem_u32(bo);
#pragma unroll
        for (int s = 0; s < KSTEPS; ++s) {
          const uint64_t ah = make_sdesc(sa + 256u * s, 128u, SBO);
          const uint64_t bd = make_sdesc(sbh + 256u * s, 128u, SBO);
          mma_bf16(tmem, ah, bd, IDESC, (nz > z0 || s > 0) ? 1u : 0u);
          mma_bf16(tmem, make_sdesc(sa + P::A_BYTES + 256u * s, 128u, SBO), bd, IDESC, 1u);
          if (SPLIT) mma_bf16(tmem, ah, make_sdesc(sbh + P::B_BYTES + 256u * s, 128u, SBO), IDESC, 1u);
        }
        mma_commit(bars + 2 + bf);
      }
      pend |= 1u << bf;
      ++consumed;
    }
    if (timed_out) break;
    // the row's products are complete once both operand buffers' MMAs are
    bool ok = true;
    if (ok && (pend & 1u)) ok = mbar_wait_bounded(bars + 2, mph & 1u);
    if (ok && (pend & 2u)) ok = mbar_wait_bounded(bars + 3, (mph >> 1) & 1u);
    if (__syncthreads_or(!ok)) { timed_out = true; break; }
    mph ^= pend;
    pend = 0;
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
            const float sv = empty ? 0.0f : acc[q + e];
            float out;
            switch (a.mode) {
              case M_Y: out = sv; break;
              case M_RES: out = a.rhs[o + q + e] - sv; break;
              case M_AXPY: out = a.xin[o + q + e] + float(a.s) * sv; break;
              default: out = float(a.s) * sv; break;
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
    // bounded drain of this CTA's own copies and MMAs before TMEM and shared memory go away
    if (tid == 0) {
      for (int k = consumed; k < issued; ++k) {
        const int bf = k & 1;
        mbar_wait_bounded(bars + bf, (fph >> bf) & 1u);
        fph ^= 1u << bf;
      }
      if (pend & 1u) mbar_wait_bounded(bars + 2, mph & 1u);
      if (pend & 2u) mbar_wait_bounded(bars + 3, (mph >> 1) & 1u);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// Self-test of the bounded-wait error path: one thread waits on an mbarrier
// that nothing arrives on, with the same bounded spin as the tensor-core
// kernel; when the spin limit runs out it records the timeout and returns.
__global__ void bounded_wait_probe_kernel(int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait_bounded(&bar, 0u)) *err = 1;
  }
}

}  // namespace

cudaError_t bounded_wait_probe(int* err, cudaStream_t st) {
  bounded_wait_probe_kernel<<<1, 32, 0, st>>>(err);
  return launched();
}

bool tc_block_size_supported(int b) { return b == 16 || b == 64; }

// resident CTAs per SM from the kernel's own needs: shared memory (227 KB
// per SM, ~1 KB reserved per CTA), TMEM (512 columns), threads (2048)
template <int B, bool SPLIT>
static int max_ctas(int R) {
  typedef TcPlan<B, SPLIT> P;
  const int smem = int(P::total(R));
  const int by_smem = (227 * 1024) / (smem + 1024);
  const int by_tmem = 512 / (B < 32 ? 32 : B);
  const int by_threads = 2048 / kTcThreads;
  return std::max(1, std::min(by_smem, std::min(by_tmem, by_threads)));
}

int tc_max_ctas_per_sm(int b, int prec, int R) {
  const bool split = prec == P_FP32;
  if (b == 16) return split ? max_ctas<16, true>(R) : max_ctas<16, false>(R);
  if (b == 64) return split ? max_ctas<64, true>(R) : max_ctas<64, false>(R);
  return 0;
}

template <int B, bool SPLIT>
static cudaError_t launch_tc(const BatchArgs& a, cudaStream_t st) {
  typedef TcPlan<B, SPLIT> P;
  const int smem = int(P::total(a.R));
  static std::once_flag once;
  static cudaError_t cfg = cudaSuccess;
  std::call_once(once, [] {
    cfg = cudaFuncSetAttribute(bsr_tc_kernel<B, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(P::total(kTcM)));
  });
  if (cfg != cudaSuccess) return cfg;
  const int fit = max_ctas<B, SPLIT>(a.R);
  const int per_sm = a.ctas_per_sm > 0 ? std::min(a.ctas_per_sm, fit) : fit;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = std::min<int64_t>(a.nrows, int64_t(std::max(sms, 1)) * per_sm);
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
