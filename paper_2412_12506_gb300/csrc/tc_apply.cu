// Batched-RHS block-row apply on the 5th-generation tensor cores (tcgen05).
//
// For R right-hand sides the element-block apply of Sec. 2.3 becomes, per
// block row i,  Y_i^T (R x b) = sum_j X_j^T (R x b) * A_ij^T (b x b),  a
// chain of dense contractions.  Each is issued as tcgen05.mma kind::f16 with
//   M = 128 (right-hand sides; rows >= R are zero),  N = b,  K = 16 per step,
// BF16 operands and an FP32 accumulator in tensor memory.  The FP32 vectors
// are split into hi + lo BF16 parts (hi = bf16(x), lo = bf16(x - hi)) and both
// are multiplied, so x enters with ~17 significant bits (|x - hi - lo| <=
// 2^-17 |x|); with BF16-stored blocks (8 bits) the block rounding dominates,
// as on the CUDA-core path that multiplies them by FP32 vectors.  FP32-stored
// blocks are split the same way (at setup) and three products are accumulated
// (A_hi x_hi + A_hi x_lo + A_lo x_hi; A_lo x_lo is below 2^-16 of the
// result): both factors then carry about 17 significant bits, between BF16
// (8) and FP32 (24), with FP32 accumulation.
//
// Operands live in shared memory in the canonical K-major, no-swizzle
// layout: 8-row x 16-byte core matrices, rows 16 B apart, core matrices
// adjacent in K 128 B apart (LBO) and adjacent in M/N (b/8)*128 B apart
// (SBO).  Both factors arrive in HBM already as these operand images: the
// matrix blocks since setup (FP32 blocks as hi and lo images), the vector
// from split_x_images, a streaming pass that splits X into hi / lo once per
// apply instead of once per use (each X_j is used by ~5 block rows).  So the
// apply moves bytes and issues MMAs; no thread touches an operand.
//
// One CTA has three roles that hand work on through mbarriers only (no CTA
// barrier inside the loop):
//   warp 0 (one thread)   bulk-copies the X_j hi / lo images and the A_ij
//                         image(s) of each (block row, block) item into a
//                         ring of stages;
//   warp 1 (one thread)   issues the MMAs of an item once its stage has
//                         landed, commits the stage back to the copier, and
//                         at the end of a block row commits the row's
//                         accumulator (two accumulators in TMEM alternate);
//   warps 2..5            read a finished accumulator from TMEM (warp w:
//                         lanes 32*(w%4)..+31, one right-hand side per lane)
//                         and apply the fused epilogue while the MMAs of the
//                         next block row run.
// Every wait is bounded; a role that gives up raises the CTA's abort flag,
// the others see it in their own waits, and the CTA drains its own copies
// and MMAs (bounded) before it frees TMEM and exits with the error flag set.
#include "kernels.h"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

namespace ldgmg {

namespace {

using namespace tcptx;

constexpr int kTcM = 128;
constexpr int kEpiThreads = 128;                    // warps 2..5: epilogue
constexpr int kTcThreads = 64 + kEpiThreads;        // + copy warp 0 and MMA warp 1
constexpr uint32_t kCtrlBytes = 256;                // 20 mbarriers, TMEM address, abort flag
constexpr uint32_t kSmemCap = 227 * 1024;           // dynamic shared memory per CTA

// Shared-memory plan of one CTA for b = B: NS stages, each
//   [X hi | X lo (BF16, M = 128 rows each; rows >= R_8 stay zero) | A_ij image(s)]
// then the control words (mbarriers, TMEM address, abort flag).  b = 16 CTAs
// are sized so that four fit on an SM.
template <int B, bool SPLIT>
struct TcPlan {
  static constexpr int KQ = B / 8;
  static constexpr int kMaxStages = 8;
  static constexpr uint32_t OPX_BYTES = kTcM * B * 2;                  // one BF16 part of X^T (M = 128 rows)
  static constexpr uint32_t IMG1 = B * B * 2;                          // one BF16 image of A_ij
  static constexpr uint32_t IMG_BYTES = IMG1 * (SPLIT ? 2 : 1);        // as stored in HBM
  static constexpr uint32_t STAGE = 2 * OPX_BYTES + ((IMG_BYTES + 127u) & ~127u);
  static constexpr uint32_t BUDGET = B == 16 ? kSmemCap / 4 - 1024 : kSmemCap - 1024;
  static constexpr int NS_FIT = int((BUDGET - kCtrlBytes) / STAGE);
  static constexpr int NS = NS_FIT < 2 ? 2 : (NS_FIT > kMaxStages ? kMaxStages : NS_FIT);
  static constexpr uint32_t TOTAL = NS * STAGE + kCtrlBytes;
  static_assert(TOTAL <= kSmemCap - 1024, "stages exceed the dynamic shared memory of a CTA");
  static_assert(STAGE % 128 == 0 && OPX_BYTES % 128 == 0, "stage parts must stay 128-byte aligned");
  static_assert((2 * kMaxStages + 4) * 8 <= 224, "mbarriers would overlap the TMEM address word");
};

// The rows of one CTA (blockIdx.x, + gridDim.x, ...) with the extent of the
// current row and, already loaded, of the next one: the row_ptr loads of a
// row are in flight while the previous row is processed.
struct RowCursor {
  int64_t row;
  int z0 = 0, z1 = 0, n0 = 0, n1 = 0;
  __device__ __forceinline__ RowCursor(const BatchArgs& a, int64_t first) : row(first) {
    if (row < a.nrows) { z0 = a.row_ptr[row]; z1 = a.row_ptr[row + 1]; }
    fetch_next(a);
  }
  __device__ __forceinline__ void fetch_next(const BatchArgs& a) {
    const int64_t nr = row + gridDim.x;
    n0 = n1 = 0;
    if (nr < a.nrows) { n0 = a.row_ptr[nr]; n1 = a.row_ptr[nr + 1]; }
  }
  __device__ __forceinline__ void advance(const BatchArgs& a) {
    row += gridDim.x;
    z0 = n0;
    z1 = n1;
    fetch_next(a);
  }
};

// ring position: stage index and the parity of its current use
struct Ring {
  int s = 0;
  uint32_t ph = 0;
  __device__ __forceinline__ void next(int n) {
    if (++s == n) { s = 0; ph ^= 1u; }
  }
};

template <int B, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads) bsr_tc_kernel(BatchArgs a) {
  static_assert(B == 16 || B == 64, "tensor-core path supports b = 16 and b = 64");
  typedef TcPlan<B, SPLIT> P;
  constexpr int KQ = P::KQ;
  constexpr int NS = P::NS;
  constexpr int KSTEPS = B / 16;
  constexpr uint32_t NACC = B < 32 ? 32 : B;     // TMEM columns of one accumulator
  constexpr uint32_t NCOLS = 2 * NACC;
  constexpr uint32_t IDESC = make_idesc(kTcM, B);
  constexpr uint32_t SBO = KQ * 128;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int R = a.R;
  const int R8 = (R + 7) & ~7;
  const uint32_t xi_bytes = uint32_t(R8) * B * 2;          // one image of X_j (hi or lo)
  auto opx = [&](int s) { return smem + s * P::STAGE; };                     // X hi; X lo at + OPX_BYTES
  auto img = [&](int s) { return smem + s * P::STAGE + 2 * P::OPX_BYTES; };
  unsigned char* ctrl = smem + NS * P::STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(ctrl);     // stage landed (transaction count)
  uint64_t* empty = full + P::kMaxStages;                   // the stage's MMAs complete (commit)
  uint64_t* accfull = empty + P::kMaxStages;                // a block row's products complete (commit)
  uint64_t* accempty = accfull + 2;                         // accumulator read out (kEpiThreads arrivals)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctrl + 224);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctrl + 228);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // rows the copies never write (>= R_8) stay zero in every stage's X operand
  for (int t = tid; t < NS * kTcM * KQ; t += kTcThreads) {
    const int s = t / (kTcM * KQ), e = t % (kTcM * KQ);
    const int m = e / KQ, kq = e % KQ;
    if (m >= R8) {
      *reinterpret_cast<uint4*>(opx(s) + core_off(m, kq, KQ)) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(opx(s) + P::OPX_BYTES + core_off(m, kq, KQ)) = make_uint4(0, 0, 0, 0);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < P::kMaxStages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(accfull + i, 1);
      mbar_init(accempty + i, kEpiThreads);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---- copier: item k goes to stage k % NS once the MMAs of item k - NS are done
    if (lane == 0) {
      const unsigned char* xim = static_cast<const unsigned char*>(a.ximg);
      int64_t k = 0;
      Ring r;
      bool ok = true;
      RowCursor rc(a, blockIdx.x);
      int col0 = rc.z0 < rc.z1 ? a.col[rc.z0] : 0;
      for (; rc.row < a.nrows && ok; rc.advance(a)) {
        const int z0 = rc.z0, z1 = rc.z1;
        // the next row's extent is in flight (RowCursor); fetch its first block column early too
        const int ncol0 = rc.n0 < rc.n1 ? a.col[rc.n0] : 0;
        for (int nz = z0; nz < z1; ++nz, ++k) {
          if (k >= NS && !wait_or_abort(empty + r.s, r.ph ^ 1u, abort_flag, a.err)) { ok = false; break; }
          const int j = nz == z0 ? col0 : a.col[nz];
          const unsigned char* xj = xim + int64_t(j) * 2 * xi_bytes;
          mbar_arrive_expect_tx(full + r.s, 2 * xi_bytes + P::IMG_BYTES);
          bulk_g2s(opx(r.s), xj, xi_bytes, full + r.s);
          bulk_g2s(opx(r.s) + P::OPX_BYTES, xj + xi_bytes, xi_bytes, full + r.s);
          bulk_g2s(img(r.s), static_cast<const unsigned char*>(a.vals) + int64_t(nz) * P::IMG_BYTES, P::IMG_BYTES,
                   full + r.s);
          r.next(NS);
        }
        col0 = ncol0;
      }
      if (!ok || *abort_flag) {
        // bounded drain of this CTA's copies in flight before shared memory goes away
        for (int s = 0; s < NS && s < k; ++s) {
          const int64_t cnt = k / NS + (s < k % NS ? 1 : 0);     // copies issued into stage s
          mbar_wait_bounded(full + s, uint32_t(cnt - 1) & 1u);
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: Y_i^T += X_j^T A_ij^T per item, accumulator t % 2 for the t-th non-empty row
    if (lane == 0) {
      int64_t t = 0;
      Ring r, last;
      bool ok = true, any = false;
      for (RowCursor rc(a, blockIdx.x); rc.row < a.nrows && ok; rc.advance(a)) {
        const int z0 = rc.z0, z1 = rc.z1;
        if (z0 == z1) continue;
        const int acc = int(t & 1);
        if (t >= 2 && !wait_or_abort(accempty + acc, uint32_t((t >> 1) - 1) & 1u, abort_flag, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(acc) * NACC;
        for (int nz = z0; nz < z1; ++nz) {
          if (!wait_or_abort(full + r.s, r.ph, abort_flag, a.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(opx(r.s)), sb = smem_u32(img(r.s));
#pragma unroll
          for (int ks = 0; ks < KSTEPS; ++ks) {
            const uint64_t ah = make_sdesc(sa + 256u * ks, 128u, SBO);
            const uint64_t bd = make_sdesc(sb + 256u * ks, 128u, SBO);
            mma_bf16(d, ah, bd, IDESC, (nz > z0 || ks > 0) ? 1u : 0u);
            mma_bf16(d, make_sdesc(sa + P::OPX_BYTES + 256u * ks, 128u, SBO), bd, IDESC, 1u);
            if (SPLIT) mma_bf16(d, ah, make_sdesc(sb + P::IMG1 + 256u * ks, 128u, SBO), IDESC, 1u);
          }
          mma_commit(empty + r.s);
          last = r;
          any = true;
          r.next(NS);
        }
        if (!ok) break;
        mma_commit(accfull + acc);
        ++t;
      }
      // after giving up: bounded wait for the MMAs already issued (the last commit covers them)
      if (!ok && any) mbar_wait_bounded(empty + last.s, last.ph);
    }
  } else {
    // ---- epilogue (warps 2..5)
    const int quad = warp & 3;                 // the TMEM lane quarter this warp may read
    const int m = quad * 32 + lane;            // this thread's right-hand side
    int64_t t = 0;
    for (RowCursor rc(a, blockIdx.x); rc.row < a.nrows; rc.advance(a)) {
      const int64_t row = rc.row;
      const bool empty_row = rc.z0 == rc.z1;
      const int acc = int(t & 1);
      if (!empty_row) {
        const bool w = wait_or_abort(accfull + acc, uint32_t(t >> 1) & 1u, abort_flag, a.err);
        if (__any_sync(0xffffffffu, !w)) break;
        tc_fence_after();
      }
#pragma unroll
      for (int c0 = 0; c0 < B; c0 += 16) {
        float v[16];
        if (!empty_row) {
          tmem_ld16(tmem + (uint32_t(quad * 32) << 16) + uint32_t(acc) * NACC + uint32_t(c0), v);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = 0.0f;
        }
        if (m < R) {
          const int64_t o = row * a.es + int64_t(m) * a.rs + c0;
          const float sc = float(a.s);
#pragma unroll
          for (int q = 0; q < 16; q += 4) {
            float4 y = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            if (a.mode == M_RES) {
              const float4 rr = *reinterpret_cast<const float4*>(a.rhs + o + q);
              y = make_float4(rr.x - y.x, rr.y - y.y, rr.z - y.z, rr.w - y.w);
            } else if (a.mode == M_AXPY) {
              const float4 xi = *reinterpret_cast<const float4*>(a.xin + o + q);
              y = make_float4(xi.x + sc * y.x, xi.y + sc * y.y, xi.z + sc * y.z, xi.w + sc * y.w);
            } else if (a.mode != M_Y) {
              y = make_float4(sc * y.x, sc * y.y, sc * y.z, sc * y.w);
            }
            *reinterpret_cast<float4*>(a.y + o + q) = y;
          }
        }
      }
      if (!empty_row) {
        tc_fence_before();
        mbar_arrive(accempty + acc);
        ++t;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
  }
}

// X ([element][rhs][mode], FP32) -> per element the hi and lo BF16 operand
// images; one thread per (element, right-hand side row, 8 modes): a 32-byte
// read and two 16-byte writes (consecutive threads: consecutive reads, and
// writes that tile 512-byte runs of the images).
template <int B>
__global__ void split_x_kernel(const float* __restrict__ x, uint32_t units, int R, int R8,
                               unsigned char* __restrict__ ximg) {
  constexpr int KQ = B / 8;
  const uint32_t per = uint32_t(R8) * KQ;
  const uint32_t xi = uint32_t(R8) * B * 2;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < units; t += gridDim.x * blockDim.x) {
    const uint32_t j = t / per, u = t % per;
    const int m = int(u / KQ), kq = int(u % KQ);
    uint4 hi = make_uint4(0, 0, 0, 0), lo = make_uint4(0, 0, 0, 0);
    if (m < R) {
      const float4* src = reinterpret_cast<const float4*>(x + (int64_t(j) * R + m) * B + kq * 8);
      const float4 v0 = src[0], v1 = src[1];
      const float f[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
      uint32_t h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(f[2 * q], f[2 * q + 1]);
        const float2 hf = __bfloat1622float2(hb);
        h[q] = *reinterpret_cast<const uint32_t*>(&hb);
        l[q] = pack_bf16(f[2 * q] - hf.x, f[2 * q + 1] - hf.y);
      }
      hi = make_uint4(h[0], h[1], h[2], h[3]);
      lo = make_uint4(l[0], l[1], l[2], l[3]);
    }
    unsigned char* dst = ximg + int64_t(j) * 2 * xi + core_off(m, kq, KQ);
    *reinterpret_cast<uint4*>(dst) = hi;
    *reinterpret_cast<uint4*>(dst + xi) = lo;
  }
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

size_t x_image_bytes(int64_t N, int R, int b) { return size_t(N) * size_t((R + 7) & ~7) * size_t(b) * 4; }

cudaError_t split_x_images(const float* x, int64_t N, int R, int b, void* ximg, cudaStream_t st) {
  if (R < 1 || R > kTcM || N < 0 || !tc_block_size_supported(b)) return cudaErrorInvalidValue;
  const int R8 = (R + 7) & ~7;
  const int64_t units = N * R8 * (b / 8);
  if (units == 0) return cudaSuccess;
  if (units >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
  const int grid = int(std::min<int64_t>((units + 255) / 256, 152 * 16));
  if (b == 16) split_x_kernel<16><<<grid, 256, 0, st>>>(x, uint32_t(units), R, R8, static_cast<unsigned char*>(ximg));
  else split_x_kernel<64><<<grid, 256, 0, st>>>(x, uint32_t(units), R, R8, static_cast<unsigned char*>(ximg));
  return launched();
}

// resident CTAs per SM from the kernel's own needs: shared memory (227 KB
// per SM, ~1 KB reserved per CTA), TMEM (512 columns), threads (2048)
template <int B, bool SPLIT>
static int max_ctas() {
  typedef TcPlan<B, SPLIT> P;
  const int by_smem = int(kSmemCap) / int(P::TOTAL + 1024);
  const int by_tmem = 512 / (2 * (B < 32 ? 32 : B));
  const int by_threads = 2048 / kTcThreads;
  return std::max(1, std::min(by_smem, std::min(by_tmem, by_threads)));
}

int tc_max_ctas_per_sm(int b, int prec, int R) {
  (void)R;
  const bool split = prec == P_FP32;
  if (b == 16) return split ? max_ctas<16, true>() : max_ctas<16, false>();
  if (b == 64) return split ? max_ctas<64, true>() : max_ctas<64, false>();
  return 0;
}

template <int B, bool SPLIT>
static cudaError_t launch_tc(const BatchArgs& a, cudaStream_t st) {
  typedef TcPlan<B, SPLIT> P;
  static std::once_flag once;
  static cudaError_t cfg = cudaSuccess;
  std::call_once(once, [] {
    cfg = cudaFuncSetAttribute(bsr_tc_kernel<B, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(P::TOTAL));
  });
  if (cfg != cudaSuccess) return cfg;
  const int fit = max_ctas<B, SPLIT>();
  const int per_sm = a.ctas_per_sm > 0 ? std::min(a.ctas_per_sm, fit) : fit;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = std::min<int64_t>(a.nrows, int64_t(std::max(sms, 1)) * per_sm);
  if (grid <= 0) return cudaSuccess;
  bsr_tc_kernel<B, SPLIT><<<unsigned(grid), kTcThreads, P::TOTAL, st>>>(a);
  return launched();
}

cudaError_t bsr_apply_tc(const BatchArgs& a, int b, int prec, cudaStream_t st) {
  if (a.R < 1 || a.R > kTcM || !a.ximg) return cudaErrorInvalidValue;
  const bool split = prec == P_FP32;
  if (!split && prec != P_BF16) return cudaErrorInvalidValue;
  switch (b) {
    case 16: return split ? launch_tc<16, true>(a, st) : launch_tc<16, false>(a, st);
    case 64: return split ? launch_tc<64, true>(a, st) : launch_tc<64, false>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ldgmg
