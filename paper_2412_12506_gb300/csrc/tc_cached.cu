// Batched-RHS block-row apply on the tensor cores with a shared-memory cache
// of converted x operands (2D meshes, b = 16: the p = 3 interface workloads).
//
// Y_i^T (R x b) = sum_j X_j^T A_ij^T per block row (R <= 64 right-hand sides),
// with FP32 x and A split into BF16 hi + lo parts as in tc_apply.cu, but laid
// out so that one tcgen05.mma per block does all the products and so that x
// is read from HBM about once:
//   * One MMA per block, M = 128, K = 16: the A operand is the x_j slot, 128
//     rows holding the hi and the lo part of each right-hand side (right-hand
//     side m: hi in row 8 (m / 4) + m % 4, lo four rows below); the B operand
//     is the block's stored image pair [A_hi | A_lo] read as one N = 32
//     operand (N = 16, A_hi alone, for BF16 storage).  The accumulator then
//     holds x_hi A_hi, x_hi A_lo, x_lo A_hi and x_lo A_lo in separate lanes and
//     columns; the epilogue adds them (columns, then lanes rho and rho ^ 4 by
//     a shuffle).  Against three MMAs of N = 16 per block this cuts the MMA
//     count (the issue-bound part of the per-use kernel) by 3 and adds the
//     lo * lo term.
//   * Rows are processed in strip order: strips of L element columns, each
//     walked along y, so a row's neighbours x_{i +- 1}, x_{i +- n} were mostly
//     needed a few rows earlier.
//   * The CTA keeps S converted x_j in shared-memory slots.  A host-built
//     schedule says, per row, which x_j to load and convert into which slot
//     and which slot each block of the row reads; every x_j is read from HBM
//     about (L + 2) / L times per apply instead of once by a separate split
//     pass plus once per use.
//   * FP32 x_j and the row's A_ij images arrive by bulk async copies into
//     rings of stages.  Two CTAs run on each SM (the tensor core overlaps
//     the MMA streams of different CTAs, not those of one), each taking a
//     contiguous range of the strip order.
// The result of a right-hand side does not depend on the others nor on R.
//
// Warp roles (two CTAs of 480 threads per SM), hand-offs by mbarriers only;
// each of the two copy streams runs as far ahead as its own ring allows:
//   warp 0      copies the row's A blocks with its schedule record;
//   warp 10     copies the raw x_j of the schedule's loads;
//   warp 1      issues the MMAs of every row, all blocks of a row into one of
//               8 TMEM accumulators, and commits the row;
//   warps 2..5  convert raw x_j into the slot the schedule names, once every
//               row that last read that slot has completed (the schedule
//               guarantees that row is at least kLag rows back);
//   warps 6..9, 11..14  read a finished accumulator and apply the fused
//               epilogue (reading the rhs / xin row itself, one row ahead),
//               the first group for even rows, the second for odd.
// Every wait is bounded; a role that gives up raises the CTA's abort flag,
// the others leave their waits, the CTA drains its own copies and MMAs
// (bounded) and exits with the error flag set.
#include "kernels.h"
#include "tc_ptx.cuh"

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace ldgmg {

// One row (step) of a CTA's schedule; 64 bytes, copied into the A and rhs stages.
struct TcStep {
  int32_t row;          // block row (element) in the matrix and in the vectors
  int32_t z0;           // its first stored block
  int32_t ld0;          // its first load in the load list
  uint16_t nnz;         // stored blocks of the row (<= 16)
  uint16_t nld;         // x_j to load and convert before this row (<= nnz)
  uint8_t slot[16];     // slot of x_{col[z0 + t]} for block t
  uint8_t lslot[16];    // slot that load t of this row fills
  uint8_t pad[16];
};
static_assert(sizeof(TcStep) == 64, "step record must be 64 bytes");

namespace {

using namespace tcptx;

constexpr int kB = 16;                  // block size
constexpr int kKQ = kB / 8;             // core matrices along K
constexpr int kMmaM = 128;              // MMA rows: hi and lo parts of 64 right-hand sides
constexpr uint32_t kSlotBytes = kMmaM * kB * 2;   // one x_j operand: 128 rows of 16 BF16
// Two CTAs per SM: the tensor core overlaps the MMA streams of different CTAs
// (one CTA's MMAs into one accumulator run at ~80 cycles each, two CTAs at
// ~40 per SM), so the rings below are sized to fit two CTAs in shared memory.
constexpr int kCtasPerSm = 2;
constexpr int kNS = 5;                  // A stages (shared memory)
constexpr int kND = 16;                 // step-done barriers (> kNAcc, > kLag, >= kNS)
constexpr int kNAcc = 8;                // TMEM accumulators, one per row in flight
constexpr uint32_t kAccCols = 32;       // columns of one accumulator
constexpr uint32_t kTmemCols = 256;     // kNAcc * kAccCols (two CTAs: the whole TMEM)
constexpr int kLag = 2;                 // the converter writes row s's slots after row s - kLag completes
constexpr int kNX = kND;                // x-ready barriers
constexpr int kNRaw = 5;                // raw x_j stages (3: 0.2196 ms, 5: 0.2147, 6: 0.2150, 7: 0.2172 at 256^2)
constexpr int kThreads = 480;
constexpr int kConvThreads = 128;
constexpr int kEpiThreads = 128;
constexpr uint32_t kRecBytes = 64;
constexpr uint32_t kRecPad = 128;       // record slot at the end of a stage (keeps stages 128-byte aligned)
constexpr uint32_t kSmemCap = (228 * 1024) / kCtasPerSm - 1024;   // dynamic shared memory per CTA
constexpr uint32_t kCtrlBytes = 1024;
constexpr int kMaxBlocksPerRow = 16;
static_assert(kLag < kND && kLag < kNX && kNAcc < kND && kNS <= kND && kNAcc % 2 == 0,
              "barrier rings must be deeper than the leads they bound; each epilogue group keeps its accumulators");
static_assert(kNAcc * kAccCols <= kTmemCols && (kTmemCols & (kTmemCols - 1)) == 0, "TMEM allocation");
static_assert((kNS + kND + kNX + kNAcc + 2 * kNRaw) * 8 + 8 <= int(kCtrlBytes), "control words");

struct CachedArgs {
  BatchArgs a;
  const TcStep* rec;     // all steps, CTA c: [seg[c], seg[c + 1])
  const int* seg;
  const int* ld_elem;     // element of every load, in schedule order
  int S;                  // x slots
  int kmax;               // stage room in blocks
  int need_rhs;           // the epilogue reads a.rhs (M_RES) or a.xin (M_AXPY)
  // shared-memory plan (byte offsets)
  uint32_t off_a, off_raw, off_ctrl;
  uint32_t stage_a, raw_bytes;
};

__device__ __forceinline__ uint32_t parity_of(int64_t use, int ring) { return uint32_t(use / ring) & 1u; }

template <bool SPLIT>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) bsr_tc_cached_kernel(CachedArgs ca) {
  constexpr uint32_t IMG1 = kB * kB * 2;
  constexpr uint32_t IMG = IMG1 * (SPLIT ? 2 : 1);
  // N = 32 for FP32 storage: the block's hi and lo images side by side (the
  // stored [hi | lo] image pair is one 32-row K-major operand); N = 16 for BF16
  constexpr uint32_t NB = SPLIT ? 2 * kB : kB;
  constexpr uint32_t IDESC = make_idesc(kMmaM, int(NB));
  constexpr uint32_t SBO = kKQ * 128;
  const BatchArgs& a = ca.a;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int R = a.R;
  const int R8 = (R + 7) & ~7;
  const uint32_t xrow_bytes = uint32_t(R) * kB * 4;       // one element's x (or rhs) for R right-hand sides
  unsigned char* xs = smem;               // S slots of kSlotBytes
  auto astage = [&](int k) { return smem + ca.off_a + uint32_t(k) * ca.stage_a; };
  auto arec = [&](int k) { return reinterpret_cast<const TcStep*>(astage(k) + uint32_t(ca.kmax) * IMG); };
  auto raw = [&](int q) { return reinterpret_cast<const float*>(smem + ca.off_raw + uint32_t(q) * ca.raw_bytes); };
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ca.off_ctrl);   // A stage landed
  uint64_t* done = full + kNS;                                         // row's MMAs complete (commit)
  uint64_t* xready = done + kND;                                       // row's slots written (converters)
  uint64_t* accempty = xready + kNX;                                   // accumulator read (epilogue)
  uint64_t* rawfull = accempty + kNAcc;
  uint64_t* rawempty = rawfull + kNRaw;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(rawempty + kNRaw);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s0 = ca.seg[blockIdx.x], s1 = ca.seg[blockIdx.x + 1];
  const int nsteps = s1 - s0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < kNS; ++i) mbar_init(full + i, 1);
    for (int i = 0; i < kND; ++i) {
      mbar_init(done + i, 1);
      mbar_init(xready + i, kConvThreads);
    }
    for (int i = 0; i < kNAcc; ++i) mbar_init(accempty + i, kEpiThreads);   // one epilogue group per row
    for (int i = 0; i < kNRaw; ++i) {
      mbar_init(rawfull + i, 1);
      mbar_init(rawempty + i, kConvThreads);
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
    // ---- copier.  The whole warp walks the steps (records are read a warp
    // window at a time and broadcast by shuffles); lane 0 waits and issues the
    // copies, and broadcasts the outcome of each wait.
    int64_t nA = 0;                         // A stages issued
    bool ok = true;
    uint32_t w[4] = {0, 0, 0, 0};           // lane l: row, z0, ld0, counts of step wbase + l
    int wbase = s0 - 64;
    auto wait0 = [&](uint64_t* bar, uint32_t par) {
      bool r = true;
      if (lane == 0) r = wait_or_abort(bar, par, abort_flag, a.err);
      return __shfl_sync(0xffffffffu, r ? 1 : 0, 0) != 0;
    };
    for (int s = s0; s < s1 && ok; ++s) {
      if (s - wbase >= 32) {
        wbase = s;
        const int t = s + lane;
        if (t < s1) {
          const uint4 v0 = *reinterpret_cast<const uint4*>(ca.rec + t);
          w[0] = v0.x; w[1] = v0.y; w[2] = v0.z; w[3] = v0.w;
        }
      }
      const int src = s - wbase;
      const int z0 = int(__shfl_sync(0xffffffffu, w[1], src));
      const int nnz = int(__shfl_sync(0xffffffffu, w[3], src) & 0xFFFFu);
      const int i = s - s0;
      // the row's A_ij images and its record (the record also tells the
      // converters which loads precede the row)
      const int ks = i % kNS;
      if (i >= kNS && !wait0(done + ((i - kNS) % kND), parity_of(i - kNS, kND))) { ok = false; break; }
      if (lane == 0) {
        mbar_arrive_expect_tx(full + ks, uint32_t(nnz) * IMG + kRecBytes);
        if (nnz > 0)
          bulk_g2s(astage(ks), static_cast<const unsigned char*>(a.vals) + int64_t(z0) * IMG, uint32_t(nnz) * IMG,
                   full + ks);
        bulk_g2s(astage(ks) + uint32_t(ca.kmax) * IMG, ca.rec + s, kRecBytes, full + ks);
      }
      ++nA;
    }
    __syncwarp();
    if (lane == 0 && (!ok || *abort_flag)) {
      // bounded drain of this CTA's copies in flight before shared memory goes
      // away: the last use of every ring entry
      auto drain = [&](uint64_t* bars, int ring, int64_t n) {
        for (int e = 0; e < ring && e < n; ++e) mbar_wait_bounded(bars + e, parity_of(e + ring * ((n - 1 - e) / ring), ring));
      };
      drain(full, kNS, nA);
    }
  } else if (warp == 10) {
    // ---- raw x copier: the CTA's loads in schedule order into the raw ring
    const int kbeg = nsteps > 0 ? ca.rec[s0].ld0 : 0;
    const int kend = nsteps > 0 ? ca.rec[s1 - 1].ld0 + int(ca.rec[s1 - 1].nld) : 0;
    int64_t nraw = 0;
    bool ok = true;
    int lw = 0;
    for (int kb = kbeg; kb < kend && ok; kb += 32) {
      lw = ca.ld_elem[kb + lane];        // the list is padded by 32 entries
      const int cnt = min(32, kend - kb);
      for (int t = 0; t < cnt; ++t) {
        const int j = __shfl_sync(0xffffffffu, lw, t);
        const int q = int(nraw % kNRaw);
        bool w = true;
        if (lane == 0 && nraw >= kNRaw) w = wait_or_abort(rawempty + q, parity_of(nraw - kNRaw, kNRaw), abort_flag, a.err);
        if (!__shfl_sync(0xffffffffu, w ? 1 : 0, 0)) { ok = false; break; }
        if (lane == 0) {
          mbar_arrive_expect_tx(rawfull + q, xrow_bytes);
          bulk_g2s(smem + ca.off_raw + uint32_t(q) * ca.raw_bytes, a.x + int64_t(j) * a.es, xrow_bytes,
                   rawfull + q);
        }
        ++nraw;
      }
    }
    __syncwarp();
    if (lane == 0 && (!ok || *abort_flag))
      for (int e = 0; e < kNRaw && e < nraw; ++e)
        mbar_wait_bounded(rawfull + e, parity_of(e + kNRaw * ((nraw - 1 - e) / kNRaw), kNRaw));
  } else if (warp == 1) {
    // ---- MMA issuer.  One thread issues every row, all blocks of a row into
    // one accumulator: consecutive MMAs into the same accumulator run at about
    // a third of the cost of MMAs that switch accumulators (measured), so the
    // rows are not interleaved.  The descriptors of slot 0 / stage block 0
    // are built once; a slot or block offset is a multiple of 16 bytes added
    // to the address field.
    bool ok = true;
    int last_done = -1;
    if (lane == 0) {
      const uint64_t dx = make_sdesc(smem_u32(xs), 128u, SBO);
      constexpr uint64_t sunit = kSlotBytes >> 4;
      for (int i = 0; i < nsteps; ++i) {
        const int ks = i % kNS, acc = i % kNAcc;
        // x-ready of row i implies its A stage has landed: the converters
        // waited for that stage (the record) before they arrived
        if (!wait_or_abort(xready + (i % kNX), parity_of(i, kNX), abort_flag, a.err) ||
            (i >= kNAcc && !wait_or_abort(accempty + acc, parity_of(i - kNAcc, kNAcc), abort_flag, a.err))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const TcStep* rc = arec(ks);
        const int nnz = rc->nnz;
        const uint4 sw = *reinterpret_cast<const uint4*>(rc->slot);
        const uint32_t words[4] = {sw.x, sw.y, sw.z, sw.w};
        const uint32_t d = tmem + uint32_t(acc) * kAccCols;
        const uint64_t da = make_sdesc(smem_u32(astage(ks)), 128u, SBO);
        // one MMA per block: [x hi; x lo] (128 rows) times [A hi | A lo]^T
#pragma unroll
        for (int t = 0; t < kMaxBlocksPerRow; ++t) {
          if (t < nnz) {
            const uint64_t sl = (words[t >> 2] >> (8 * (t & 3))) & 0xFFu;
            mma_bf16(d, dx + sl * sunit, da + uint64_t(t) * (IMG >> 4), IDESC, t > 0 ? 1u : 0u);
          }
        }
        mma_commit(done + (i % kND));
        last_done = i;
      }
      // after giving up: bounded wait for the MMAs already issued (the last commit covers them)
      if (!ok && last_done >= 0) mbar_wait_bounded(done + (last_done % kND), parity_of(last_done, kND));
    }
    __syncwarp();
  } else if (warp >= 2 && warp < 6) {
    // ---- converters: raw FP32 x_j -> BF16 hi / lo operand images in its slot
    const int ct = tid - 64;
    int64_t nraw = 0;
    const int units = R8 * kKQ;
    for (int i = 0; i < nsteps; ++i) {
      const int ks = i % kNS;
      if (!wait_or_abort(full + ks, parity_of(i, kNS), abort_flag, a.err)) break;
      const TcStep* rc = arec(ks);
      const int nld = rc->nld;
      // every row <= i - kLag has completed: this wait covers row i - kLag, the
      // waits of the earlier rows cover the rows before it (whichever issuer)
      if (i >= kLag && !wait_or_abort(done + ((i - kLag) % kND), parity_of(i - kLag, kND), abort_flag, a.err)) break;
      bool ok = true;
      for (int t = 0; t < nld; ++t) {
        const int q = int(nraw % kNRaw);
        if (!wait_or_abort(rawfull + q, parity_of(nraw, kNRaw), abort_flag, a.err)) { ok = false; break; }
        const uint32_t sl = rc->lslot[t];
        unsigned char* dsl = xs + sl * kSlotBytes;
        const float* src = raw(q);
        for (int u = ct; u < units; u += kConvThreads) {
          const int m = u / kKQ, kq = u % kKQ;
          uint4 hi = make_uint4(0, 0, 0, 0), lo = make_uint4(0, 0, 0, 0);
          if (m < R) {
            const float4* p = reinterpret_cast<const float4*>(src + m * kB + kq * 8);
            const float4 v0 = p[0], v1 = p[1];
            const float f[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const __nv_bfloat162 hb = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
              const float2 hf = __bfloat1622float2(hb);
              h[e] = *reinterpret_cast<const uint32_t*>(&hb);
              l[e] = pack_bf16(f[2 * e] - hf.x, f[2 * e + 1] - hf.y);
            }
            hi = make_uint4(h[0], h[1], h[2], h[3]);
            lo = make_uint4(l[0], l[1], l[2], l[3]);
          }
          // right-hand side m: hi in row 8 (m / 4) + m % 4, lo four rows below,
          // so both land in the same 8-lane group of the accumulator
          const int rh = 8 * (m >> 2) + (m & 3);
          *reinterpret_cast<uint4*>(dsl + core_off(rh, kq, kKQ)) = hi;
          *reinterpret_cast<uint4*>(dsl + core_off(rh + 4, kq, kKQ)) = lo;
        }
        mbar_arrive(rawempty + q);
        ++nraw;
      }
      if (!ok) break;
      fence_proxy_async();     // the slot writes are read by the tensor cores (async proxy)
      mbar_arrive(xready + (i % kNX));
    }
  } else {
    // ---- epilogue: warps 6..9 take the even rows, warps 11..14 the odd ones;
    // warp w reads TMEM lanes 32 * (w % 4) .. + 31.  Lane rho holds the hi
    // (rho % 8 < 4) or lo part of right-hand side 4 (rho / 8) + rho % 4 in 32
    // columns: 0..15 times A hi, 16..31 (FP32 storage) times A lo.  The two
    // halves add up in the lane, then lanes rho and rho ^ 4.  The rows'
    // records are read a warp window at a time; the rhs / xin row of the
    // group's next row is loaded while the current one is finished.
    const int quad = warp & 3;
    const int rho = quad * 32 + lane;
    const int m = 4 * (rho >> 3) + (rho & 3);  // this lane's right-hand side
    const bool writer = (rho & 4) == 0 && m < R;
    const int egrp = warp < 10 ? 0 : 1;
    const float sc = float(a.s);
    const bool need = ca.need_rhs != 0;
    const float* vsrc = a.mode == M_RES ? a.rhs : a.xin;
    uint32_t wrow = 0, wcnt = 0;               // lane l: row and counts of the group's row kb + l
    int kb = -64;
    auto rec_of = [&](int k, int& row, int& nnz) {      // warp-uniform
      if (k - kb >= 32) {
        kb = k;
        const int t = egrp + 2 * (k + lane);
        if (t < nsteps) {
          const uint4 v = *reinterpret_cast<const uint4*>(ca.rec + s0 + t);
          wrow = v.x;
          wcnt = v.w;
        }
      }
      row = int(__shfl_sync(0xffffffffu, wrow, k - kb));
      nnz = int(__shfl_sync(0xffffffffu, wcnt, k - kb) & 0xFFFFu);
    };
    auto load_row = [&](int row, float4* dst) {
      const float4* src = reinterpret_cast<const float4*>(vsrc + int64_t(row) * a.es + int64_t(m) * a.rs);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = src[q];
    };
    float4 cur[4], nxt[4];
    int row_c = 0, nnz_c = 0;
    if (egrp < nsteps) {
      rec_of(0, row_c, nnz_c);
      if (need && writer) load_row(row_c, cur);
    }
    for (int i = egrp, k = 0; i < nsteps; i += 2, ++k) {
      const int kd = i % kND, acc = i % kNAcc;
      int row_n = 0, nnz_n = 0;
      if (i + 2 < nsteps) {
        rec_of(k + 1, row_n, nnz_n);
        if (need && writer) load_row(row_n, nxt);
      }
      const bool w = wait_or_abort(done + kd, parity_of(i, kND), abort_flag, a.err);
      if (__any_sync(0xffffffffu, !w)) break;
      tc_fence_after();
      float v[16];
      if (nnz_c > 0) {
        const uint32_t ta = tmem + (uint32_t(quad * 32) << 16) + uint32_t(acc) * kAccCols;
        tmem_ld16(ta, v);
        if (SPLIT) {
          float w2[16];
          tmem_ld16(ta + 16u, w2);
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] += w2[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = 0.0f;
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] += __shfl_xor_sync(0xffffffffu, v[e], 4);
      if (writer) {
        float4* yo = reinterpret_cast<float4*>(a.y + int64_t(row_c) * a.es + int64_t(m) * a.rs);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float4 y = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          if (a.mode == M_RES) {
            const float4 r4 = cur[q];
            y = make_float4(r4.x - y.x, r4.y - y.y, r4.z - y.z, r4.w - y.w);
          } else if (a.mode == M_AXPY) {
            const float4 xi = cur[q];
            y = make_float4(xi.x + sc * y.x, xi.y + sc * y.y, xi.z + sc * y.z, xi.w + sc * y.w);
          } else if (a.mode != M_Y) {
            y = make_float4(sc * y.x, sc * y.y, sc * y.z, sc * y.w);
          }
          yo[q] = y;
        }
      }
      tc_fence_before();
      mbar_arrive(accempty + acc);
#pragma unroll
      for (int q = 0; q < 4; ++q) cur[q] = nxt[q];
      row_c = row_n;
      nnz_c = nnz_n;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// Shared-memory plan of one CTA for R right-hand sides, kmax blocks per row
// and S x slots (byte offsets into the dynamic shared memory).
struct CachedPlan {
  uint32_t off_a, stage_a, off_raw, raw_bytes, off_ctrl, total;
};

CachedPlan cached_plan(int R, int kmax, bool split, int S) {
  CachedPlan p{};
  const uint32_t img = kB * kB * 2 * (split ? 2 : 1);
  auto up = [](uint32_t v) { return (v + 127u) & ~127u; };
  p.off_a = uint32_t(S) * kSlotBytes;                           // the x slots
  p.stage_a = uint32_t(kmax) * img + kRecPad;
  p.off_raw = p.off_a + kNS * p.stage_a;
  p.raw_bytes = up(uint32_t(R) * kB * 4);
  p.off_ctrl = p.off_raw + kNRaw * p.raw_bytes;
  p.total = p.off_ctrl + kCtrlBytes;
  return p;
}

// most x slots that fit for (R, kmax)
int cached_slots(int R, int kmax, bool split) {
  int S = 0;
  while (S < 255 && cached_plan(R, kmax, split, S + 1).total <= kSmemCap) ++S;
  return S;
}

template <bool SPLIT>
cudaError_t launch_cached(const CachedArgs& ca, uint32_t smem, int grid, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t cfg = cudaSuccess;
  std::call_once(once, [] {
    cfg = cudaFuncSetAttribute(bsr_tc_cached_kernel<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(kSmemCap));
  });
  if (cfg != cudaSuccess) return cfg;
  bsr_tc_cached_kernel<SPLIT><<<unsigned(grid), kThreads, smem, st>>>(ca);
  return launched();
}

}  // namespace

// Host side of the schedule.  Processing order: strips of L element columns
// (x), each walked along y, rows x-fastest inside a strip.  CTA c takes steps
// [c N / G, (c + 1) N / G).  Per CTA an x_j already in a slot is not loaded
// again; a load takes a free slot, else evicts the slot whose x_j is needed
// again furthest ahead in the CTA's steps (Belady's rule), among the slots
// whose last reader is at least kLag rows back (the converter waits for that
// row's MMAs, never for a specific older one).  If no slot qualifies the plan
// fails and the caller uses the per-use kernel (tc_apply.cu).
std::string tc_sched_plan(int dim, int n, int64_t nrows, const int64_t* row_ptr, const int32_t* col, int rcap,
                          int prec, int G, int L, TcSchedHost* out) {
  if (dim != 2 || int64_t(n) * n != nrows) return "the cached tensor-core apply takes 2D meshes";
  if (rcap < 1 || rcap > 64) return "the cached tensor-core apply takes at most 64 right-hand sides";
  if (L < 1 || G < 1) return "bad strip width or CTA count";
  int kmax = 0;
  for (int64_t r = 0; r < nrows; ++r) kmax = std::max<int>(kmax, int(row_ptr[r + 1] - row_ptr[r]));
  if (kmax > kMaxBlocksPerRow) return "more than 16 blocks in a row";
  if (row_ptr[nrows] >= (int64_t(1) << 31)) return "too many blocks";
  const bool split = prec == P_FP32;
  const int S = std::min(cached_slots(rcap, std::max(kmax, 1), split), 255);
  if (S < 8) return "too few x slots fit in shared memory";
  L = std::min(L, n);
  std::vector<int32_t> order;
  order.reserve(size_t(nrows));
  for (int x0 = 0; x0 < n; x0 += L) {
    const int w = std::min(L, n - x0);
    for (int y = 0; y < n; ++y)
      for (int i = 0; i < w; ++i) order.push_back(int32_t(x0 + i + int64_t(n) * y));
  }
  const int g = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(G) * kCtasPerSm, nrows / 8)));
  out->G = g;
  out->S = S;
  out->L = L;
  out->kmax = std::max(kmax, 1);
  out->rcap = rcap;
  out->seg.assign(size_t(g) + 1, 0);
  for (int c = 0; c <= g; ++c) out->seg[size_t(c)] = int(int64_t(c) * nrows / g);
  out->rec.assign(size_t(nrows) * sizeof(TcStep), 0);
  out->ld_elem.clear();
  constexpr int64_t kNever = INT64_MAX;
  std::vector<int32_t> slot_of(size_t(nrows), -1);     // element -> slot (this CTA)
  std::vector<int32_t> content(size_t(S), -1);          // slot -> element
  std::vector<int64_t> last_use(size_t(S), -1);         // slot -> last step that read it
  // uses of each element in this CTA's steps, in order (next-use lookups)
  std::vector<int64_t> use_head(size_t(nrows), -1), use_next;
  std::vector<int64_t> use_step;
  for (int c = 0; c < g; ++c) {
    const int a = out->seg[size_t(c)], b = out->seg[size_t(c) + 1];
    use_step.clear();
    use_next.clear();
    std::vector<int64_t> tail;
    // linked lists of uses per element, built backwards so heads are the first use
    for (int s = b - 1; s >= a; --s) {
      const int32_t row = order[size_t(s)];
      for (int64_t z = row_ptr[row]; z < row_ptr[row + 1]; ++z) {
        const int32_t j = col[z];
        if (use_head[size_t(j)] >= 0 && use_step[size_t(use_head[size_t(j)])] == s) continue;
        use_step.push_back(s);
        use_next.push_back(use_head[size_t(j)]);
        use_head[size_t(j)] = int64_t(use_step.size()) - 1;
      }
    }
    auto next_use = [&](int32_t j, int s) -> int64_t {     // first use of j at or after step s
      int64_t u = use_head[size_t(j)];
      while (u >= 0 && use_step[size_t(u)] < s) u = use_next[size_t(u)];
      use_head[size_t(j)] = u;
      return u >= 0 ? use_step[size_t(u)] : kNever;
    };
    std::fill(content.begin(), content.end(), -1);
    std::fill(last_use.begin(), last_use.end(), int64_t(-1));
    std::string fail;
    for (int s = a; s < b && fail.empty(); ++s) {
      const int32_t row = order[size_t(s)];
      TcStep rec{};
      rec.row = row;
      rec.z0 = int32_t(row_ptr[row]);
      rec.ld0 = int32_t(out->ld_elem.size());
      rec.nnz = uint16_t(row_ptr[row + 1] - row_ptr[row]);
      for (int64_t z = row_ptr[row]; z < row_ptr[row + 1]; ++z) {
        const int32_t j = col[z];
        if (slot_of[size_t(j)] < 0) {
          int best = -1;
          int64_t best_next = -1;
          for (int sl = 0; sl < S; ++sl) {
            if (content[size_t(sl)] < 0) { best = sl; break; }
            if (last_use[size_t(sl)] > int64_t(s) - kLag) continue;
            const int64_t nu = next_use(content[size_t(sl)], s);
            if (nu > best_next) {
              best_next = nu;
              best = sl;
            }
          }
          if (best < 0) {
            fail = "x slot ring too small for this strip width";
            break;
          }
          if (content[size_t(best)] >= 0) slot_of[size_t(content[size_t(best)])] = -1;
          content[size_t(best)] = j;
          slot_of[size_t(j)] = best;
          out->ld_elem.push_back(j);
          rec.lslot[rec.nld] = uint8_t(best);
          ++rec.nld;
        }
        const int sl = slot_of[size_t(j)];
        rec.slot[z - row_ptr[row]] = uint8_t(sl);
        last_use[size_t(sl)] = s;
      }
      std::memcpy(out->rec.data() + size_t(s) * sizeof(TcStep), &rec, sizeof(TcStep));
    }
    for (int32_t e : content)
      if (e >= 0) slot_of[size_t(e)] = -1;
    for (int s = a; s < b; ++s) {
      const int32_t row = order[size_t(s)];
      for (int64_t z = row_ptr[row]; z < row_ptr[row + 1]; ++z) use_head[size_t(col[z])] = -1;
    }
    if (!fail.empty()) return fail;
  }
  out->nloads = int64_t(out->ld_elem.size());
  out->ld_elem.resize(out->ld_elem.size() + 32, 0);     // the copier reads 32-entry windows
  return "";
}

cudaError_t bsr_apply_tc_cached(const BatchArgs& a, const TcSched& sc, int prec, cudaStream_t st) {
  if (a.R < 1 || a.R > sc.rcap || !sc.rec || a.es != int64_t(a.R) * kB || a.rs != kB)
    return cudaErrorInvalidValue;
  const bool split = prec == P_FP32;
  if (!split && prec != P_BF16) return cudaErrorInvalidValue;
  if (a.nrows == 0) return cudaSuccess;
  const CachedPlan p = cached_plan(a.R, sc.kmax, split, sc.S);
  if (p.total > kSmemCap) return cudaErrorInvalidValue;
  CachedArgs ca;
  ca.a = a;
  ca.rec = static_cast<const TcStep*>(sc.rec);
  ca.seg = sc.seg;
  ca.ld_elem = sc.ld_elem;
  ca.S = sc.S;
  ca.kmax = sc.kmax;
  ca.need_rhs = (a.mode == M_RES || a.mode == M_AXPY) ? 1 : 0;
  ca.off_a = p.off_a;
  ca.off_raw = p.off_raw;
  ca.off_ctrl = p.off_ctrl;
  ca.stage_a = p.stage_a;
  ca.raw_bytes = p.raw_bytes;
  return split ? launch_cached<true>(ca, p.total, sc.G, st) : launch_cached<false>(ca, p.total, sc.G, st);
}

}  // namespace ldgmg
