// Grouped solve: many small independent scalar problems, of any mix of
// classes (mesh, degree, coefficient field, smoother, V-cycle precision), in
// one kernel launch.
//
// Each problem is a whole preconditioned CG solve (Sec. 2.2) with the
// V-cycle of Algorithm 1 as the preconditioner: smoothing by SAI (Eqs. B1 /
// BT, Sec. 2.3.3), damped block Jacobi (Sec. 2.3.1) or multi-coloured block
// Gauss-Seidel (Sec. 2.3.2), restriction and prolongation by the tensor-
// product polynomial injection (Sec. 2.2), and the dense pseudo-inverse on
// the bottom level.  One thread-block cluster of C CTAs (C = 1, 2, 4 or 8)
// runs one problem from start to finish: every step is spread over the
// cluster's threads and followed by a cluster barrier (release / acquire at
// cluster scope, which orders the global-memory vectors the next step
// reads).  Inner products are reduced inside each CTA, the C partial sums
// are exchanged through distributed shared memory and added in rank order,
// so every CTA holds the same value and takes the same branch: the barrier
// sequence is identical across the cluster.  Problems too small to fill the
// GPU on their own (a few thousand to a few ten thousand unknowns) then cost
// one launch per group instead of a few hundred launches and a few host
// round trips per problem.
//
// The arithmetic follows the per-problem path: matrix entries in their
// storage precision accumulated in FP64 (FP64 storage) or FP32 (otherwise),
// level vectors in the V-cycle precision, the outer CG in FP64 against the
// FP64 operator, flexible CG (Polak-Ribiere beta) with a reduced-precision
// V-cycle, and the same stopping test and FP64 true-residual confirmation
// with restarts.  Sums are taken in a different order, so results agree with
// ldgmg_solve to rounding, not bitwise.
#pragma once

#include "kernels.h"

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <mutex>

namespace ldgmg {

namespace {

namespace cg = cooperative_groups;

constexpr int kGT = 512;            // threads per CTA
constexpr int kGW = kGT / 32;
constexpr int kMaxRestarts = 16;    // FP64 true-residual restarts of the flexible CG

static_assert(sizeof(GroupProblem) % 8 == 0, "descriptor copied as 8-byte words");

struct Smem {
  GroupProblem P;
  double Ps[2][8][8];               // one-dimensional injection matrices P[s][i][j]
  double red[2][kGW];
  double slot[2][2];                // ping-pong slots of the CTA's partial inner products (two sums each)
};

template <class TA> struct AccT { typedef float T; };
template <> struct AccT<double> { typedef double T; };

template <class TACC, class TA> __device__ __forceinline__ TACC cv(TA v) { return TACC(v); }
template <> __device__ __forceinline__ float cv<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float cv<float, __half>(__half v) { return __half2float(v); }

// the C CTAs of one cluster; t = this thread's index within the cluster
template <int C> struct Team {
  int rank, t, stride;
  __device__ Team() {
    rank = C == 1 ? 0 : int(cg::this_cluster().block_rank());
    t = rank * kGT + int(threadIdx.x);
    stride = C * kGT;
  }
  __device__ void sync() const {
    if (C == 1) __syncthreads();
    else cg::this_cluster().sync();
  }
};

// (sum_i a_i b_i, sum_i c_i d_i) over the cluster in one pass, the same
// values in every thread of every CTA: each CTA reduces its part (warp
// shuffles, then its warps in order), the C partial sums are exchanged
// through distributed shared memory and added in rank order.  c may be null
// (one sum).
template <int C>
__device__ void team_dot2(const Team<C>& tm, Smem& sm, int& pp, const double* a, const double* b, const double* c,
                          const double* d, int64_t n, double* out0, double* out1) {
  double s0 = 0.0, s1 = 0.0;
  if (c) {
    for (int64_t i = tm.t; i < n; i += tm.stride) {
      s0 += a[i] * b[i];
      s1 += c[i] * d[i];
    }
  } else {
    for (int64_t i = tm.t; i < n; i += tm.stride) s0 += a[i] * b[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sm.red[0][threadIdx.x >> 5] = s0;
    sm.red[1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int w = 0; w < kGW; ++w) v += sm.red[threadIdx.x][w];
    sm.slot[pp][threadIdx.x] = v;
  }
  tm.sync();
  double t0 = 0.0, t1 = 0.0;
  if (C == 1) {
    t0 = sm.slot[pp][0];
    t1 = sm.slot[pp][1];
  } else {
    cg::cluster_group cl = cg::this_cluster();
    for (int r = 0; r < C; ++r) {
      t0 += *cl.map_shared_rank(&sm.slot[pp][0], r);
      t1 += *cl.map_shared_rank(&sm.slot[pp][1], r);
    }
  }
  pp ^= 1;
  *out0 = t0;
  if (out1) *out1 = t1;
}

template <int C>
__device__ double team_dot(const Team<C>& tm, Smem& sm, int& pp, const double* a, const double* b, int64_t n) {
  double v;
  team_dot2(tm, sm, pp, a, b, nullptr, nullptr, n, &v, nullptr);
  return v;
}

// y = epilogue(M x) on block rows 0..nrows-1 or on the nrows rows listed in
// `rows`: one thread per (row, output mode), the b x b block columns
// streamed in column-major order.  The problems are small and their data sit
// in L2, so a step costs a few L2 round trips per thread: the block size is
// a template parameter and two blocks are read per round, every load of a
// round issued before its products are summed (one round trip per two blocks
// for b <= 16).
template <int B, class TA, class TV, int C>
__device__ __forceinline__ void apply_b(const Team<C>& tm, const GroupMat& M, int64_t nrows, const int* rows, int mode,
                                        const TV* x, const TV* rhs, const TV* xin, TV* y, double s) {
  typedef typename AccT<TA>::T TACC;
  constexpr int U = B < 16 ? B : 16;       // columns per round
  const TA* vals = static_cast<const TA*>(M.vals);
  const int cs = M.cs;
  const int64_t tot = nrows * B;
  for (int64_t idx = tm.t; idx < tot; idx += tm.stride) {
    const int64_t i = idx / B;
    const int r = int(idx - i * B);
    const int64_t row = rows ? int64_t(rows[i]) : i;
    TACC acc = TACC(0);
    const int z1 = M.row_ptr[row + 1];
    for (int z = M.row_ptr[row]; z < z1; z += 2) {
      const bool two = z + 1 < z1;
      const TA* b0 = vals + int64_t(z) * B * cs + r;
      const TA* b1 = two ? b0 + int64_t(B) * cs : b0;
      const TV* x0 = x + int64_t(M.col[z]) * B;
      const TV* x1 = two ? x + int64_t(M.col[z + 1]) * B : x0;
#pragma unroll 1
      for (int c0 = 0; c0 < B; c0 += U) {
        TACC pa[U], pb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c = c0 + u;
          pa[u] = c < B ? cv<TACC>(b0[c * cs]) * TACC(x0[c]) : TACC(0);
          pb[u] = (c < B && two) ? cv<TACC>(b1[c * cs]) * TACC(x1[c]) : TACC(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc += pa[u];
#pragma unroll
        for (int u = 0; u < U; ++u) acc += pb[u];
      }
    }
    acc *= TACC(M.inv_scale);
    const int64_t o = row * B + r;
    switch (mode) {
      case M_Y: y[o] = TV(acc); break;
      case M_RES: y[o] = TV(TACC(rhs[o]) - acc); break;
      case M_AXPY: y[o] = TV(TACC(xin[o]) + TACC(s) * acc); break;
      default: y[o] = TV(TACC(s) * acc); break;
    }
  }
}

template <class TA, class TV, int C>
__device__ __forceinline__ void apply_t(const Team<C>& tm, const GroupMat& M, int b, int64_t nrows, const int* rows,
                                        int mode, const TV* x, const TV* rhs, const TV* xin, TV* y, double s) {
  switch (b) {
    case 4: apply_b<4, TA, TV, C>(tm, M, nrows, rows, mode, x, rhs, xin, y, s); break;
    case 8: apply_b<8, TA, TV, C>(tm, M, nrows, rows, mode, x, rhs, xin, y, s); break;
    case 9: apply_b<9, TA, TV, C>(tm, M, nrows, rows, mode, x, rhs, xin, y, s); break;
    case 16: apply_b<16, TA, TV, C>(tm, M, nrows, rows, mode, x, rhs, xin, y, s); break;
    case 25: apply_b<25, TA, TV, C>(tm, M, nrows, rows, mode, x, rhs, xin, y, s); break;
    case 27: apply_b<27, TA, TV, C>(tm, M, nrows, rows, mode, x, rhs, xin, y, s); break;
    case 36: apply_b<36, TA, TV, C>(tm, M, nrows, rows, mode, x, rhs, xin, y, s); break;
    default: apply_b<64, TA, TV, C>(tm, M, nrows, rows, mode, x, rhs, xin, y, s); break;
  }
}

// one instance per (vector type, cluster size): the block-size and storage
// switch is compiled once, not at every call site
template <class TV, int C>
__device__ __noinline__ void apply(const Team<C>& tm, const GroupMat& M, int b, int64_t nrows, const int* rows,
                                   int mode, const TV* x, const TV* rhs, const TV* xin, TV* y, double s) {
  if constexpr (sizeof(TV) == 8) {
    apply_t<double, double, C>(tm, M, b, nrows, rows, mode, x, rhs, xin, y, s);
  } else {
    switch (M.prec) {
      case P_FP32: apply_t<float, float, C>(tm, M, b, nrows, rows, mode, x, rhs, xin, y, s); break;
      case P_BF16: apply_t<__nv_bfloat16, float, C>(tm, M, b, nrows, rows, mode, x, rhs, xin, y, s); break;
      default: apply_t<__half, float, C>(tm, M, b, nrows, rows, mode, x, rhs, xin, y, s); break;
    }
  }
}

// rc_C = sum over the 2^d children s of (P_s1 (x) ... )^T rf_child(s): the
// weight of fine mode k for coarse mode t is prod_a P[s_a][k_a][t_a]
// (mode t = t_0 + t_1 q + t_2 q^2; element e = i_0 + i_1 n + i_2 n^2).
template <class TV, int C>
__device__ __noinline__ void restrict_t(const Team<C>& tm, const Smem& sm, int d, int q, int nf, const TV* rf, TV* rc) {
  const int b = d == 2 ? q * q : q * q * q;
  const int nch = 1 << d;
  const int nc = nf / 2;
  const int64_t nf2 = int64_t(nf) * nf;
  const int64_t Nc = d == 2 ? int64_t(nc) * nc : int64_t(nc) * nc * nc;
  const int q2 = d == 3 ? q : 1;
  for (int64_t idx = tm.t; idx < Nc * b; idx += tm.stride) {
    const int64_t ce = idx / b;
    const int t = int(idx - ce * b);
    const int t0 = t % q, t1 = (t / q) % q, t2 = t / (q * q);
    const int64_t c0 = ce % nc, c1 = (ce / nc) % nc, c2 = ce / (int64_t(nc) * nc);
    const int64_t fbase = 2 * c0 + 2 * c1 * nf + 2 * c2 * nf2;
    TV acc = TV(0);
    // children and fine modes along x unrolled (predicated), so a round's
    // loads are in flight together
    for (int k2 = 0; k2 < q2; ++k2) {
      for (int k1 = 0; k1 < q; ++k1) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          if (s < nch) {
            const int s0 = s & 1, s1 = (s >> 1) & 1, s2 = (s >> 2) & 1;
            const TV w = (d == 3 ? TV(sm.Ps[s2][k2][t2]) : TV(1)) * TV(sm.Ps[s1][k1][t1]);
            const TV* sk = rf + (fbase + s0 + s1 * nf + s2 * nf2) * b + k1 * q + k2 * q * q;
#pragma unroll
            for (int k0 = 0; k0 < 8; ++k0)
              if (k0 < q) acc += w * TV(sm.Ps[s0][k0][t0]) * sk[k0];
          }
        }
      }
    }
    rc[idx] = acc;
  }
}

// xf_e += (P_s1 (x) ...) xc_parent(e): weight of coarse mode k for fine mode t
// is prod_a P[s_a][t_a][k_a], s the child position of e in its parent
template <class TV, int C>
__device__ __noinline__ void prolong_t(const Team<C>& tm, const Smem& sm, int d, int q, int nf, const TV* xc, TV* xf) {
  const int b = d == 2 ? q * q : q * q * q;
  const int nc = nf / 2;
  const int64_t nf2 = int64_t(nf) * nf;
  const int64_t Nf = d == 2 ? nf2 : nf2 * nf;
  const int q2 = d == 3 ? q : 1;
  for (int64_t idx = tm.t; idx < Nf * b; idx += tm.stride) {
    const int64_t e = idx / b;
    const int t = int(idx - e * b);
    const int t0 = t % q, t1 = (t / q) % q, t2 = t / (q * q);
    const int64_t i0 = e % nf, i1 = (e / nf) % nf, i2 = e / nf2;
    const int s0 = int(i0 & 1), s1 = int(i1 & 1), s2 = int(i2 & 1);
    const TV* src = xc + ((i0 >> 1) + (i1 >> 1) * nc + (i2 >> 1) * int64_t(nc) * nc) * b;
    TV acc = TV(0);
    for (int k2 = 0; k2 < q2; ++k2) {
      const TV w2 = d == 3 ? TV(sm.Ps[s2][t2][k2]) : TV(1);
      for (int k1 = 0; k1 < q; ++k1) {
        const TV w1 = w2 * TV(sm.Ps[s1][t1][k1]);
        const TV* sk = src + k1 * q + k2 * q * q;
#pragma unroll
        for (int k0 = 0; k0 < 8; ++k0)
          if (k0 < q) acc += w1 * TV(sm.Ps[s0][t0][k0]) * sk[k0];
      }
    }
    xf[idx] += acc;
  }
}

// y = Pinv v (bottom level), one warp per row, FP64 sums
template <class TV, int C>
__device__ void bottom(const Team<C>& tm, const double* pinv, int64_t n, const TV* v, TV* y) {
  const int lane = threadIdx.x & 31;
  for (int64_t row = tm.t >> 5; row < n; row += tm.stride >> 5) {
    const double* pr = pinv + row * n;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += pr[j] * double(v[j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = TV(s);
  }
}

template <class TV, int C>
__device__ void fill(const Team<C>& tm, TV* v, int64_t n) {
  for (int64_t i = tm.t; i < n; i += tm.stride) v[i] = TV(0);
}

// one smoothing step on level D: x <- x + M (rhs - A x) (x = 0 before it
// when xz); the level's rhs, x and r are consecutive in lvec
template <class TV, int C>
__device__ void smooth(const Team<C>& tm, const GroupProblem& P, const GroupLevel& D, TV* lvec, bool bt, bool xz) {
  const int64_t nb = D.N * D.b;
  TV* rhs = lvec + D.voff;
  TV* x = rhs + nb;
  TV* r = x + nb;
  if (P.smoother == G_GS) {
    // colour by colour (forward for B1, backward for BT), omega = 1
    if (xz) {
      fill(tm, x, nb);
      tm.sync();
    }
    for (int k = 0; k < D.ncolours; ++k) {
      const int c = bt ? D.ncolours - 1 - k : k;
      const int c0 = D.cptr[c], c1 = D.cptr[c + 1];
      const int* rows = D.crows + c0;
      if (xz && k == 0) {
        apply<TV, C>(tm, D.S, D.b, c1 - c0, rows, M_SCALE, rhs, nullptr, nullptr, x, 1.0);
        tm.sync();
        continue;
      }
      apply<TV, C>(tm, D.A, D.b, c1 - c0, rows, M_RES, x, rhs, nullptr, r, 1.0);
      tm.sync();
      apply<TV, C>(tm, D.S, D.b, c1 - c0, rows, M_AXPY, r, nullptr, x, x, 1.0);
      tm.sync();
    }
    return;
  }
  const bool jac = P.smoother == G_JACOBI;
  const GroupMat& M = jac ? D.S : (bt ? D.ST : D.S);
  const double w = jac ? P.omega : 1.0;
  if (xz) {
    apply<TV, C>(tm, M, D.b, D.N, nullptr, jac ? M_SCALE : M_Y, rhs, nullptr, nullptr, x, w);
  } else {
    apply<TV, C>(tm, D.A, D.b, D.N, nullptr, M_RES, x, rhs, nullptr, r, 1.0);
    tm.sync();
    apply<TV, C>(tm, M, D.b, D.N, nullptr, M_AXPY, r, nullptr, x, x, w);
  }
  tm.sync();
}

// Algorithm 1 on level l, first half: pre-smoothing from x = 0, then the
// restricted residual becomes the right-hand side of level l + 1
template <class TV, int C>
__device__ void vc_down(const Team<C>& tm, const Smem& sm, TV* lvec, int l) {
  const GroupProblem& P = sm.P;
  const GroupLevel& D = P.lv[l];
  const int64_t nb = D.N * D.b;
  TV* rhs = lvec + D.voff;
  TV* x = rhs + nb;
  TV* r = x + nb;
  for (int s = 0; s < P.nu1; ++s) smooth(tm, P, D, lvec, P.pre_bt != 0, s == 0);
  TV* rc = lvec + P.lv[l + 1].voff;
  if (P.nu1 == 0) {
    restrict_t(tm, sm, P.dim, P.q, D.n, rhs, rc);
  } else {
    apply<TV, C>(tm, D.A, D.b, D.N, nullptr, M_RES, x, rhs, nullptr, r, 1.0);
    tm.sync();
    restrict_t(tm, sm, P.dim, P.q, D.n, r, rc);
  }
  tm.sync();
}

// second half: correction from level l + 1, then post-smoothing
template <class TV, int C>
__device__ void vc_up(const Team<C>& tm, const Smem& sm, TV* lvec, int l) {
  const GroupProblem& P = sm.P;
  const GroupLevel& D = P.lv[l];
  const GroupLevel& Dc = P.lv[l + 1];
  TV* x = lvec + D.voff + D.N * D.b;
  if (P.nu1 == 0) {
    fill(tm, x, D.N * D.b);
    tm.sync();
  }
  prolong_t(tm, sm, P.dim, P.q, D.n, lvec + Dc.voff + Dc.N * Dc.b, x);
  tm.sync();
  for (int s = 0; s < P.nu2; ++s) smooth(tm, P, D, lvec, P.post_bt != 0, false);
}

// levels lo .. nl - 1: x_lo = V_lo rhs_lo
template <class TV, int C>
__device__ void vcycle_from(const Team<C>& tm, const Smem& sm, TV* lvec, int lo) {
  const GroupProblem& P = sm.P;
  for (int l = lo; l + 1 < P.nl; ++l) vc_down(tm, sm, lvec, l);
  const GroupLevel& B = P.lv[P.nl - 1];
  TV* rhs = lvec + B.voff;
  bottom(tm, P.pinv, P.nbot, rhs, rhs + B.N * B.b);
  tm.sync();
  for (int l = P.nl - 2; l >= lo; --l) vc_up(tm, sm, lvec, l);
}

// level 0: x = V rhs (Algorithm 1, x = 0 initially).  In a cluster, the
// coarse levels (at most kSoloDofs unknowns, two per thread of one CTA) run on
// the first CTA alone with CTA barriers; the others wait at the cluster
// barrier that hands the coarse correction back.
constexpr int64_t kSoloDofs = 2 * kGT;

template <class TV, int C>
__device__ void vcycle(const Team<C>& tm, const Smem& sm, TV* lvec) {
  if constexpr (C == 1) {
    vcycle_from(tm, sm, lvec, 0);
  } else {
    const GroupProblem& P = sm.P;
    int lc = 0;
    while (lc < P.nl && P.lv[lc].N * P.lv[lc].b > kSoloDofs) ++lc;
    if (lc == P.nl) {
      vcycle_from(tm, sm, lvec, 0);
      return;
    }
    for (int l = 0; l < lc; ++l) vc_down(tm, sm, lvec, l);
    if (tm.rank == 0) {
      const Team<1> solo;
      vcycle_from(solo, sm, lvec, lc);
    }
    tm.sync();
    for (int l = lc - 1; l >= 0; --l) vc_up(tm, sm, lvec, l);
  }
}

// z = V r: FP64 vectors in, the V-cycle in the level-vector precision
template <class TV, int C>
__device__ void apply_V(const Team<C>& tm, const Smem& sm, TV* lvec, const double* r, double* z) {
  const int64_t n = sm.P.n0;
  TV* rhs0 = lvec + sm.P.lv[0].voff;
  for (int64_t i = tm.t; i < n; i += tm.stride) rhs0[i] = TV(r[i]);
  tm.sync();
  vcycle(tm, sm, lvec);
  const TV* x0 = rhs0 + n;
  for (int64_t i = tm.t; i < n; i += tm.stride) z[i] = double(x0[i]);
  tm.sync();
}

template <class TV, int C>
__device__ void solve_item(const Team<C>& tm, Smem& sm, const GroupItem& I, bool leader) {
  const GroupProblem& P = sm.P;
  const int64_t n = P.n0;
  const int b0 = P.lv[0].b;
  const int64_t N0 = P.lv[0].N;
  TV* lvec = static_cast<TV*>(I.lvec);
  double* r = I.cg;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  const double* bv = I.b;
  double* x = I.x;
  int pp = 0;
  const double bb = team_dot(tm, sm, pp, bv, bv, n);
  if (!isfinite(bb)) {
    if (leader) *I.out = GroupOut{0, 3, 0.0};
    return;
  }
  for (int64_t i = tm.t; i < n; i += tm.stride) {
    x[i] = 0.0;
    r[i] = bv[i];
  }
  tm.sync();
  if (bb == 0.0) {
    if (leader) *I.out = GroupOut{0, 0, 0.0};
    return;
  }
  const double tol2 = I.tol * I.tol;
  apply_V(tm, sm, lvec, r, z);
  for (int64_t i = tm.t; i < n; i += tm.stride) p[i] = z[i];
  double rz = team_dot(tm, sm, pp, r, z, n);
  int k = 0, status = 1;
  double rrt = 0.0;
  bool fresh = false;
  for (int round = 0;; ++round) {
    while (k < P.max_iter) {
      apply<double, C>(tm, P.A0, b0, N0, nullptr, M_Y, p, nullptr, nullptr, q, 1.0);
      tm.sync();
      const double pq = team_dot(tm, sm, pp, p, q, n);
      const double alpha = rz / pq;
      for (int64_t i = tm.t; i < n; i += tm.stride) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      // ||r||^2 and, for the flexible beta, r . z_old in one pass
      double rr = 0.0, rzold = 0.0;
      team_dot2(tm, sm, pp, r, r, P.flexible ? r : nullptr, z, n, &rr, &rzold);
      ++k;
      if (!isfinite(rr)) {
        status = 2;
        break;
      }
      if (rr <= tol2 * bb) {
        status = 0;
        break;
      }
      apply_V(tm, sm, lvec, r, z);
      const double rznew = team_dot(tm, sm, pp, r, z, n);
      const double beta = (P.flexible ? rznew - rzold : rznew) / rz;
      rz = rznew;
      for (int64_t i = tm.t; i < n; i += tm.stride) p[i] = z[i] + beta * p[i];
      tm.sync();
    }
    // a reduced-precision V-cycle lets the recurrence residual drift from
    // b - A x: confirm on the FP64 residual and restart CG from it if missed
    if (!P.flexible || status != 0 || round >= kMaxRestarts) break;
    tm.sync();
    apply<double, C>(tm, P.A0, b0, N0, nullptr, M_RES, x, bv, nullptr, r, 1.0);
    tm.sync();
    rrt = team_dot(tm, sm, pp, r, r, n);
    fresh = true;
    if (rrt <= tol2 * bb) break;
    fresh = false;
    status = 1;
    if (k >= P.max_iter) break;
    apply_V(tm, sm, lvec, r, z);
    for (int64_t i = tm.t; i < n; i += tm.stride) p[i] = z[i];
    rz = team_dot(tm, sm, pp, r, z, n);
  }
  if (!fresh) {
    tm.sync();
    apply<double, C>(tm, P.A0, b0, N0, nullptr, M_RES, x, bv, nullptr, r, 1.0);
    tm.sync();
    rrt = team_dot(tm, sm, pp, r, r, n);
  }
  if (leader) *I.out = GroupOut{k, status, sqrt(rrt / bb)};
}

template <int C>
__global__ void __launch_bounds__(kGT, 1) group_kernel(const GroupProblem* __restrict__ probs,
                                                    const GroupItem* __restrict__ items) {
  __shared__ Smem sm;
  const GroupItem I = items[blockIdx.x / C];
  const uint64_t* src = reinterpret_cast<const uint64_t*>(probs + I.prob);
  uint64_t* dst = reinterpret_cast<uint64_t*>(&sm.P);
  for (int i = threadIdx.x; i < int(sizeof(GroupProblem) / 8); i += kGT) dst[i] = src[i];
  __syncthreads();
  const int q = sm.P.q;
  for (int i = threadIdx.x; i < 2 * q * q; i += kGT) sm.Ps[i / (q * q)][(i / q) % q][i % q] = sm.P.P[i];
  __syncthreads();
  Team<C> tm;
  const bool leader = tm.t == 0;
  if (sm.P.vprec == 0) solve_item<double, C>(tm, sm, I, leader);
  else solve_item<float, C>(tm, sm, I, leader);
  tm.sync();   // no CTA leaves while another may still read its shared memory
}

template <int C>
cudaError_t launch_group(const GroupProblem* probs, const GroupItem* items, int count, cudaStream_t st) {
  // the kernel keeps its few kilobytes of shared state and reads everything
  // else through L1: ask for the largest L1 share (a hint, set once)
  static std::once_flag once;
  static cudaError_t cfg_err = cudaSuccess;
  std::call_once(once, [] {
    cfg_err = cudaFuncSetAttribute(group_kernel<C>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  });
  if (cfg_err != cudaSuccess) return cfg_err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(count) * C, 1, 1);
  cfg.blockDim = dim3(kGT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = C > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, group_kernel<C>, probs, items);
}

}  // namespace

}  // namespace ldgmg
