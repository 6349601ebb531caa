// Batched FP64 least squares on the device for the SAI setup (Sec. 2.3.3).
//
// Every distinct balanced column problem  min ||Atilde[R(i), S(i)] X - E[R(i), i]||_F
// of a level is one CTA: Householder QR of W = [M | Rhs] in place in device
// memory (column-major, m rows), then back substitution R X = Q^T Rhs.  The
// arithmetic follows the host version (csrc/host.cpp householder_ls: the same
// reflector sign, 2 / v^T v, the same 1e-12 rank test), with the sums taken in
// a different order.  Problems whose R has |R_jj| <= 1e-12 max |R_jj| are
// reported back; the host then takes the minimum-norm solution.
//
// One CTA of 256 threads per problem: each Householder step reduces the
// column norm over the CTA, keeps the reflector v in shared memory, and lets
// each warp update whole columns (a dot product with v, then the update);
// the back substitution runs one warp per right-hand side with its solution
// in shared memory.  The work is FP64 and memory bound (W of a 3D p = 3
// column is 1600 x 512 doubles); it is setup, not the hot path.
#include "host.h"
#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace ldgmg {

namespace {

constexpr int kLsThreads = 256;
constexpr int kLsWarps = kLsThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the CTA, returned to every thread
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kLsWarps; ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(kLsThreads) ls_qr_kernel(const int* __restrict__ dims,
                                                           const int64_t* __restrict__ woff,
                                                           const int64_t* __restrict__ xoff, double* __restrict__ Wall,
                                                           double* __restrict__ Xall, int* __restrict__ okall) {
  extern __shared__ double sm[];
  const int k = blockIdx.x;
  const int m = dims[3 * k], nc = dims[3 * k + 1], nr = dims[3 * k + 2];
  const int ncol = nc + nr;
  double* W = Wall + woff[k];
  double* X = Xall + xoff[k];
  double* v = sm;                      // m: the current reflector
  double* diag = v + m;                // nc: R_jj
  double* red = diag + nc;             // kLsWarps
  double* xs = red + kLsWarps;         // kLsWarps x nc: one solution column per warp
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int j = 0; j < nc; ++j) {
    const double* wj = W + int64_t(j) * m;
    double s = 0.0;
    for (int i = j + tid; i < m; i += kLsThreads) s += wj[i] * wj[i];
    s = block_sum(s, red);
    const double wjj = wj[j];
    const double nrm = sqrt(s);
    const double alpha = wjj > 0.0 ? -nrm : nrm;
    const double vv = s - wjj * wjj + (wjj - alpha) * (wjj - alpha);
    if (nrm == 0.0 || vv == 0.0) {       // nothing to reflect (same test on every thread)
      if (tid == 0) diag[j] = nrm == 0.0 ? 0.0 : alpha;
      __syncthreads();
      continue;
    }
    for (int i = j + tid; i < m; i += kLsThreads) v[i] = i == j ? wjj - alpha : wj[i];
    __syncthreads();
    const double beta = 2.0 / vv;
    for (int c = j + 1 + warp; c < ncol; c += kLsWarps) {
      double* wc = W + int64_t(c) * m;
      double d = 0.0;
      for (int i = j + lane; i < m; i += 32) d += v[i] * wc[i];
      d = warp_sum(d) * beta;
      for (int i = j + lane; i < m; i += 32) wc[i] -= d * v[i];
    }
    if (tid == 0) diag[j] = alpha;
    __syncthreads();
  }
  // rank test of R
  double dmax = 0.0;
  for (int j = tid; j < nc; j += kLsThreads) dmax = fmax(dmax, fabs(diag[j]));
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  __syncthreads();
  if (lane == 0) red[warp] = dmax;
  __syncthreads();
  dmax = 0.0;
  for (int w = 0; w < kLsWarps; ++w) dmax = fmax(dmax, red[w]);
  int bad = 0;
  for (int j = tid; j < nc; j += kLsThreads) bad |= !(fabs(diag[j]) > 1e-12 * dmax);
  bad = __syncthreads_or(bad);
  if (tid == 0) okall[k] = bad ? 0 : 1;
  if (bad) return;
  // back substitution R x = (Q^T rhs)[0 : nc], one warp per right-hand side
  double* x = xs + int64_t(warp) * nc;
  for (int c = warp; c < nr; c += kLsWarps) {
    const double* rc = W + int64_t(nc + c) * m;
    for (int j = nc - 1; j >= 0; --j) {
      double d = 0.0;
      for (int l = j + 1 + lane; l < nc; l += 32) d += W[int64_t(l) * m + j] * x[l];
      d = warp_sum(d);
      if (lane == 0) x[j] = (rc[j] - d) / diag[j];
      __syncwarp();
    }
    for (int j = lane; j < nc; j += 32) X[int64_t(c) * nc + j] = x[j];
    __syncwarp();
  }
}

template <class T>
cudaError_t dev_alloc(T** p, size_t n) {
  *p = nullptr;
  return n ? cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)) : cudaSuccess;
}

}  // namespace

std::string sai_ls_device(std::vector<LsProblem>& batch, cudaStream_t st) {
  const int np = int(batch.size());
  if (np == 0) return "";
  std::vector<int> dims(size_t(np) * 3);
  std::vector<int64_t> woff(np), xoff(np);
  int64_t wtot = 0, xtot = 0;
  int max_m = 0, max_nc = 0;
  for (int k = 0; k < np; ++k) {
    const LsProblem& P = batch[size_t(k)];
    dims[3 * k] = P.m;
    dims[3 * k + 1] = P.nc;
    dims[3 * k + 2] = P.nr;
    woff[k] = wtot;
    xoff[k] = xtot;
    wtot += int64_t(P.m) * (P.nc + P.nr);
    xtot += int64_t(P.nc) * P.nr;
    max_m = std::max(max_m, P.m);
    max_nc = std::max(max_nc, P.nc);
  }
  const size_t smem = (size_t(max_m) + max_nc + kLsWarps + size_t(kLsWarps) * max_nc) * sizeof(double);
  if (smem > 227 * 1024) return "SAI least squares too large for the device solver";
  int* d_dims = nullptr;
  int* d_ok = nullptr;
  int64_t *d_woff = nullptr, *d_xoff = nullptr;
  double *d_W = nullptr, *d_X = nullptr;
  std::string err;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && err.empty()) err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  if (ck(dev_alloc(&d_dims, dims.size()), "cudaMalloc") && ck(dev_alloc(&d_ok, size_t(np)), "cudaMalloc") &&
      ck(dev_alloc(&d_woff, size_t(np)), "cudaMalloc") && ck(dev_alloc(&d_xoff, size_t(np)), "cudaMalloc") &&
      ck(dev_alloc(&d_W, size_t(wtot)), "cudaMalloc") && ck(dev_alloc(&d_X, size_t(xtot)), "cudaMalloc")) {
    bool go = ck(cudaMemcpyAsync(d_dims, dims.data(), dims.size() * sizeof(int), cudaMemcpyHostToDevice, st), "copy") &&
              ck(cudaMemcpyAsync(d_woff, woff.data(), woff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st),
                 "copy") &&
              ck(cudaMemcpyAsync(d_xoff, xoff.data(), xoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st),
                 "copy");
    for (int k = 0; k < np && go; ++k)
      go = ck(cudaMemcpyAsync(d_W + woff[k], batch[size_t(k)].W.data(), batch[size_t(k)].W.size() * sizeof(double),
                              cudaMemcpyHostToDevice, st),
              "copy W");
    if (go && smem > 48 * 1024)
      go = ck(cudaFuncSetAttribute(ls_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
              "shared memory opt-in");
    if (go) {
      ls_qr_kernel<<<unsigned(np), kLsThreads, smem, st>>>(d_dims, d_woff, d_xoff, d_W, d_X, d_ok);
      go = ck(launched(), "ls_qr_kernel launch");
    }
    std::vector<int> ok(np, 0);
    std::vector<double> Xh(static_cast<size_t>(xtot));
    if (go) go = ck(cudaMemcpyAsync(ok.data(), d_ok, size_t(np) * sizeof(int), cudaMemcpyDeviceToHost, st), "copy ok");
    if (go && xtot)
      go = ck(cudaMemcpyAsync(Xh.data(), d_X, size_t(xtot) * sizeof(double), cudaMemcpyDeviceToHost, st), "copy X");
    if (go) go = ck(cudaStreamSynchronize(st), "SAI least squares");
    if (go)
      for (int k = 0; k < np; ++k) {
        LsProblem& P = batch[size_t(k)];
        P.ok = ok[k] != 0;
        if (P.ok) P.X.assign(Xh.begin() + xoff[k], Xh.begin() + xoff[k] + int64_t(P.nc) * P.nr);
      }
  }
  cudaFree(d_dims);
  cudaFree(d_ok);
  cudaFree(d_woff);
  cudaFree(d_xoff);
  cudaFree(d_W);
  cudaFree(d_X);
  return err;
}

}  // namespace ldgmg
