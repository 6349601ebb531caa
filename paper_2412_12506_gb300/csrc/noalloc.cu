// Allocation-free variant of the kernel projection (ldgmg_project_kernel_noalloc).
//
// Who needs it: callers that must not call cudaMalloc -- code whose device
// memory is wholly owned by another allocator (for instance a framework's
// caching allocator that has reserved the GPU, where an extra cudaMalloc can
// fail or fragment its pool), or a latency-critical loop that cannot take the
// implicit device synchronisation cudaMalloc may incur.  They also cannot hold
// an ldgmg_op, because creating one allocates.  This entry point needs neither:
// its only scratch is the file-scope device array below.
//
// The scratch (g_noalloc_scratch) is fixed at build time and is held by every
// GPU that loads this library until the process exits.  All calls share it, so
// calls that overlap on the GPU (different streams without ordering, or
// different host threads) race and give wrong results.  Every scratch word a
// call reads is written earlier in the same call, so nothing has to be cleared
// between calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "ldgmg.h"

void ldgmg_set_error(const std::string& msg);

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int64_t kChunk = int64_t(kThreads) * kPerThread;      // elements per partial sum
constexpr int64_t kMaxPartials = LDGMG_NOALLOC_MAX_ELEMENTS / kChunk;

// [0, kMaxPartials): one partial sum per chunk of elements; [kMaxPartials]: total
static __device__ __align__(256) double g_noalloc_scratch[kMaxPartials + 1];

// partial[k] = sum of the mode-0 coefficients of elements [k*kChunk, (k+1)*kChunk)
__global__ void chunk_sums(int64_t N, int64_t b, const double* __restrict__ v, double* __restrict__ partial) {
  const int64_t base = int64_t(blockIdx.x) * kChunk;
  double s = 0.0;
  for (int i = 0; i < kPerThread; ++i) {
    const int64_t e = base + int64_t(i) * kThreads + threadIdx.x;
    if (e < N) s += v[e * b];
  }
  __shared__ double ws[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// total = sum of the partials in a fixed order
__global__ void total_sum(int64_t nparts, double* __restrict__ partial) {
  __shared__ double ws[kThreads / 32];
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < nparts; k += kThreads) s += partial[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
    partial[kMaxPartials] = t;
  }
}

__global__ void subtract_mean(int64_t N, int64_t b, double* __restrict__ v, const double* __restrict__ total) {
  const double m = total[0] / double(N);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < N; e += int64_t(gridDim.x) * blockDim.x)
    v[e * b] -= m;
}

// Device address of g_noalloc_scratch, resolved once per device with that
// device current (a host-side reference to the symbol is not a device address).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

ldgmg_status scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    ldgmg_set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return LDGMG_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    ldgmg_set_error("device ordinal out of range for the no-alloc scratch table");
    return LDGMG_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      ldgmg_set_error(std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
      return LDGMG_ECUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return LDGMG_OK;
}

}  // namespace

extern "C" ldgmg_status ldgmg_project_kernel_noalloc(int64_t N, int b, double* v_dev, void* stream) {
  if (!v_dev) {
    ldgmg_set_error("null vector");
    return LDGMG_EINVAL;
  }
  if (N < 1 || b < 1) {
    ldgmg_set_error("N and b must be positive");
    return LDGMG_EINVAL;
  }
  if (N > LDGMG_NOALLOC_MAX_ELEMENTS) {
    ldgmg_set_error("ldgmg_project_kernel_noalloc: N = " + std::to_string(N) + " elements exceeds the maximum " +
                    std::to_string(LDGMG_NOALLOC_MAX_ELEMENTS) + " (use ldgmg_project_kernel)");
    return LDGMG_EINVAL;
  }
  double* scratch = nullptr;
  ldgmg_status s = scratch_for_current_device(&scratch);
  if (s != LDGMG_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nparts = (N + kChunk - 1) / kChunk;
  chunk_sums<<<unsigned(nparts), kThreads, 0, st>>>(N, b, v_dev, scratch);
  total_sum<<<1, kThreads, 0, st>>>(nparts, scratch);
  const int64_t grid = std::min<int64_t>((N + kThreads - 1) / kThreads, 152 * 8);
  subtract_mean<<<unsigned(grid), kThreads, 0, st>>>(N, b, v_dev, scratch + kMaxPartials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ldgmg_set_error(std::string("ldgmg_project_kernel_noalloc launch: ") + cudaGetErrorString(e));
    return LDGMG_ECUDA;
  }
  return LDGMG_OK;
}
