// Grouped solve (group_solve.cuh), the instances for clusters of 1 and 2
// CTAs, and the launcher.  The instances are split over two translation
// units so that the library builds in parallel.
#include "group_solve.cuh"

namespace ldgmg {

cudaError_t group_launch_c48(const GroupProblem* probs, const GroupItem* items, int count, int cluster,
                             cudaStream_t st);

cudaError_t group_solve(const GroupProblem* probs, const GroupItem* items, int count, int cluster, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  cudaError_t e;
  switch (cluster) {
    case 1: e = launch_group<1>(probs, items, count, st); break;
    case 2: e = launch_group<2>(probs, items, count, st); break;
    case 4:
    case 8: e = group_launch_c48(probs, items, count, cluster, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return launched();
}

}  // namespace ldgmg
