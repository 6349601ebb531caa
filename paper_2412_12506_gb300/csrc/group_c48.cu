// Grouped solve (group_solve.cuh), the instances for clusters of 4 and 8 CTAs.
#include "group_solve.cuh"

namespace ldgmg {

cudaError_t group_launch_c48(const GroupProblem* probs, const GroupItem* items, int count, int cluster,
                             cudaStream_t st) {
  return cluster == 4 ? launch_group<4>(probs, items, count, st) : launch_group<8>(probs, items, count, st);
}

}  // namespace ldgmg
