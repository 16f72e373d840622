// fsm_extend_quota.cu -- two-vertex exploration with Section 5's sampling quotas (a fixed number
// of candidate pieces per key group when joining, of edges per key vertex when an edge list is
// joined, of candidates per vertex when size-3 subgraphs are matched).  Levels of size 1..7
// (k <= 9; Section 6 mines 9-vertex patterns this way).
#include "fsm_extend_variant.cuh"

namespace fsm {

cudaError_t launch_extend_quota(int pass, int L, const ExtArgs &A, int grid, cudaStream_t st) {
    return launch_variant<FSM_EXPLORE_TV_QUOTA, 7>(pass, L, A, grid, st);
}

cudaError_t occupancy_extend_quota(int pass, int L, int *blocks_per_sm) {
    return occupancy_variant<FSM_EXPLORE_TV_QUOTA, 7>(pass, L, blocks_per_sm);
}

} // namespace fsm
