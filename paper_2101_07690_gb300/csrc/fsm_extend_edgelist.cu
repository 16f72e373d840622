// fsm_extend_edgelist.cu -- two-vertex exploration with edge-list quick patterns: the ablation
// of Section 6 that index-based quick patterns are measured against.  The 64-bit edge-list key
// holds up to seven vertices, so levels of size 1..5 are extended (k <= 7).
#include "fsm_extend_variant.cuh"

namespace fsm {

cudaError_t launch_extend_edgelist(int pass, int L, const ExtArgs &A, int grid, cudaStream_t st) {
    return launch_variant<FSM_EXPLORE_TV_EDGELIST, 5>(pass, L, A, grid, st);
}

cudaError_t occupancy_extend_edgelist(int pass, int L, int *blocks_per_sm) {
    return occupancy_variant<FSM_EXPLORE_TV_EDGELIST, 5>(pass, L, blocks_per_sm);
}

} // namespace fsm
