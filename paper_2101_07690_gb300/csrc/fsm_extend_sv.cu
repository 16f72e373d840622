// fsm_extend_sv.cu -- single-vertex exploration (l -> l+1) instantiations of the extension
// kernel: the ablation of Section 6 that two-vertex exploration is measured against.  Levels
// of size 1..6 are extended (k <= 7).
#include "fsm_extend_variant.cuh"

namespace fsm {

cudaError_t launch_extend_sv(int pass, int L, const ExtArgs &A, int grid, cudaStream_t st) {
    return launch_variant<FSM_EXPLORE_SV, 6>(pass, L, A, grid, st);
}

cudaError_t occupancy_extend_sv(int pass, int L, int *blocks_per_sm) {
    return occupancy_variant<FSM_EXPLORE_SV, 6>(pass, L, blocks_per_sm);
}

} // namespace fsm
