// fsm_extend_count.cu -- instantiations of the extension kernel for PASS_COUNT.
#include "fsm_extend.cuh"

namespace fsm {

cudaError_t launch_extend_count(int L, int V, const ExtArgs &A, int grid, cudaStream_t st) {
    if (V == FSM_EXPLORE_SV) return launch_extend_sv(PASS_COUNT, L, A, grid, st);
    if (V == FSM_EXPLORE_TV_EDGELIST) return launch_extend_edgelist(PASS_COUNT, L, A, grid, st);
    if (V == FSM_EXPLORE_TV_QUOTA) return launch_extend_quota(PASS_COUNT, L, A, grid, st);
    switch (L) {
    case 1: extend_kernel<1, PASS_COUNT><<<grid, 256, FSM_COUNT_SMEM, st>>>(A); break;
    case 2: extend_kernel<2, PASS_COUNT><<<grid, 256, FSM_COUNT_SMEM, st>>>(A); break;
    case 3: extend_kernel<3, PASS_COUNT><<<grid, 256, FSM_COUNT_SMEM, st>>>(A); break;
    case 4: extend_kernel<4, PASS_COUNT><<<grid, 256, FSM_COUNT_SMEM, st>>>(A); break;
    case 5: extend_kernel<5, PASS_COUNT><<<grid, 256, FSM_COUNT_SMEM, st>>>(A); break;
    case 6: extend_kernel<6, PASS_COUNT><<<grid, 256, FSM_COUNT_SMEM, st>>>(A); break;
    case 7: return launch_extend_l7(PASS_COUNT, A, grid, st);
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t occupancy_extend_count(int L, int V, int *blocks_per_sm) {
    if (V == FSM_EXPLORE_SV) return occupancy_extend_sv(PASS_COUNT, L, blocks_per_sm);
    if (V == FSM_EXPLORE_TV_EDGELIST) return occupancy_extend_edgelist(PASS_COUNT, L, blocks_per_sm);
    if (V == FSM_EXPLORE_TV_QUOTA) return occupancy_extend_quota(PASS_COUNT, L, blocks_per_sm);
    switch (L) {
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<1, PASS_COUNT>, 256, FSM_COUNT_SMEM);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<2, PASS_COUNT>, 256, FSM_COUNT_SMEM);
    case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<3, PASS_COUNT>, 256, FSM_COUNT_SMEM);
    case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<4, PASS_COUNT>, 256, FSM_COUNT_SMEM);
    case 5: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<5, PASS_COUNT>, 256, FSM_COUNT_SMEM);
    case 6: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<6, PASS_COUNT>, 256, FSM_COUNT_SMEM);
    case 7: return occupancy_extend_l7(PASS_COUNT, blocks_per_sm);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace fsm
