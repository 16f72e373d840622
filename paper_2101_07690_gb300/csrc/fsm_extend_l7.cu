// fsm_extend_l7.cu -- the extension kernel from stored size-7 embeddings to size 9 (two-vertex
// exploration, index-based quick patterns): the count and domain passes of the last level of
// 9-vertex mining (Section 6 mines 9-vertex patterns).  A size-9 level is always the last, so
// there is no emission pass.  Its own translation unit keeps the parallel build balanced.
#include "fsm_extend.cuh"

namespace fsm {

cudaError_t launch_extend_l7(int pass, const ExtArgs &A, int grid, cudaStream_t st) {
    switch (pass) {
    case PASS_COUNT: extend_kernel<7, PASS_COUNT><<<grid, 256, FSM_COUNT_SMEM, st>>>(A); break;
    case PASS_DOMAIN: extend_kernel<7, PASS_DOMAIN><<<grid, 256, 0, st>>>(A); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t occupancy_extend_l7(int pass, int *blocks_per_sm) {
    switch (pass) {
    case PASS_COUNT:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<7, PASS_COUNT>, 256, FSM_COUNT_SMEM);
    case PASS_DOMAIN:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<7, PASS_DOMAIN>, 256, 0);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace fsm
