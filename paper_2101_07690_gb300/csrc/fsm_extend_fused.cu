// fsm_extend_fused.cu -- instantiations of the extension kernel for PASS_FUSED, the one-pass last
// level (levels of size 1..5 are extended: its packed pattern codes hold up to seven vertices).
#include "fsm_extend.cuh"

namespace fsm {

cudaError_t launch_extend_fused(int L, const ExtArgs &A, int grid, cudaStream_t st) {
    switch (L) {
    case 1: extend_kernel<1, PASS_FUSED><<<grid, 256, sizeof(CountCache), st>>>(A); break;
    case 2: extend_kernel<2, PASS_FUSED><<<grid, 256, sizeof(CountCache), st>>>(A); break;
    case 3: extend_kernel<3, PASS_FUSED><<<grid, 256, sizeof(CountCache), st>>>(A); break;
    case 4: extend_kernel<4, PASS_FUSED><<<grid, 256, sizeof(CountCache), st>>>(A); break;
    case 5: extend_kernel<5, PASS_FUSED><<<grid, 256, sizeof(CountCache), st>>>(A); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t occupancy_extend_fused(int L, int *blocks_per_sm) {
    switch (L) {
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<1, PASS_FUSED>, 256, sizeof(CountCache));
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<2, PASS_FUSED>, 256, sizeof(CountCache));
    case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<3, PASS_FUSED>, 256, sizeof(CountCache));
    case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<4, PASS_FUSED>, 256, sizeof(CountCache));
    case 5: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, extend_kernel<5, PASS_FUSED>, 256, sizeof(CountCache));
    default: return cudaErrorInvalidValue;
    }
}

} // namespace fsm
