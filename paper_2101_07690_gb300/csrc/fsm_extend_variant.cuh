// fsm_extend_variant.cuh -- launch and occupancy switches of one exploration variant of the
// extension kernel (the ablations of Section 6), for its count, domain and emit passes.
#pragma once
#include "fsm_extend.cuh"

namespace fsm {

template <int PASS, int V, int MAXL>
cudaError_t launch_variant_pass(int L, const ExtArgs &A, int grid, cudaStream_t st) {
    const size_t smem = PASS == PASS_COUNT ? FSM_COUNT_SMEM : 0;
    switch (L) {
    case 1: extend_kernel<1, PASS, V><<<grid, 256, smem, st>>>(A); break;
    case 2: extend_kernel<2, PASS, V><<<grid, 256, smem, st>>>(A); break;
    case 3: extend_kernel<3, PASS, V><<<grid, 256, smem, st>>>(A); break;
    case 4: extend_kernel<4, PASS, V><<<grid, 256, smem, st>>>(A); break;
    case 5: extend_kernel<5, PASS, V><<<grid, 256, smem, st>>>(A); break;
    case 6:
        if constexpr (MAXL >= 6) { extend_kernel<6, PASS, V><<<grid, 256, smem, st>>>(A); break; }
        return cudaErrorInvalidValue;
    case 7:   // a size-9 level is the last one: no emission pass
        if constexpr (MAXL >= 7 && PASS != PASS_EMIT) { extend_kernel<7, PASS, V><<<grid, 256, smem, st>>>(A); break; }
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int PASS, int V, int MAXL>
cudaError_t occupancy_variant_pass(int L, int *bps) {
    const size_t smem = PASS == PASS_COUNT ? FSM_COUNT_SMEM : 0;
    switch (L) {
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, extend_kernel<1, PASS, V>, 256, smem);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, extend_kernel<2, PASS, V>, 256, smem);
    case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, extend_kernel<3, PASS, V>, 256, smem);
    case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, extend_kernel<4, PASS, V>, 256, smem);
    case 5: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, extend_kernel<5, PASS, V>, 256, smem);
    case 6:
        if constexpr (MAXL >= 6) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, extend_kernel<6, PASS, V>, 256, smem);
        return cudaErrorInvalidValue;
    case 7:
        if constexpr (MAXL >= 7 && PASS != PASS_EMIT)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, extend_kernel<7, PASS, V>, 256, smem);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int V, int MAXL>
cudaError_t launch_variant(int pass, int L, const ExtArgs &A, int grid, cudaStream_t st) {
    switch (pass) {
    case PASS_COUNT: return launch_variant_pass<PASS_COUNT, V, MAXL>(L, A, grid, st);
    case PASS_DOMAIN: return launch_variant_pass<PASS_DOMAIN, V, MAXL>(L, A, grid, st);
    case PASS_EMIT: return launch_variant_pass<PASS_EMIT, V, MAXL>(L, A, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int V, int MAXL>
cudaError_t occupancy_variant(int pass, int L, int *bps) {
    switch (pass) {
    case PASS_COUNT: return occupancy_variant_pass<PASS_COUNT, V, MAXL>(L, bps);
    case PASS_DOMAIN: return occupancy_variant_pass<PASS_DOMAIN, V, MAXL>(L, bps);
    case PASS_EMIT: return occupancy_variant_pass<PASS_EMIT, V, MAXL>(L, bps);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace fsm
