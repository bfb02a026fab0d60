// Block- and warp-level building blocks of the radix passes (sort.cu and
// bucket_sort.cu): a block-wide exclusive scan and the warp-level multisplit
// of 8-bit digits by ballots.
#pragma once

#include <stdint.h>

namespace hc {

// Exclusive scan of one value per thread over a block of NW warps; warp_sums
// holds NW words of shared memory and ends with the inclusive warp totals.
template <int NW>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) warp_sums[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t before = warp ? warp_sums[warp - 1] : 0u;
    __syncthreads();  // warp_sums may be reused by the caller
    return before + x - v;
}

// Lanes of the warp whose 8-bit digit equals this lane's (warp-level
// multisplit by ballots, one per digit bit).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

}  // namespace hc
