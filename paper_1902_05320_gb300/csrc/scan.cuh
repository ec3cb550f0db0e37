// scan.cuh -- block-wide exclusive prefix sums shared by the ragged-batch
// bookkeeping kernels (digest offsets, cost-bucket bases).
#pragma once

#include <cstdint>

namespace kb {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t &excl) {
    __shared__ uint64_t warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint64_t s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint64_t before = warp ? warp_sums[warp - 1] : 0;
    const uint64_t total = warp_sums[(blockDim.x >> 5) - 1];
    excl = before + x - v;
    __syncthreads();
    return total;
}

}  // namespace kb
