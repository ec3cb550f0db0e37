// sha3_ragged.cu -- ragged batches: messages of any lengths and any mix of
// the six variants in one call (the batch mode of Section 4 with the paper's
// equal-length restriction of Section 4.3 lifted).
//
// Three schedules, chosen by KB_TUNE_RAGGED_SCHEDULE:
//  * the cost-bucketed persistent work queue of sha3_queue.cu (default), with
//    one thread per message or, in its lane-parallel form, one warp per
//    message;
//  * input order, kept as the plain one-launch control: digest offsets by an
//    exclusive prefix sum of out_lens (three small kernels), then one thread
//    per message in a grid-stride loop.
#include <cuda_runtime.h>

#include "keccak_core.cuh"
#include "queue_host.h"
#include "runtime.cuh"
#include "scan.cuh"
#include "sponge.cuh"

namespace kb {
namespace {

__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const uint32_t *__restrict__ out_lens, uint64_t n,
                                                            uint64_t *__restrict__ tile_sums) {
    const uint64_t base = uint64_t(blockIdx.x) * kScanTile + uint64_t(threadIdx.x) * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < n) s += out_lens[base + j];
    uint64_t excl;
    const uint64_t total = block_exclusive_scan(s, excl);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block: exclusive scan of the tile sums in place.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(uint64_t *tile_sums, uint64_t ntiles) {
    uint64_t carry = 0;
    for (uint64_t start = 0; start < ntiles; start += kScanThreads) {
        const uint64_t i = start + threadIdx.x;
        const uint64_t v = i < ntiles ? tile_sums[i] : 0;
        uint64_t excl;
        const uint64_t total = block_exclusive_scan(v, excl);
        if (i < ntiles) tile_sums[i] = carry + excl;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_apply_scan(const uint32_t *__restrict__ out_lens, uint64_t n,
                                                             const uint64_t *__restrict__ tile_sums,
                                                             uint64_t *__restrict__ out_off) {
    const uint64_t base = uint64_t(blockIdx.x) * kScanTile + uint64_t(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < n ? out_lens[base + j] : 0u;
        s += v[j];
    }
    uint64_t excl;
    block_exclusive_scan(s, excl);
    uint64_t acc = tile_sums[blockIdx.x] + excl;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out_off[base + j] = acc;
        acc += v[j];
    }
}

// One thread per message, in input order.
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_sha3_ragged(const uint8_t *__restrict__ msgs, const uint64_t *__restrict__ offsets,
                  const uint64_t *__restrict__ lens, const uint8_t *__restrict__ variants,
                  const uint32_t *__restrict__ out_lens, const uint64_t *__restrict__ out_off,
                  uint8_t *__restrict__ digests, uint64_t n, unsigned int *status) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step)
        hash_ragged_message(msgs, offsets, lens, variants, out_lens, out_off, digests, i, status);
}

}  // namespace

int launch_digest_offsets(const uint32_t *out_lens, uint64_t n, uint64_t *out_off, uint64_t *tile_sums,
                          cudaStream_t stream) {
    const uint64_t ntiles = (n + kScanTile - 1) / kScanTile;
    k_tile_sums<<<unsigned(ntiles), kScanThreads, 0, stream>>>(out_lens, n, tile_sums);
    k_scan_tiles<<<1, kScanThreads, 0, stream>>>(tile_sums, ntiles);
    k_apply_scan<<<unsigned(ntiles), kScanThreads, 0, stream>>>(out_lens, n, tile_sums, out_off);
    return cuda_status(cudaGetLastError());
}

uint64_t digest_offsets_tiles(uint64_t n) { return (n + kScanTile - 1) / kScanTile; }

int launch_ragged(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                  const uint32_t *out_lens, uint8_t *digests, uint64_t n, cudaStream_t stream,
                  const DeviceInfo &dev) {
    if (tuning_get(KB_TUNE_RAGGED_SCHEDULE) != KB_SCHEDULE_INPUT_ORDER)
        return launch_ragged_queue(msgs, offsets, lens, variants, out_lens, digests, n, stream, dev);
    // Input order: one thread per message, grid-stride.
    const uint64_t ntiles = digest_offsets_tiles(n);
    int err = KB_OK;
    uint8_t *scratch = static_cast<uint8_t *>(stream_scratch(stream, size_t(8 * (n + ntiles)), &err));
    if (!scratch) return err;
    uint64_t *out_off = reinterpret_cast<uint64_t *>(scratch);
    uint64_t *tile_sums = out_off + n;
    if ((err = launch_digest_offsets(out_lens, n, out_off, tile_sums, stream)) != KB_OK) return err;
    const void *fn = reinterpret_cast<const void *>(&k_sha3_ragged);
    const uint64_t grid = persistent_grid(fn, kThreads, 0, n, dev);
    k_sha3_ragged<<<unsigned(grid), kThreads, 0, stream>>>(msgs, offsets, lens, variants, out_lens, out_off,
                                                           digests, n, dev.d_status);
    return cuda_status(cudaGetLastError());
}

}  // namespace kb
