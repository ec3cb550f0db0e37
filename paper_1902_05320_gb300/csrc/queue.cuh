// queue.cuh -- device side of the cost-bucketed work queue for ragged batches
// (the batch mode of Section 4 for messages of mixed lengths and variants),
// shared by the translation units that instantiate its kernels.
//
// A message's cost is its number of Keccak-f permutations: floor(len/r) + 1
// absorbed blocks plus ceil(d/r) - 1 extra squeezes.  Costs fall into cost
// buckets (exact below 64, 32 per octave above, so the messages of one warp
// differ in cost by at most 1/32; costs of 2^40 and more share the top one),
// and each cost bucket is split by the variant's rate (five rates), so that a
// warp's 32 messages normally share one rate and the absorb can use the
// rate's compile-time form.  The work order lists the buckets longest first.
//   1. k_prep: digest-offset tile sums and a bucket histogram;
//   2. k_plan: one block scans the tile sums, lays the buckets out longest
//      first and sets the queue heads;
//   3. k_scatter: digest offsets, and each message's slot in the work order;
//   4. k_sha3_queue: a persistent grid; each warp takes a group of 32
//      consecutive entries of the order with one atomic and hashes one
//      message per thread.  Warps run messages of nearly equal cost.  The
//      queue has two ends: on every SM sub-partition the warp in the lowest
//      hardware slot takes groups from the costly end (the longest chains
//      start first), the others from the cheap end.
//   Optionally k_sha3_lanes runs the first K entries of the order (the K
//   costliest messages) one warp per message, concurrently with the queue
//   kernel, which then covers the entries from K on.
//
// Why two ends.  Measured on GB300: when two warps of one sub-partition both
// have ALU work ready, the one in the lower hardware warp slot (%warpid)
// issues, and once blocks are prefetched a warp rarely stalls, so the other
// warp only runs in its partner's gaps.  With one queue end, a long chain of
// permutations that landed in a higher slot waited behind its partner's
// stream of groups and finished milliseconds after everything else.  With two
// ends the long chains go to the slots that issue first, and a warp in a
// higher slot only ever holds a cheap group, which it can finish late without
// a tail.  The order of the slots affects only speed: every group is taken
// exactly once, whichever warp takes it.
#pragma once

#include <cstdint>

#include "../../include/sha3gb.h"
#include "keccak_core.cuh"
#include "lane_parallel.cuh"
#include "runtime.cuh"
#include "scan.cuh"
#include "sponge.cuh"
#include "sponge_staged.cuh"

namespace kb {

constexpr int kBucketsPerOctave = 32;
constexpr int kCostBuckets = 64 + 34 * kBucketsPerOctave;  // costs below 2^40 apart; above, one bucket
constexpr int kRateClasses = 5;                              // rates 72, 104, 136, 144, 168 bytes
constexpr int kBuckets = kCostBuckets * kRateClasses;

// How the queue kernel reads message blocks (low two bits) and whether its
// permutation loops over all 24 rounds (kLooped).
constexpr int kStageDirect = 0;  // each thread loads its block's words when it absorbs them
constexpr int kStageAsync = 1;   // the next block is copied into shared memory during the permutation
constexpr int kStageRegs = 2;    // the next block is loaded into registers before the permutation
constexpr int kLooped = 4;

// Permutations a message costs (0 for an invalid variant, which the hashing
// kernel flags and skips).
__device__ __forceinline__ uint64_t message_cost(uint64_t len, int v, uint32_t dlen) {
    if (v > 5) return 0;
    const uint32_t rate = uint32_t(variant_rate(v));
    return len / rate + 1 + (dlen > rate ? (dlen - 1) / rate : 0);
}

__device__ __forceinline__ uint32_t cost_bucket(uint64_t c) {
    if (c < 64) return uint32_t(c);
    const int e = 63 - __clzll(static_cast<long long>(c));  // >= 6
    if (e >= 40) return uint32_t(kCostBuckets - 1);
    return uint32_t(64 + (e - 6) * kBucketsPerOctave + int((c >> (e - 5)) & (kBucketsPerOctave - 1)));
}

// 0..4 by increasing rate; SHA3-256 and SHAKE256 share a rate.
__device__ __forceinline__ uint32_t rate_class(int v) {
    return v == 3 ? 0u : v == 2 ? 1u : (v == 1 || v == 5) ? 2u : v == 0 ? 3u : 4u;
}

// Bucket of a message: cost bucket x rate class, or (for the per-variant
// control schedule) its variant, 6 standing for an invalid one.
template <bool BY_VARIANT>
__device__ __forceinline__ uint32_t bucket_key(uint64_t len, int v, uint32_t dlen) {
    if constexpr (BY_VARIANT) return v > 5 ? 6u : uint32_t(v);
    else return cost_bucket(message_cost(len, v, dlen)) * kRateClasses + (v > 5 ? 0u : rate_class(v));
}

struct Control {
    uint32_t count[kBuckets];        // messages per bucket
    uint32_t cursor[kBuckets];       // next free slot of each bucket in the order
    unsigned long long head;         // warp-per-message schedule: next entry of the order
    unsigned long long lane_head;    // hybrid: next of the first K entries (one warp each)
    unsigned long long ends;         // queue: groups taken from the back (high 32 bits) and front (low)
    unsigned long long queue_start;  // queue: first entry of the order it covers (K)
};

template <bool BY_VARIANT>
__global__ void __launch_bounds__(kScanThreads)
    k_prep(const uint64_t *__restrict__ lens, const uint8_t *__restrict__ variants,
           const uint32_t *__restrict__ out_lens, uint64_t n, uint64_t *__restrict__ tile_sums, Control *ctl) {
    __shared__ uint32_t hist[kBuckets];
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint64_t base = uint64_t(blockIdx.x) * kScanTile + uint64_t(threadIdx.x) * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint64_t i = base + j;
        if (i < n) {
            const uint32_t d = out_lens[i];
            s += d;
            atomicAdd(&hist[bucket_key<BY_VARIANT>(lens[i], variants[i], d)], 1u);
        }
    }
    uint64_t excl;
    const uint64_t total = block_exclusive_scan(s, excl);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
    __syncthreads();
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x)
        if (hist[b]) atomicAdd(&ctl->count[b], hist[b]);
}

// One block: exclusive scan of the tile sums, bucket starts in descending
// order (bucket kBuckets-1 first), and the queue kernel's first entry.
static __global__ void __launch_bounds__(kScanThreads)
    k_plan(uint64_t *tile_sums, uint64_t ntiles, Control *ctl, uint64_t queue_start) {
    uint64_t carry = 0;
    for (uint64_t start = 0; start < ntiles; start += kScanThreads) {
        const uint64_t i = start + threadIdx.x;
        const uint64_t v = i < ntiles ? tile_sums[i] : 0;
        uint64_t excl;
        const uint64_t total = block_exclusive_scan(v, excl);
        if (i < ntiles) tile_sums[i] = carry + excl;
        carry += total;
    }
    carry = 0;
    for (int start = 0; start < kBuckets; start += kScanThreads) {
        const int t = start + int(threadIdx.x);
        const int b = kBuckets - 1 - t;
        const uint64_t v = t < kBuckets ? ctl->count[b] : 0;
        uint64_t excl;
        const uint64_t total = block_exclusive_scan(v, excl);
        if (t < kBuckets) ctl->cursor[b] = uint32_t(carry + excl);
        carry += total;
    }
    if (threadIdx.x == 0) ctl->queue_start = queue_start;
}

template <bool BY_VARIANT>
__global__ void __launch_bounds__(kScanThreads)
    k_scatter(const uint64_t *__restrict__ lens, const uint8_t *__restrict__ variants,
              const uint32_t *__restrict__ out_lens, uint64_t n, const uint64_t *__restrict__ tile_sums,
              uint64_t *__restrict__ out_off, uint32_t *__restrict__ order, Control *ctl) {
    __shared__ uint32_t hist[kBuckets];
    __shared__ uint32_t start[kBuckets];
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint64_t base = uint64_t(blockIdx.x) * kScanTile + uint64_t(threadIdx.x) * kScanItems;
    uint32_t d[kScanItems], key[kScanItems], rank[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint64_t i = base + j;
        d[j] = 0;
        key[j] = 0;
        rank[j] = 0;
        if (i < n) {
            d[j] = out_lens[i];
            key[j] = bucket_key<BY_VARIANT>(lens[i], variants[i], d[j]);
            rank[j] = atomicAdd(&hist[key[j]], 1u);
        }
        s += d[j];
    }
    uint64_t excl;
    block_exclusive_scan(s, excl);
    uint64_t acc = tile_sums[blockIdx.x] + excl;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out_off[base + j] = acc;
        acc += d[j];
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x)
        start[b] = hist[b] ? atomicAdd(&ctl->cursor[b], hist[b]) : 0u;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < n) order[start[key[j]] + rank[j]] = uint32_t(base + j);
}

// The persistent queue kernel: one thread per message, 32 messages per
// dequeue.  STAGE picks how blocks are read and the permutation's form
// (kStage* | kLooped).
template <int MINB, int STAGE>
__global__ void __launch_bounds__(kThreads, MINB)
    k_sha3_queue(const uint8_t *__restrict__ msgs, const uint64_t *__restrict__ offsets,
                 const uint64_t *__restrict__ lens, const uint8_t *__restrict__ variants,
                 const uint32_t *__restrict__ out_lens, const uint64_t *__restrict__ out_off,
                 const uint32_t *__restrict__ order, uint8_t *__restrict__ digests, uint64_t n, Control *ctl,
                 unsigned int *status) {
    static_assert(kThreads == 128, "the stage layout assumes 128 threads per block");
    constexpr int kRead = STAGE & 3;
    constexpr bool kLoop = (STAGE & kLooped) != 0;
    __shared__ uint32_t stage_mem[kRead == kStageAsync ? 2 * kStageWords * kThreads : 1];
    const int lane = threadIdx.x & 31;
    const uint64_t start = ctl->queue_start;
    const unsigned long long ngroups = n > start ? (n - start + 31) / 32 : 0;
    unsigned slot;
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(slot));
    const bool front = slot < 4;  // the lowest hardware slot of each sub-partition
    for (;;) {
        // One atomic on both ends: group g is taken at most once, from the
        // front (g = f) or the back (g = ngroups - 1 - b), and the two ends
        // never pass each other.
        unsigned long long old = 0;
        if (lane == 0) old = atomicAdd(&ctl->ends, front ? 1ull : (1ull << 32));
        old = __shfl_sync(0xffffffffu, old, 0);
        const unsigned long long f = old & 0xffffffffull, b = old >> 32;
        if (f + b >= ngroups) break;
        const uint64_t idx = start + (front ? f : ngroups - 1 - b) * 32 + lane;
        if (idx < n) {
            if constexpr (STAGE == kStageDirect) {
                hash_ragged_message(msgs, offsets, lens, variants, out_lens, out_off, digests, order[idx], status);
            } else {
                const uint32_t i = order[idx];
                const int v = variants[i];
                const uint32_t dlen = out_lens[i];
                if (v > 5) {
                    atomicOr(status, KB_DEV_BAD_VARIANT);
                } else if (v < 4 && dlen != uint32_t(variant_digest(v))) {
                    atomicOr(status, KB_DEV_BAD_OUTLEN);
                } else if constexpr (kRead == kStageAsync) {
                    const Stage st = make_stage(stage_mem);
                    sponge_rt_staged<kLoop>(st, msgs + offsets[i], lens[i], v, digests + out_off[i], dlen);
                } else if constexpr (kRead == kStageRegs) {
                    sponge_rt_prefetch<kLoop>(msgs + offsets[i], lens[i], v, digests + out_off[i], dlen);
                } else {
                    sponge_rt_direct<kLoop>(msgs + offsets[i], lens[i], v, digests + out_off[i], dlen);
                }
            }
        }
    }
}

// Device scratch of one call for n messages (the layout queue_issue carves):
// the control block, the digest offsets (8 B per message), the digest scan's
// tile sums (8 B per kScanTile messages) and the work order (4 B per
// message), each part 256-byte aligned where it starts a region.
constexpr size_t queue_scratch_size(uint64_t n) {
    return (sizeof(Control) + 255) / 256 * 256 + 8 * n + 8 * ((n + kScanTile - 1) / kScanTile) +
           (4 * n + 255) / 256 * 256;
}

// Kernel entry points of the staged instances (sha3_queue_staged.cu); nullptr
// for a combination that is not compiled.
const void *queue_kernel_staged(int minb, int stage);

}  // namespace kb
