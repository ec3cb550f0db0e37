// runtime.cuh -- host-side runtime shared by the library's translation units:
// per-device state (SM count, the device status word), per-stream scratch
// arenas, and the launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>

#include "../../include/sha3gb.h"

namespace kb {

// NVTX range for the host side of an entry point (visible in Nsight tools;
// free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Threads per block of the thread-per-message kernels.
constexpr int kThreads = 128;
// Minimum resident blocks per SM asked of ptxas for the sponge kernels: caps
// them at 128 registers per thread (16 warps per SM).
constexpr int kMinBlocks = 4;

struct DeviceInfo {
    int device = -1;
    int sm_count = 0;
    unsigned int *d_status = nullptr;  // device status word (KB_DEV_* bits)
};

// State of the calling thread's current device, created on first use.
// Returns nullptr (and sets *err) when the CUDA runtime fails.
DeviceInfo *device_info(int *err);

// A scratch arena cached per (device, stream): returns at least `bytes` of
// device memory reserved for work enqueued on `stream`.  Growing the arena
// synchronises the stream before the old block is freed.
void *stream_scratch(cudaStream_t stream, size_t bytes, int *err);

// Frees all cached state of the current device.
void release_device();

// Blocks of `threads` that keep every SM busy for kernel `fn` (occupancy x SMs),
// capped by the number of blocks the work needs.
uint64_t persistent_grid(const void *fn, int threads, size_t smem, uint64_t work_items,
                         const DeviceInfo &dev);

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? KB_OK : KB_ERR_CUDA; }

// Process-wide tuning knobs (kb_tune_key values of sha3gb.h).
int64_t tuning_get(int key);
int tuning_set(int key, int64_t value);

// Launchers (one per translation unit of kernels).
int launch_uniform(const uint8_t *msgs, uint64_t stride, uint64_t len, int variant, uint32_t out_len,
                   uint8_t *digests, uint64_t n, cudaStream_t stream, const DeviceInfo &dev);
int launch_ragged(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                  const uint32_t *out_lens, uint8_t *digests, uint64_t n, cudaStream_t stream,
                  const DeviceInfo &dev);
uint64_t digest_offsets_tiles(uint64_t n);
int launch_digest_offsets(const uint32_t *out_lens, uint64_t n, uint64_t *out_off, uint64_t *tile_sums,
                          cudaStream_t stream);
// Streaming states (stream.cu).
int launch_stream_init(uint8_t *states, const uint8_t *variants, uint64_t n, cudaStream_t stream,
                       const DeviceInfo &dev);
int launch_stream_absorb(uint8_t *states, const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                         uint64_t n, cudaStream_t stream, const DeviceInfo &dev);
int launch_stream_final(uint8_t *states, const uint32_t *out_lens, uint8_t *digests, uint64_t n,
                        cudaStream_t stream, const DeviceInfo &dev);
// One fused step: optionally start from fresh states (init, variants read),
// absorb a piece (msgs may be null for none), optionally pad and squeeze
// (final_, outputs at the exclusive scan of out_lens).
int launch_stream_step(bool init, bool final_, uint8_t *states, const uint8_t *variants, const uint8_t *msgs,
                       const uint64_t *offsets, const uint64_t *lens, const uint32_t *out_lens, uint8_t *digests,
                       uint64_t n, cudaStream_t stream, const DeviceInfo &dev);
// The cost-bucketed persistent path is declared in queue_host.h.
uint64_t merkle_nodes(uint64_t n_leaves);
int launch_merkle_levels(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes, uint8_t *nodes,
                         cudaStream_t stream, const DeviceInfo &dev);
uint64_t merkle_message_leaves(uint64_t len, uint64_t chunk_bytes);
int launch_keccak_p(uint64_t *states, int b, int nr, uint64_t n, cudaStream_t stream, const DeviceInfo &dev);
int launch_merkle_many(const uint8_t *buf, uint64_t n_trees, uint64_t leaves_per_tree, uint64_t leaf_bytes,
                       uint8_t *roots, cudaStream_t stream, const DeviceInfo &dev);
int launch_merkle_message(const uint8_t *msg, uint64_t len, uint64_t chunk_bytes, uint8_t *nodes,
                          cudaStream_t stream, const DeviceInfo &dev);

}  // namespace kb
