// queue_host.h -- host-side interface of the ragged-batch work queue
// (sha3_queue.cu): its configuration, its launch sequence on caller-owned
// scratch, and the autotuner.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "runtime.cuh"

namespace kb {

// One configuration of the queue schedule (the dimensions the autotuner
// searches).  stage is a kStage* value of queue.cuh.
struct QueueConfig {
    int minb = 2;               // register budget: blocks of 128 threads per SM compiled for
    int blocks_per_sm = 0;      // blocks per SM of the launch (0: as many as fit)
    int stage = 2 | 4;          // how message blocks are read: registers, looped permutation (kStageRegs | kLooped)
    int64_t warp_messages = 0;  // the K costliest messages run one warp each (0: one thread for every message)
    bool lanes = false;         // control: every message one warp
    bool per_variant = false;   // control: one launch per variant, unsorted
    float ms = 0;               // the autotuner's time for this configuration
};

// The hybrid splits the autotuner tries on its best one-thread-per-message
// configuration: one warp each for the 32 or the 608 (4 per SM on 152 SMs)
// costliest messages.
constexpr int64_t kHybridChoices[] = {32, 608};

// Side stream and fork/join events of the hybrid schedule for one stream.
struct AuxStream {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

// Device scratch of one call for n messages: the queue's control block, the
// digest offsets (8 B per message), the scan's tile sums and the work order
// (4 B per message).
size_t queue_scratch_bytes(uint64_t n);

// Whether the configuration names a compiled kernel.
bool queue_config_valid(const QueueConfig &cfg);

// Blocks of the hashing launch for n messages on a device of sm_count SMs
// (occupancy queried once per kernel and device).
uint64_t queue_grid_for(const QueueConfig &cfg, uint64_t n, int device, int sm_count);

// Enqueues the whole pipeline on `stream` using `scratch`
// (queue_scratch_bytes(n) bytes, 256-byte aligned): no allocation, no
// synchronisation.  status is the device status word per-message errors go
// to; aux is required when cfg.warp_messages > 0.
int queue_issue(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                const uint32_t *out_lens, uint8_t *digests, uint64_t n, uint8_t *scratch, const QueueConfig &cfg,
                uint64_t grid, int sm_count, unsigned int *status, cudaStream_t stream, const AuxStream *aux);

// keccak_batch's queue path: configuration from knobs, tuned entries and the
// cache file; graph capture and replay.
int launch_ragged_queue(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                        const uint32_t *out_lens, uint8_t *digests, uint64_t n, cudaStream_t stream,
                        const DeviceInfo &dev);

// The autotuner; writes the chosen configuration (with its time) to *chosen
// when not null.
int autotune_ragged_queue(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                          const uint32_t *out_lens, uint8_t *digests, uint64_t n, cudaStream_t stream,
                          const DeviceInfo &dev, QueueConfig *chosen);

// The tuning knobs applied over a configuration.
void apply_knobs(QueueConfig &cfg);

// The configuration keccak_batch would use for n messages on this device.
QueueConfig queue_config_for(uint64_t n, const DeviceInfo &dev);

// The KB_QUEUE_STAGING_* value of a configuration.
int queue_staging_value(const QueueConfig &cfg);

void release_queue_graphs(int device);
void forget_tuning(int device);
// keccak_batch_noalloc: forget the cached device address of its array.
void forget_noalloc_setup();

}  // namespace kb
