// capi.cu -- the extern "C" entry points declared in include/sha3gb.h:
// argument checks on the host, dispatch to the kernels, status and constant
// queries (the host-buffer entry points are in host_path.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "host_path.h"
#include "keccak_core.cuh"
#include "queue_host.h"
#include "runtime.cuh"

namespace kb {
namespace {

bool valid_out_len(int variant, uint32_t out_len) {
    const int d = variant_digest(variant);
    return d == 0 || out_len == uint32_t(d);
}

// Checks that (n-1)*stride + len and n*out_len fit in 64 bits.
bool sizes_fit(uint64_t stride, uint64_t len, uint32_t out_len, uint64_t n) {
    if (n == 0) return true;
    if (stride != 0 && (n - 1) > (UINT64_MAX - len) / stride) return false;
    if (out_len != 0 && n > UINT64_MAX / out_len) return false;
    return true;
}

}  // namespace
}  // namespace kb

using namespace kb;

extern "C" {

int keccak_batch_uniform(const uint8_t *msgs, uint64_t stride, uint64_t len, int variant,
                         uint32_t out_len, uint8_t *digests, uint64_t n, void *stream) {
    if (variant < 0 || variant > 5 || !valid_out_len(variant, out_len)) return KB_ERR_INVALID;
    if (n == 0) return KB_OK;
    if ((len > 0 && !msgs) || (out_len > 0 && !digests) || !sizes_fit(stride, len, out_len, n))
        return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_batch_uniform");
    return launch_uniform(msgs, stride, len, variant, out_len, digests, n,
                          static_cast<cudaStream_t>(stream), *dev);
}

int keccak_batch(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                 const uint8_t *variant, const uint32_t *out_lens, uint8_t *digests,
                 uint64_t n, void *stream) {
    if (n == 0) return KB_OK;
    if (!msgs || !offsets || !lens || !variant || !out_lens || !digests) return KB_ERR_INVALID;
    if (n > UINT32_MAX) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_batch");
    return launch_ragged(msgs, offsets, lens, variant, out_lens, digests, n,
                         static_cast<cudaStream_t>(stream), *dev);
}

int keccak_batch_autotune_ex(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                             const uint8_t *variant, const uint32_t *out_lens, uint8_t *digests, uint64_t n,
                             void *stream, kb_queue_config *chosen) {
    if (n == 0) return KB_OK;
    if (!msgs || !offsets || !lens || !variant || !out_lens || !digests) return KB_ERR_INVALID;
    if (n > UINT32_MAX) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_batch_autotune");
    QueueConfig best;
    const int rc = autotune_ragged_queue(msgs, offsets, lens, variant, out_lens, digests, n,
                                         static_cast<cudaStream_t>(stream), *dev, &best);
    if (rc == KB_OK && chosen) {
        chosen->min_blocks = best.minb;
        chosen->blocks_per_sm = best.blocks_per_sm;
        chosen->staging = queue_staging_value(best);
        chosen->warp_messages = best.warp_messages;
        chosen->ms = best.ms;
    }
    return rc;
}

int keccak_batch_autotune(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                          const uint8_t *variant, const uint32_t *out_lens, uint8_t *digests, uint64_t n,
                          void *stream, int64_t *chosen_min_blocks, int64_t *chosen_blocks_per_sm,
                          float *ms) {
    kb_queue_config cfg{};
    const int rc = keccak_batch_autotune_ex(msgs, offsets, lens, variant, out_lens, digests, n, stream, &cfg);
    if (rc == KB_OK && n) {
        if (chosen_min_blocks) *chosen_min_blocks = cfg.min_blocks;
        if (chosen_blocks_per_sm) *chosen_blocks_per_sm = cfg.blocks_per_sm;
        if (ms) *ms = cfg.ms;
    }
    return rc;
}

int keccak_tuned_config_ex(uint64_t n, kb_queue_config *cfg) {
    if (!cfg) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    const QueueConfig c = queue_config_for(n, *dev);
    cfg->min_blocks = c.minb;
    cfg->blocks_per_sm = c.blocks_per_sm;
    cfg->staging = queue_staging_value(c);
    cfg->warp_messages = c.warp_messages;
    cfg->ms = 0;
    return KB_OK;
}

int keccak_tuned_config(uint64_t n, int64_t *min_blocks, int64_t *blocks_per_sm) {
    kb_queue_config cfg{};
    const int rc = keccak_tuned_config_ex(n, &cfg);
    if (rc != KB_OK) return rc;
    if (min_blocks) *min_blocks = cfg.min_blocks;
    if (blocks_per_sm) *blocks_per_sm = cfg.blocks_per_sm;
    return KB_OK;
}

uint64_t merkle_node_count(uint64_t n_leaves) { return merkle_nodes(n_leaves); }

int merkle_sha3_256_levels(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes,
                           uint8_t *nodes, void *stream) {
    if (n_leaves == 0 || leaf_bytes == 0 || !buf || !nodes) return KB_ERR_INVALID;
    if (n_leaves > UINT64_MAX / leaf_bytes || n_leaves > (UINT64_MAX >> 7)) return KB_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(nodes) & 31) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("merkle_sha3_256_levels");
    return launch_merkle_levels(buf, n_leaves, leaf_bytes, nodes, static_cast<cudaStream_t>(stream), *dev);
}

int merkle_sha3_256(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes, uint8_t *root,
                    void *stream) {
    if (n_leaves == 0 || leaf_bytes == 0 || !buf || !root) return KB_ERR_INVALID;
    if (n_leaves > UINT64_MAX / leaf_bytes || n_leaves > (UINT64_MAX >> 7)) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("merkle_sha3_256");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t total = merkle_nodes(n_leaves);
    uint8_t *nodes = static_cast<uint8_t *>(stream_scratch(s, size_t(32 * total), &err));
    if (!nodes) return err;
    if ((err = launch_merkle_levels(buf, n_leaves, leaf_bytes, nodes, s, *dev)) != KB_OK) return err;
    if (cudaMemcpyAsync(root, nodes + 32 * (total - 1), 32, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return KB_ERR_CUDA;
    return KB_OK;
}

int merkle_sha3_256_many(const uint8_t *buf, uint64_t n_trees, uint64_t leaves_per_tree, uint64_t leaf_bytes,
                         uint8_t *roots, void *stream) {
    if (n_trees == 0) return KB_OK;
    if (!buf || !roots || leaves_per_tree == 0 || leaf_bytes == 0) return KB_ERR_INVALID;
    if (leaves_per_tree >= (uint64_t(1) << 39)) return KB_ERR_INVALID;
    if (leaves_per_tree > UINT64_MAX / leaf_bytes || n_trees > UINT64_MAX / (leaves_per_tree * leaf_bytes))
        return KB_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(roots) & 15) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("merkle_sha3_256_many");
    return launch_merkle_many(buf, n_trees, leaves_per_tree, leaf_bytes, roots, static_cast<cudaStream_t>(stream),
                              *dev);
}

int merkle_sha3_256_message(const uint8_t *msg, uint64_t len, uint64_t chunk_bytes, uint8_t *root, void *stream) {
    if (chunk_bytes == 0 || !root || (len > 0 && !msg)) return KB_ERR_INVALID;
    const uint64_t n = merkle_message_leaves(len, chunk_bytes);
    if (n > (UINT64_MAX >> 7)) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("merkle_sha3_256_message");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t total = merkle_nodes(n);
    uint8_t *nodes = static_cast<uint8_t *>(stream_scratch(s, size_t(32 * total), &err));
    if (!nodes) return err;
    if ((err = launch_merkle_message(msg, len, chunk_bytes, nodes, s, *dev)) != KB_OK) return err;
    if (cudaMemcpyAsync(root, nodes + 32 * (total - 1), 32, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return KB_ERR_CUDA;
    return KB_OK;
}

int keccak_stream_init(uint8_t *states, const uint8_t *variant, uint64_t n, void *stream) {
    if (n == 0) return KB_OK;
    if (!states || !variant || n > UINT64_MAX / KB_STATE_BYTES) return KB_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(states) & 7) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_stream_init");
    return launch_stream_init(states, variant, n, static_cast<cudaStream_t>(stream), *dev);
}

int keccak_stream_absorb(uint8_t *states, const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                         uint64_t n, void *stream) {
    if (n == 0) return KB_OK;
    if (!states || !msgs || !offsets || !lens || n > UINT64_MAX / KB_STATE_BYTES) return KB_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(states) & 7) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_stream_absorb");
    return launch_stream_absorb(states, msgs, offsets, lens, n, static_cast<cudaStream_t>(stream), *dev);
}

int keccak_stream_final(uint8_t *states, const uint32_t *out_lens, uint8_t *digests, uint64_t n, void *stream) {
    if (n == 0) return KB_OK;
    if (!states || !out_lens || !digests || n > UINT32_MAX) return KB_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(states) & 7) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_stream_final");
    return launch_stream_final(states, out_lens, digests, n, static_cast<cudaStream_t>(stream), *dev);
}

int keccak_stream_init_absorb(uint8_t *states, const uint8_t *variant, const uint8_t *msgs, const uint64_t *offsets,
                              const uint64_t *lens, uint64_t n, void *stream) {
    if (n == 0) return KB_OK;
    if (!states || !variant || !msgs || !offsets || !lens || n > UINT64_MAX / KB_STATE_BYTES) return KB_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(states) & 7) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_stream_init_absorb");
    return launch_stream_step(true, false, states, variant, msgs, offsets, lens, nullptr, nullptr, n,
                              static_cast<cudaStream_t>(stream), *dev);
}

int keccak_stream_absorb_final(uint8_t *states, const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                               const uint32_t *out_lens, uint8_t *digests, uint64_t n, void *stream) {
    if (n == 0) return KB_OK;
    if (!states || !msgs || !offsets || !lens || !out_lens || !digests || n > UINT32_MAX) return KB_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(states) & 7) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_stream_absorb_final");
    return launch_stream_step(false, true, states, nullptr, msgs, offsets, lens, out_lens, digests, n,
                              static_cast<cudaStream_t>(stream), *dev);
}

int keccak_p_batch(uint64_t *states, int b, int nr, uint64_t n, void *stream) {
    if (nr < 0 || nr > 1000000) return KB_ERR_INVALID;
    bool width_ok = false;
    for (int k = 0; k <= 6; ++k) width_ok = width_ok || b == 25 * (1 << k);
    if (!width_ok) return KB_ERR_INVALID;
    if (n == 0 || nr == 0) return KB_OK;
    if (!states || (reinterpret_cast<uintptr_t>(states) & 7) || n > UINT64_MAX / 200) return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_p_batch");
    return launch_keccak_p(states, b, nr, n, static_cast<cudaStream_t>(stream), *dev);
}

int keccak_last_error(void *stream) {
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return KB_ERR_CUDA;
    unsigned int word = 0;
    if (cudaMemcpy(&word, dev->d_status, sizeof word, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(dev->d_status, 0, sizeof word) != cudaSuccess)
        return KB_ERR_CUDA;
    return int(word & 0x7fffffffu);
}

void keccak_release(void) {
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceSynchronize();
        release_queue_graphs(dev);
        forget_tuning(dev);
        forget_noalloc_setup();
        release_host_pipeline(dev);
    }
    release_device();
}

int sha3gb_round_constants(uint64_t *rc24) {
    if (!rc24) return KB_ERR_INVALID;
    for (int i = 0; i < 24; ++i) rc24[i] = round_constant(i);
    return KB_OK;
}

int sha3gb_rho_offsets(uint32_t *rho25) {
    if (!rho25) return KB_ERR_INVALID;
    for (int i = 0; i < 25; ++i) rho25[i] = uint32_t(rho_offset(i));
    return KB_OK;
}

int keccak_tune_set(int key, int64_t value) { return tuning_set(key, value); }

int64_t keccak_tune_get(int key) { return tuning_get(key); }

const char *sha3gb_version(void) { return "sha3gb 0.1.0 (sm_103a)"; }

}  // extern "C"
