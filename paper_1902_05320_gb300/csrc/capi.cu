// capi.cu -- the extern "C" entry points declared in include/sha3gb.h:
// argument checks on the host, dispatch to the kernels, the pipelined
// host-buffer path, status and constant queries.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "host_chunks.h"
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

// Device address of a host buffer the GPU can access (page-locked memory),
// or nullptr for pageable memory.
const void *device_view(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged) return a.devicePointer;
    return nullptr;
}

// ---- host-buffer pipeline ---------------------------------------------------
// Three streams, one per role: copies in, hashing, copies out.  A chunk's
// buffers are reused kStages chunks later; events order each reuse after the
// work that last read or wrote the buffer, and nothing else, so the copies
// in run back to back whatever the copies out are doing (a stream per chunk
// slot would queue a chunk's copy in behind an earlier chunk's copy out).
constexpr int kStages = 4;

struct Pipeline {
    cudaStream_t in = nullptr, hash = nullptr, out = nullptr;
    uint8_t *d_in[kStages] = {};
    uint8_t *d_out[kStages] = {};
    cudaEvent_t copied[kStages] = {};   // the copy into d_in[s] is done
    cudaEvent_t hashed[kStages] = {};   // the hashing of d_in[s] into d_out[s] is done
    cudaEvent_t drained[kStages] = {};  // the copy out of d_out[s] is done
    size_t in_bytes = 0, out_bytes = 0;
    bool ready = false;
};

std::mutex g_pipe_mu;
std::map<int, Pipeline> g_pipes;

void free_buffers(Pipeline &p) {
    for (int s = 0; s < kStages; ++s) {
        if (p.d_in[s]) cudaFree(p.d_in[s]);
        if (p.d_out[s]) cudaFree(p.d_out[s]);
        p.d_in[s] = p.d_out[s] = nullptr;
    }
    p.in_bytes = p.out_bytes = 0;
}

void sync_pipeline(Pipeline &p) {
    for (cudaStream_t st : {p.in, p.hash, p.out})
        if (st) cudaStreamSynchronize(st);
}

void free_pipeline(Pipeline &p) {
    sync_pipeline(p);
    free_buffers(p);
    for (int s = 0; s < kStages; ++s)
        for (cudaEvent_t *e : {&p.copied[s], &p.hashed[s], &p.drained[s]})
            if (*e) {
                cudaEventDestroy(*e);
                *e = nullptr;
            }
    for (cudaStream_t *st : {&p.in, &p.hash, &p.out})
        if (*st) {
            cudaStreamDestroy(*st);
            *st = nullptr;
        }
    p.ready = false;
}

int ensure_pipeline(Pipeline &p, size_t in_bytes, size_t out_bytes) {
    if (!p.ready) {
        for (cudaStream_t *st : {&p.in, &p.hash, &p.out})
            if (cudaStreamCreateWithFlags(st, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                free_pipeline(p);
                return KB_ERR_CUDA;
            }
        for (int s = 0; s < kStages; ++s)
            for (cudaEvent_t *e : {&p.copied[s], &p.hashed[s], &p.drained[s]})
                if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
                    cudaGetLastError();
                    free_pipeline(p);
                    return KB_ERR_CUDA;
                }
        p.ready = true;
    }
    if (p.in_bytes < in_bytes || p.out_bytes < out_bytes) {
        sync_pipeline(p);
        const size_t want_in = std::max(p.in_bytes, in_bytes), want_out = std::max(p.out_bytes, out_bytes);
        free_buffers(p);
        for (int s = 0; s < kStages; ++s) {
            if (cudaMalloc(&p.d_in[s], want_in ? want_in : 16) != cudaSuccess ||
                cudaMalloc(&p.d_out[s], want_out ? want_out : 16) != cudaSuccess) {
                cudaGetLastError();
                free_buffers(p);
                return KB_ERR_NOMEM;
            }
        }
        p.in_bytes = want_in;
        p.out_bytes = want_out;
    }
    return KB_OK;
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

int keccak_batch_uniform_host(const uint8_t *h_msgs, uint64_t stride, uint64_t len, int variant,
                              uint32_t out_len, uint8_t *h_digests, uint64_t n, void *stream) {
    if (variant < 0 || variant > 5 || !valid_out_len(variant, out_len)) return KB_ERR_INVALID;
    if (n == 0) return KB_OK;
    if ((len > 0 && !h_msgs) || (out_len > 0 && !h_digests) || !sizes_fit(stride, len, out_len, n))
        return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    NvtxRange range("keccak_batch_uniform_host");
    // In place (KB_HOST_PATH_ZERO_COPY): the kernel reads the messages and
    // writes the digests in page-locked host memory directly.  Measured slower
    // than the staged copies on GB300, so it is not the default.
    const int64_t path = tuning_get(KB_TUNE_HOST_PATH);
    const void *d_in = len ? device_view(h_msgs) : h_msgs;
    const void *d_out = out_len ? device_view(h_digests) : h_digests;
    if (path == KB_HOST_PATH_ZERO_COPY && d_in && d_out) {
        cudaStream_t user = static_cast<cudaStream_t>(stream);
        int rc = launch_uniform(static_cast<const uint8_t *>(d_in), stride, len, variant, out_len,
                                static_cast<uint8_t *>(const_cast<void *>(d_out)), n, user, *dev);
        if (rc == KB_OK && cudaStreamSynchronize(user) != cudaSuccess) rc = KB_ERR_CUDA;
        return rc;
    }
    if (path == KB_HOST_PATH_ZERO_COPY) return KB_ERR_INVALID;  // asked for, but the buffers are pageable
    // Chunks of about 32 MiB of input (at least one message each).
    const uint64_t target = uint64_t(32) << 20;
    uint64_t chunk = stride ? std::max<uint64_t>(1, target / stride) : n;
    chunk = std::min(chunk, n);
    const size_t in_bytes = size_t((chunk - 1) * stride + len);
    const size_t out_bytes = size_t(chunk * out_len);
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    Pipeline &p = g_pipes[dev->device];
    if ((err = ensure_pipeline(p, in_bytes, out_bytes)) != KB_OK) return err;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaEvent_t start;
    if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) return KB_ERR_CUDA;
    int rc = cuda_status(cudaEventRecord(start, user));
    for (cudaStream_t st : {p.in, p.hash, p.out})
        if (rc == KB_OK) rc = cuda_status(cudaStreamWaitEvent(st, start, 0));
    // Chunk sizes ramp up from chunk/16 at the start and back down at the
    // end, so that the first copy in and the last copy out, which nothing
    // overlaps, are short.
    const std::vector<uint64_t> counts = pipeline_chunks(n, chunk);
    uint64_t first = 0;
    for (size_t idx = 0; idx < counts.size() && rc == KB_OK; first += counts[idx], ++idx) {
        const int s = int(idx % kStages);
        const bool reuse = idx >= size_t(kStages);
        const uint64_t cnt = counts[idx];
        const size_t span = size_t((cnt - 1) * stride + len);
        // In: once the hashing of the chunk that last used d_in[s] is done.
        if (reuse) rc = cuda_status(cudaStreamWaitEvent(p.in, p.hashed[s], 0));
        if (rc == KB_OK && span)
            rc = cuda_status(cudaMemcpyAsync(p.d_in[s], h_msgs + first * stride, span, cudaMemcpyHostToDevice, p.in));
        if (rc == KB_OK) rc = cuda_status(cudaEventRecord(p.copied[s], p.in));
        // Hash: once this chunk is in and d_out[s] has been copied out.
        if (rc == KB_OK) rc = cuda_status(cudaStreamWaitEvent(p.hash, p.copied[s], 0));
        if (rc == KB_OK && reuse) rc = cuda_status(cudaStreamWaitEvent(p.hash, p.drained[s], 0));
        if (rc == KB_OK) rc = launch_uniform(p.d_in[s], stride, len, variant, out_len, p.d_out[s], cnt, p.hash, *dev);
        if (rc == KB_OK) rc = cuda_status(cudaEventRecord(p.hashed[s], p.hash));
        // Out: once this chunk is hashed.
        if (rc == KB_OK) rc = cuda_status(cudaStreamWaitEvent(p.out, p.hashed[s], 0));
        if (rc == KB_OK && out_len)
            rc = cuda_status(cudaMemcpyAsync(h_digests + first * out_len, p.d_out[s], size_t(cnt * out_len),
                                             cudaMemcpyDeviceToHost, p.out));
        if (rc == KB_OK) rc = cuda_status(cudaEventRecord(p.drained[s], p.out));
    }
    for (cudaStream_t st : {p.in, p.hash, p.out})
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = KB_ERR_CUDA;
    cudaEventDestroy(start);
    return rc;
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
        std::lock_guard<std::mutex> lk(g_pipe_mu);
        auto it = g_pipes.find(dev);
        if (it != g_pipes.end()) {
            free_pipeline(it->second);
            g_pipes.erase(it);
        }
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
