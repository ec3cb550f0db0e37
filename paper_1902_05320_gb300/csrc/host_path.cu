// host_path.cu -- keccak_batch_uniform_host (the fixed-stride batch on HOST
// buffers, transfers included) and page-locked host memory placed on the host
// NUMA node nearest the GPU.
//
// Two ways to move the data, both exact:
//  * staged: chunks copied in by the copy engines, hashed, and the digests
//    copied out, pipelined over three streams (one per role);
//  * in place: the kernel reads the messages from, and writes the digests
//    to, page-locked host memory directly (loads by the SMs over the host
//    link).
// Which one is faster depends on the host link and on where the buffers sit
// (a buffer on a far NUMA node crosses the link between the CPUs as well),
// so with KB_HOST_PATH_AUTO the first call of a size class on a device times
// both on parts of its own batch and keeps the faster for later calls of that
// class (a "host-path decision").
#include <cuda_runtime.h>

#include <sys/syscall.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "host_chunks.h"
#include "host_path.h"
#include "keccak_core.cuh"
#include "runtime.cuh"

namespace kb {
namespace {

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


// ---- one range of messages by each path ------------------------------------

// Staged: copies in, hashing, copies out, pipelined; synchronous.
int run_staged(Pipeline &p, const uint8_t *h_msgs, uint64_t stride, uint64_t len, int variant, uint32_t out_len,
               uint8_t *h_digests, uint64_t n, cudaStream_t user, const DeviceInfo &dev) {
    if (n == 0) return KB_OK;
    // Chunks of about 64 MiB of input (at least one message each): copies
    // in and out running together move more per second in larger pieces
    // (measured on GB300, 1 GiB in + 0.5 GiB out: targets of 16, 32, 64 and
    // 128 MiB gave 2633, 2741-2751, 2777-2787 and 2741-2743 Mhash/s).
    const uint64_t target = uint64_t(64) << 20;
    uint64_t chunk = stride ? std::max<uint64_t>(1, target / stride) : n;
    chunk = std::min(chunk, n);
    const size_t in_bytes = size_t((chunk - 1) * stride + len);
    const size_t out_bytes = size_t(chunk * out_len);
    int err = ensure_pipeline(p, in_bytes, out_bytes);
    if (err != KB_OK) return err;
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
        if (rc == KB_OK) rc = launch_uniform(p.d_in[s], stride, len, variant, out_len, p.d_out[s], cnt, p.hash, dev);
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

// In place on page-locked memory (device views of the host buffers); synchronous.
int run_in_place(const uint8_t *d_msgs, uint64_t stride, uint64_t len, int variant, uint32_t out_len,
                 uint8_t *d_digests, uint64_t n, cudaStream_t user, const DeviceInfo &dev) {
    if (n == 0) return KB_OK;
    int rc = launch_uniform(d_msgs, stride, len, variant, out_len, d_digests, n, user, dev);
    if (rc == KB_OK && cudaStreamSynchronize(user) != cudaSuccess) rc = KB_ERR_CUDA;
    return rc;
}

// ---- host-path decisions (KB_HOST_PATH_AUTO) --------------------------------

std::mutex g_path_mu;
std::map<std::pair<int, int>, int> g_paths;  // (device, floor(log2 n)) -> KB_HOST_PATH_STAGED / _ZERO_COPY

int size_class(uint64_t n) { return n ? 63 - __builtin_clzll(n) : 0; }

// Below this many messages a call is too short to time both paths usefully;
// it runs staged and decides nothing.
constexpr uint64_t kTrialMin = 1u << 14;

// ---- page-locked host memory near the GPU ------------------------------------

constexpr unsigned long kMpolFNodeAddr = 3;   // MPOL_F_NODE | MPOL_F_ADDR
constexpr int kMaxNodes = 1024;
constexpr int kLongBits = int(8 * sizeof(unsigned long));

struct HostBlock {
    size_t bytes;
};
std::mutex g_host_mu;
std::map<void *, HostBlock> g_host_blocks;

constexpr int kMpolPreferred = 1;              // MPOL_PREFERRED

// While alive, the calling thread allocates new pages on NUMA node `node`
// when it can (a preferred-node policy); the thread's previous policy comes
// back at the end.  Does nothing for node < 0 or when the system refuses.
class PreferNode {
  public:
    explicit PreferNode(int node) {
        if (node < 0 || node >= kMaxNodes) return;
        if (syscall(SYS_get_mempolicy, &old_mode_, old_mask_, static_cast<unsigned long>(kMaxNodes) + 1, nullptr,
                    0UL) != 0)
            return;
        unsigned long mask[kMaxNodes / kLongBits + 1] = {};  // one spare word for kernels that read maxnode bits
        mask[node / kLongBits] = 1UL << (node % kLongBits);
        set_ = syscall(SYS_set_mempolicy, kMpolPreferred, mask, static_cast<unsigned long>(kMaxNodes) + 1) == 0;
    }
    ~PreferNode() {
        if (set_) syscall(SYS_set_mempolicy, old_mode_, old_mask_, static_cast<unsigned long>(kMaxNodes) + 1);
    }

  private:
    int old_mode_ = 0;
    unsigned long old_mask_[kMaxNodes / kLongBits + 1] = {};
    bool set_ = false;
};

// Copies n16 16-byte words from src (host memory seen through its device
// view) to dst with SM loads and stores (link diagnostic).
__global__ void k_read_host(const uint4 *__restrict__ src, uint4 *__restrict__ dst, uint64_t n16) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n16; i += step) dst[i] = src[i];
}

}  // namespace

void release_host_pipeline(int device) {
    {
        std::lock_guard<std::mutex> lk(g_pipe_mu);
        auto it = g_pipes.find(device);
        if (it != g_pipes.end()) {
            free_pipeline(it->second);
            g_pipes.erase(it);
        }
    }
    std::lock_guard<std::mutex> lk(g_path_mu);
    for (auto it = g_paths.begin(); it != g_paths.end();)
        it = it->first.first == device ? g_paths.erase(it) : std::next(it);
}

}  // namespace kb

using namespace kb;

namespace {
bool valid_out_len(int variant, uint32_t out_len) {
    const int d = variant_digest(variant);
    return d == 0 || out_len == uint32_t(d);
}
bool sizes_fit(uint64_t stride, uint64_t len, uint32_t out_len, uint64_t n) {
    if (n == 0) return true;
    if (stride != 0 && (n - 1) > (UINT64_MAX - len) / stride) return false;
    if (out_len != 0 && n > UINT64_MAX / out_len) return false;
    return true;
}
double seconds_since(std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t).count();
}
}  // namespace

extern "C" {

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
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    const int64_t knob = tuning_get(KB_TUNE_HOST_PATH);
    const uint8_t *d_in = static_cast<const uint8_t *>(len ? device_view(h_msgs) : h_msgs);
    uint8_t *d_out = static_cast<uint8_t *>(const_cast<void *>(out_len ? device_view(h_digests) : h_digests));
    const bool in_place_ok = d_in && d_out;
    if (knob == KB_HOST_PATH_ZERO_COPY) {
        if (!in_place_ok) return KB_ERR_INVALID;  // asked for, but the buffers are pageable
        return run_in_place(d_in, stride, len, variant, out_len, d_out, n, user, *dev);
    }
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    Pipeline &p = g_pipes[dev->device];
    if (knob == KB_HOST_PATH_STAGED || !in_place_ok)
        return run_staged(p, h_msgs, stride, len, variant, out_len, h_digests, n, user, *dev);
    // KB_HOST_PATH_AUTO on page-locked buffers: the decision for this size
    // class, or a trial on this batch.
    const auto key = std::make_pair(dev->device, size_class(n));
    int decided = 0;
    {
        std::lock_guard<std::mutex> lk2(g_path_mu);
        auto it = g_paths.find(key);
        if (it != g_paths.end()) decided = it->second;
    }
    if (decided == KB_HOST_PATH_ZERO_COPY) return run_in_place(d_in, stride, len, variant, out_len, d_out, n, user, *dev);
    if (decided == KB_HOST_PATH_STAGED || n < kTrialMin)
        return run_staged(p, h_msgs, stride, len, variant, out_len, h_digests, n, user, *dev);
    // Trial: a short warm-up of each path, then two eighths of the batch each,
    // alternating, timed on the host (both paths are synchronous); each path
    // keeps the faster of its two timings, so that one call slowed by
    // something outside it (a stall of the copy engines was seen to last
    // tens of milliseconds) does not decide.  The rest of the batch goes by
    // the faster path; every message is hashed once, by one path or the other.
    const uint64_t warm = std::max<uint64_t>(1, n / 64), eighth = n / 8;
    uint64_t at = 0;
    auto staged = [&](uint64_t cnt) {
        const int rc = run_staged(p, h_msgs + at * stride, stride, len, variant, out_len, h_digests + at * out_len,
                                  cnt, user, *dev);
        at += cnt;
        return rc;
    };
    auto in_place = [&](uint64_t cnt) {
        const int rc = run_in_place(d_in + at * stride, stride, len, variant, out_len, d_out + at * out_len, cnt,
                                    user, *dev);
        at += cnt;
        return rc;
    };
    int rc = staged(warm);
    if (rc == KB_OK) rc = in_place(warm);
    double t_staged = 1e30, t_in_place = 1e30;
    for (int round = 0; round < 2 && rc == KB_OK; ++round) {
        auto t = std::chrono::steady_clock::now();
        rc = staged(eighth);
        t_staged = std::min(t_staged, seconds_since(t));
        if (rc != KB_OK) break;
        t = std::chrono::steady_clock::now();
        rc = in_place(eighth);
        t_in_place = std::min(t_in_place, seconds_since(t));
    }
    if (rc != KB_OK) return rc;
    const int choice = t_in_place < t_staged ? KB_HOST_PATH_ZERO_COPY : KB_HOST_PATH_STAGED;
    {
        std::lock_guard<std::mutex> lk2(g_path_mu);
        g_paths[key] = choice;
    }
    return choice == KB_HOST_PATH_ZERO_COPY ? in_place(n - at) : staged(n - at);
}

int keccak_host_path_for(uint64_t n) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return KB_ERR_CUDA;
    const int64_t knob = tuning_get(KB_TUNE_HOST_PATH);
    if (knob != KB_HOST_PATH_AUTO) return int(knob);
    std::lock_guard<std::mutex> lk(g_path_mu);
    auto it = g_paths.find(std::make_pair(dev, size_class(n)));
    return it != g_paths.end() ? it->second : KB_HOST_PATH_AUTO;
}

int keccak_host_alloc(size_t bytes, void **ptr) {
    if (!ptr || bytes == 0) return KB_ERR_INVALID;
    *ptr = nullptr;
    int dev = -1, node = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return KB_ERR_CUDA;
    if (cudaDeviceGetAttribute(&node, cudaDevAttrHostNumaId, dev) != cudaSuccess) {
        cudaGetLastError();
        node = -1;
    }
    // The driver's own page-locked allocation, populated by this thread
    // under a preferred-node policy.  (Anonymous memory bound with mbind and
    // then registered lands on the node too, but the device then reaches it
    // through mappings that degrade as the host's memory fragments: the
    // serving loop's gathers of random 16 KiB pieces of a 4 GiB pool slowed
    // from one process to the next on the same machine, p99 26 -> 35 -> 175
    // ms, while pools from cudaHostAlloc gave 25.9-26.0 ms every time.)
    void *p = nullptr;
    {
        PreferNode prefer(node);
        if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess || !p) {
            cudaGetLastError();
            return KB_ERR_NOMEM;
        }
    }
    std::lock_guard<std::mutex> lk(g_host_mu);
    g_host_blocks[p] = HostBlock{bytes};
    *ptr = p;
    return KB_OK;
}

int keccak_host_free(void *ptr) {
    if (!ptr) return KB_OK;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        auto it = g_host_blocks.find(ptr);
        if (it == g_host_blocks.end()) return KB_ERR_INVALID;
        g_host_blocks.erase(it);
    }
    if (cudaFreeHost(ptr) != cudaSuccess) {
        cudaGetLastError();
        return KB_ERR_CUDA;
    }
    return KB_OK;
}

int sha3gb_host_link_probe(const void *host, void *device, size_t bytes, int mode, int reps, double *gb_s,
                           void *stream) {
    if (!host || !device || !gb_s || bytes < 32 || (bytes & 15) || mode < 0 || mode > 3 || reps < 1)
        return KB_ERR_INVALID;
    int err = KB_OK;
    DeviceInfo *dev = device_info(&err);
    if (!dev) return err;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint8_t *d_host = static_cast<const uint8_t *>(device_view(host));
    if (mode == 3 && !d_host) return KB_ERR_INVALID;  // SM loads need page-locked memory
    cudaStream_t other = nullptr;
    cudaEvent_t a = nullptr, b = nullptr, fork = nullptr, join = nullptr;
    int rc = KB_OK;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess ||
        (mode == 2 && cudaStreamCreateWithFlags(&other, cudaStreamNonBlocking) != cudaSuccess))
        rc = KB_ERR_CUDA;
    const size_t half = bytes / 2 / 16 * 16;
    uint8_t *h = const_cast<uint8_t *>(static_cast<const uint8_t *>(host));
    uint8_t *d = static_cast<uint8_t *>(device);
    auto once = [&]() -> int {
        switch (mode) {
            case 0: return cuda_status(cudaMemcpyAsync(d, host, bytes, cudaMemcpyHostToDevice, s));
            case 1: return cuda_status(cudaMemcpyAsync(h, device, bytes, cudaMemcpyDeviceToHost, s));
            case 2:  // one half each way at once, on two streams
                if (cudaEventRecord(fork, s) != cudaSuccess || cudaStreamWaitEvent(other, fork, 0) != cudaSuccess ||
                    cudaMemcpyAsync(d, host, half, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                    cudaMemcpyAsync(h + half, d + half, bytes - half, cudaMemcpyDeviceToHost, other) != cudaSuccess ||
                    cudaEventRecord(join, other) != cudaSuccess || cudaStreamWaitEvent(s, join, 0) != cudaSuccess)
                    return KB_ERR_CUDA;
                return KB_OK;
            default:
                k_read_host<<<dev->sm_count * 4, 256, 0, s>>>(reinterpret_cast<const uint4 *>(d_host),
                                                               reinterpret_cast<uint4 *>(d), bytes / 16);
                return cuda_status(cudaGetLastError());
        }
    };
    if (rc == KB_OK) rc = once();  // untimed first pass
    if (rc == KB_OK) rc = cuda_status(cudaEventRecord(a, s));
    for (int r = 0; r < reps && rc == KB_OK; ++r) rc = once();
    if (rc == KB_OK) rc = cuda_status(cudaEventRecord(b, s));
    if (rc == KB_OK) rc = cuda_status(cudaEventSynchronize(b));
    float ms = 0;
    if (rc == KB_OK) rc = cuda_status(cudaEventElapsedTime(&ms, a, b));
    if (rc == KB_OK) *gb_s = double(bytes) * reps / (double(ms) * 1e6);
    for (cudaEvent_t e : {a, b, fork, join})
        if (e) cudaEventDestroy(e);
    if (other) {
        cudaStreamSynchronize(other);
        cudaStreamDestroy(other);
    }
    return rc;
}

int keccak_host_numa_node(const void *ptr) {
    if (!ptr) return -1;
    int node = -1;
    if (syscall(SYS_get_mempolicy, &node, nullptr, 0UL, const_cast<void *>(ptr), kMpolFNodeAddr) != 0) return -1;
    return node;
}

}  // extern "C"
