// sha3_queue.cu -- ragged batches in one persistent launch fed by a
// cost-bucketed work queue (the batch mode of Section 4 for messages of mixed
// lengths and variants).
//
// A message's cost is its number of Keccak-f permutations: floor(len/r) + 1
// absorbed blocks plus ceil(d/r) - 1 extra squeezes.  Costs fall into 1920
// buckets (exact below 64, 32 per octave above, so the messages of one warp
// differ in cost by at most 1/32).  On the device:
//   1. k_prep: digest-offset tile sums and a bucket histogram;
//   2. k_plan: one block scans the tile sums and lays the buckets out
//      longest-first;
//   3. k_scatter: digest offsets, and each message's slot in the work order;
//   4. k_sha3_queue: a grid of (blocks per SM x SMs) blocks; each warp takes
//      the next 32 entries of the order with one atomic and hashes one
//      message per thread.  Warps therefore run messages of nearly equal
//      cost, and the longest messages start first so the tail is short.
// The five operations (a memset and four kernels) are captured once per call
// signature into a CUDA graph and replayed afterwards.  A control schedule
// groups the messages by variant instead and hashes each variant with its
// own launch (the plain per-variant form the queue is measured against).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include <unistd.h>

#include "keccak_core.cuh"
#include "lane_parallel.cuh"
#include "runtime.cuh"
#include "scan.cuh"
#include "sponge.cuh"

namespace kb {
namespace {

constexpr int kBucketsPerOctave = 32;
constexpr int kBuckets = 64 + 58 * kBucketsPerOctave;  // costs up to 2^64 - 1

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
    return uint32_t(64 + (e - 6) * kBucketsPerOctave + int((c >> (e - 5)) & (kBucketsPerOctave - 1)));
}

// Bucket of a message: its cost bucket, or (for the per-variant control
// schedule) its variant, 6 standing for an invalid one.
template <bool BY_VARIANT>
__device__ __forceinline__ uint32_t bucket_key(uint64_t len, int v, uint32_t dlen) {
    if constexpr (BY_VARIANT) return v > 5 ? 6u : uint32_t(v);
    else return cost_bucket(message_cost(len, v, dlen));
}

struct Control {
    uint32_t count[kBuckets];   // messages per bucket
    uint32_t cursor[kBuckets];  // next free slot of each bucket in the order
    unsigned long long head;    // work-queue position
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

// One block: exclusive scan of the tile sums, and bucket starts in
// descending cost order (bucket kBuckets-1 first).
__global__ void __launch_bounds__(kScanThreads) k_plan(uint64_t *tile_sums, uint64_t ntiles, Control *ctl) {
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

template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
    k_sha3_queue(const uint8_t *__restrict__ msgs, const uint64_t *__restrict__ offsets,
                 const uint64_t *__restrict__ lens, const uint8_t *__restrict__ variants,
                 const uint32_t *__restrict__ out_lens, const uint64_t *__restrict__ out_off,
                 const uint32_t *__restrict__ order, uint8_t *__restrict__ digests, uint64_t n, Control *ctl,
                 unsigned int *status) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctl->head, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const uint64_t idx = base + lane;
        if (idx < n) hash_ragged_message(msgs, offsets, lens, variants, out_lens, out_off, digests, order[idx], status);
    }
}

// Lane-parallel schedule: each warp takes one message at a time from the same
// longest-first order and runs its sponge across 25 threads.
__global__ void __launch_bounds__(kThreads)
    k_sha3_lanes(const uint8_t *__restrict__ msgs, const uint64_t *__restrict__ offsets,
                 const uint64_t *__restrict__ lens, const uint8_t *__restrict__ variants,
                 const uint32_t *__restrict__ out_lens, const uint64_t *__restrict__ out_off,
                 const uint32_t *__restrict__ order, uint8_t *__restrict__ digests, uint64_t n, Control *ctl,
                 unsigned int *status) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(&ctl->head, 1ull);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= n) break;
        const uint32_t i = order[idx];
        const int v = variants[i];
        const uint32_t dlen = out_lens[i];
        if (v > 5 || (v < 4 && dlen != uint32_t(variant_digest(v)))) {
            if (lane == 0) atomicOr(status, v > 5 ? KB_DEV_BAD_VARIANT : KB_DEV_BAD_OUTLEN);
            continue;
        }
        const uint8_t *p = msgs + offsets[i];
        if ((reinterpret_cast<uintptr_t>(p) & 7) == 0) lane_sponge<true>(p, lens[i], v, digests + out_off[i], dlen);
        else lane_sponge<false>(p, lens[i], v, digests + out_off[i], dlen);
    }
}

// Per-variant control schedule: one launch per variant, each over the
// messages of that variant (grouped by the same bucket pipeline keyed on the
// variant), one thread per message with the variant's rate fixed at compile
// time and no ordering by length.
template <int V>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_sha3_variant(const uint8_t *__restrict__ msgs, const uint64_t *__restrict__ offsets,
                   const uint64_t *__restrict__ lens, const uint32_t *__restrict__ out_lens,
                   const uint64_t *__restrict__ out_off, const uint32_t *__restrict__ order,
                   uint8_t *__restrict__ digests, const Control *ctl, unsigned int *status) {
    using P = Variant<V>;
    const uint64_t end = ctl->cursor[V], begin = end - ctl->count[V];
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t k = begin + uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < end; k += step) {
        const uint32_t i = order[k];
        const uint32_t dlen = out_lens[i];
        if (P::digest && dlen != uint32_t(P::digest)) {
            atomicOr(status, KB_DEV_BAD_OUTLEN);
            continue;
        }
        sponge<P::rate, P::domain, false, PlainRep>(msgs + offsets[i], lens[i], digests + out_off[i], dlen);
    }
}

__global__ void k_flag_invalid_variants(const Control *ctl, unsigned int *status) {
    if (ctl->count[6]) atomicOr(status, KB_DEV_BAD_VARIANT);
}

// Register budgets the tuner can choose (minimum resident blocks of 128
// threads per SM, which caps registers per thread at 65536 / (128 x MINB)).
const int kMinBlocksChoices[] = {2, 3, 4, 5, 6, 8};

const void *queue_kernel(int minb) {
    switch (minb) {
        case 2: return reinterpret_cast<const void *>(&k_sha3_queue<2>);
        case 3: return reinterpret_cast<const void *>(&k_sha3_queue<3>);
        case 5: return reinterpret_cast<const void *>(&k_sha3_queue<5>);
        case 6: return reinterpret_cast<const void *>(&k_sha3_queue<6>);
        case 8: return reinterpret_cast<const void *>(&k_sha3_queue<8>);
        default: return reinterpret_cast<const void *>(&k_sha3_queue<4>);
    }
}

struct QueueConfig {
    int minb = 3;              // register budget (template instance): 3 blocks of 128 threads per SM
    int blocks_per_sm = 0;     // 0: as many as fit
    bool lanes = false;        // one warp per message (lane-parallel sponge)
    bool per_variant = false;  // control: one launch per variant, unsorted
};

struct Buffers {
    uint64_t *out_off;
    uint64_t *tile_sums;
    uint32_t *order;
    Control *ctl;
};

size_t scratch_bytes(uint64_t n, uint64_t ntiles) {
    const size_t a = 8 * n, b = 8 * ntiles, c = (4 * n + 255) / 256 * 256;
    return 256 + a + b + c + sizeof(Control);
}

Buffers carve(uint8_t *scratch, uint64_t n, uint64_t ntiles) {
    Buffers bf;
    bf.ctl = reinterpret_cast<Control *>(scratch);
    uint8_t *p = scratch + (sizeof(Control) + 255) / 256 * 256;
    bf.out_off = reinterpret_cast<uint64_t *>(p);
    bf.tile_sums = bf.out_off + n;
    bf.order = reinterpret_cast<uint32_t *>(bf.tile_sums + ntiles);
    return bf;
}

uint64_t queue_grid(const QueueConfig &cfg, uint64_t n, const DeviceInfo &dev) {
    if (cfg.per_variant)
        return persistent_grid(reinterpret_cast<const void *>(&k_sha3_variant<1>), kThreads, 0, n, dev);
    if (cfg.lanes)
        return persistent_grid(reinterpret_cast<const void *>(&k_sha3_lanes), kThreads, 0, n * 32, dev);
    uint64_t grid = persistent_grid(queue_kernel(cfg.minb), kThreads, 0, (n + 31) / 32 * 32, dev);
    if (cfg.blocks_per_sm > 0) grid = std::min<uint64_t>(grid, uint64_t(cfg.blocks_per_sm) * dev.sm_count);
    return grid;
}

// Enqueues the whole ragged pipeline on `stream` (capturable: no allocation,
// no synchronisation, no occupancy queries).
int issue(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
          const uint32_t *out_lens, uint8_t *digests, uint64_t n, const Buffers &bf, uint64_t ntiles,
          const QueueConfig &cfg, uint64_t grid, cudaStream_t stream, const DeviceInfo &dev) {
    if (cudaMemsetAsync(bf.ctl, 0, sizeof(Control), stream) != cudaSuccess) return KB_ERR_CUDA;
    if (cfg.per_variant) {
        k_prep<true><<<unsigned(ntiles), kScanThreads, 0, stream>>>(lens, variants, out_lens, n, bf.tile_sums, bf.ctl);
        k_plan<<<1, kScanThreads, 0, stream>>>(bf.tile_sums, ntiles, bf.ctl);
        k_scatter<true><<<unsigned(ntiles), kScanThreads, 0, stream>>>(lens, variants, out_lens, n, bf.tile_sums,
                                                                       bf.out_off, bf.order, bf.ctl);
        const unsigned g = unsigned(grid);
        k_sha3_variant<0><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, dev.d_status);
        k_sha3_variant<1><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, dev.d_status);
        k_sha3_variant<2><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, dev.d_status);
        k_sha3_variant<3><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, dev.d_status);
        k_sha3_variant<4><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, dev.d_status);
        k_sha3_variant<5><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, dev.d_status);
        k_flag_invalid_variants<<<1, 1, 0, stream>>>(bf.ctl, dev.d_status);
        return cuda_status(cudaGetLastError());
    }
    k_prep<false><<<unsigned(ntiles), kScanThreads, 0, stream>>>(lens, variants, out_lens, n, bf.tile_sums, bf.ctl);
    k_plan<<<1, kScanThreads, 0, stream>>>(bf.tile_sums, ntiles, bf.ctl);
    k_scatter<false><<<unsigned(ntiles), kScanThreads, 0, stream>>>(lens, variants, out_lens, n, bf.tile_sums,
                                                                    bf.out_off, bf.order, bf.ctl);
    const void *fn = cfg.lanes ? reinterpret_cast<const void *>(&k_sha3_lanes) : queue_kernel(cfg.minb);
    void *args[] = {&msgs, &offsets, &lens, &variants, &out_lens, const_cast<uint64_t **>(&bf.out_off),
                    const_cast<uint32_t **>(&bf.order), &digests, &n, const_cast<Control **>(&bf.ctl),
                    const_cast<unsigned int **>(&dev.d_status)};
    if (cudaLaunchKernel(fn, dim3(unsigned(grid)), dim3(kThreads), args, 0, stream) != cudaSuccess)
        return KB_ERR_CUDA;
    return cuda_status(cudaGetLastError());
}

// ---- graph cache --------------------------------------------------------------

struct GraphKey {
    const void *ptrs[7];
    uint64_t n;
    cudaStream_t stream;
    int minb, blocks_per_sm, device;
    bool operator==(const GraphKey &o) const {
        return std::memcmp(ptrs, o.ptrs, sizeof ptrs) == 0 && n == o.n && stream == o.stream && minb == o.minb &&
               blocks_per_sm == o.blocks_per_sm && device == o.device;
    }
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
};

constexpr size_t kGraphCacheSize = 16;
std::mutex g_graph_mu;
std::list<GraphEntry> g_graphs;  // most recently used first

void drop_graphs_locked(int device) {
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        if (device < 0 || it->key.device == device) {
            cudaGraphExecDestroy(it->exec);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

// ---- tuned configurations -------------------------------------------------------

std::mutex g_tune_mu;
struct TuneEntry {
    int device;
    int size_class;
    QueueConfig cfg;
};
std::list<TuneEntry> g_tuned;

int size_class(uint64_t n) { return n ? 63 - __builtin_clzll(n) : 0; }

// ---- the tuned configurations kept in a file (SHA3GB_TUNE_CACHE) ---------------
//
// When SHA3GB_TUNE_CACHE names a file, configurations found by the autotuner
// are written there and read back by later processes.  The file holds JSON
// Lines, one object per entry in the fixed form this file writes:
//   {"gpu": NAME, "sms": SMs, "size_class": floor(log2 n),
//    "min_blocks": register budget (blocks per SM compiled for),
//    "blocks_per_sm": blocks per SM of the launch}
// Entries are matched on the GPU's name and SM count; lines that do not
// parse are ignored, and I/O failures leave the in-memory tuning as it is.

struct CacheLine {
    std::string gpu;
    int sms = 0, size_class = 0, minb = 0, bps = 0;
};

const char *cache_path() {
    const char *p = std::getenv("SHA3GB_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

std::string gpu_name(int device) {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string name = prop.name;
    for (char &ch : name)  // kept out of the JSON string: quotes, backslashes, controls
        if (ch == '"' || ch == '\\' || static_cast<unsigned char>(ch) < 0x20) ch = '_';
    return name;
}

constexpr const char *kCacheFormat =
    "{\"gpu\": \"%s\", \"sms\": %d, \"size_class\": %d, \"min_blocks\": %d, \"blocks_per_sm\": %d}\n";

bool valid_minb(int m) { return m == 2 || m == 3 || m == 4 || m == 5 || m == 6 || m == 8; }

std::vector<CacheLine> read_cache(const char *path) {
    std::vector<CacheLine> out;
    FILE *f = std::fopen(path, "r");
    if (!f) return out;
    char buf[512];
    while (std::fgets(buf, sizeof buf, f)) {
        CacheLine c;
        char name[256];
        if (std::sscanf(buf, "{\"gpu\": \"%255[^\"]\", \"sms\": %d, \"size_class\": %d, \"min_blocks\": %d, "
                             "\"blocks_per_sm\": %d}",
                        name, &c.sms, &c.size_class, &c.minb, &c.bps) != 5)
            continue;
        c.gpu = name;
        if (c.size_class < 0 || c.size_class > 63 || !valid_minb(c.minb) || c.bps < 0 || c.bps > 32) continue;
        out.push_back(c);
    }
    std::fclose(f);
    return out;
}

std::set<int> g_cache_loaded;  // devices whose file entries are in g_tuned (under g_tune_mu)

// Adds this GPU's entries of the file to g_tuned, once per device.
void load_cache_locked(const DeviceInfo &dev) {
    if (g_cache_loaded.count(dev.device)) return;
    g_cache_loaded.insert(dev.device);
    const char *path = cache_path();
    if (!path) return;
    const std::string name = gpu_name(dev.device);
    for (const CacheLine &c : read_cache(path)) {
        if (c.gpu != name || c.sms != dev.sm_count) continue;
        bool have = false;
        for (const auto &t : g_tuned) have = have || (t.device == dev.device && t.size_class == c.size_class);
        if (have) continue;
        QueueConfig cfg;
        cfg.minb = c.minb;
        cfg.blocks_per_sm = c.bps;
        g_tuned.push_back(TuneEntry{dev.device, c.size_class, cfg});
    }
}

// Writes one entry to the file, replacing an older one with the same key.
void save_cache_entry(const DeviceInfo &dev, int sc, const QueueConfig &cfg) {
    const char *path = cache_path();
    if (!path) return;
    const std::string name = gpu_name(dev.device);
    std::vector<CacheLine> lines = read_cache(path);
    lines.erase(std::remove_if(lines.begin(), lines.end(),
                               [&](const CacheLine &c) {
                                   return c.gpu == name && c.sms == dev.sm_count && c.size_class == sc;
                               }),
                lines.end());
    lines.push_back(CacheLine{name, dev.sm_count, sc, cfg.minb, cfg.blocks_per_sm});
    // A name of this process's own, so that processes saving at once do not
    // write into each other's file; the last rename wins.
    const std::string tmp = std::string(path) + ".tmp." + std::to_string(static_cast<long>(getpid()));
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const CacheLine &c : lines)
        std::fprintf(f, kCacheFormat, c.gpu.c_str(), c.sms, c.size_class, c.minb, c.bps);
    if (std::fclose(f) != 0 || std::rename(tmp.c_str(), path) != 0) std::remove(tmp.c_str());
}

// SHA3GB_TUNE: "off" ignores tuned configurations, "full" tunes a batch's
// size class on first sight inside keccak_batch, anything else (or unset)
// uses the configurations keccak_batch_autotune found ("cached").
enum class TuneMode { Cached, Off, Full };
TuneMode tune_mode() {
    static const TuneMode mode = [] {
        const char *m = std::getenv("SHA3GB_TUNE");
        if (m && std::strcmp(m, "off") == 0) return TuneMode::Off;
        if (m && std::strcmp(m, "full") == 0) return TuneMode::Full;
        return TuneMode::Cached;
    }();
    return mode;
}

bool use_tuned() { return tuning_get(KB_TUNE_AUTOTUNE) != 0 && tune_mode() != TuneMode::Off; }

bool have_tuned(uint64_t n, const DeviceInfo &dev) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_cache_locked(dev);
    for (const auto &t : g_tuned)
        if (t.device == dev.device && t.size_class == size_class(n)) return true;
    return false;
}

QueueConfig choose_config(uint64_t n, const DeviceInfo &dev) {
    QueueConfig cfg;
    const int64_t regs = tuning_get(KB_TUNE_QUEUE_MIN_BLOCKS);
    const int64_t bps = tuning_get(KB_TUNE_QUEUE_BLOCKS_PER_SM);
    if (use_tuned()) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_cache_locked(dev);
        for (const auto &t : g_tuned)
            if (t.device == dev.device && t.size_class == size_class(n)) {
                cfg = t.cfg;
                break;
            }
    }
    if (regs > 0) cfg.minb = int(regs);
    if (bps > 0) cfg.blocks_per_sm = int(bps);
    cfg.lanes = tuning_get(KB_TUNE_RAGGED_SCHEDULE) == KB_SCHEDULE_LANE_PARALLEL;
    cfg.per_variant = tuning_get(KB_TUNE_RAGGED_SCHEDULE) == KB_SCHEDULE_PER_VARIANT;
    return cfg;
}

}  // namespace

void release_queue_graphs(int device) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    drop_graphs_locked(device);
}

int launch_ragged_queue(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                        const uint32_t *out_lens, uint8_t *digests, uint64_t n, cudaStream_t stream,
                        const DeviceInfo &dev) {
    const uint64_t ntiles = digest_offsets_tiles(n);
    int err = KB_OK;
    // SHA3GB_TUNE=full: a size class seen for the first time is tuned here
    // (synchronously), which also leaves this batch's digests.
    cudaStreamCaptureStatus cap0 = cudaStreamCaptureStatusNone;
    if (tune_mode() == TuneMode::Full && use_tuned() && tuning_get(KB_TUNE_RAGGED_SCHEDULE) == KB_SCHEDULE_QUEUE &&
        tuning_get(KB_TUNE_QUEUE_MIN_BLOCKS) == 0 && tuning_get(KB_TUNE_QUEUE_BLOCKS_PER_SM) == 0 &&
        cudaStreamIsCapturing(stream, &cap0) == cudaSuccess && cap0 == cudaStreamCaptureStatusNone &&
        !have_tuned(n, dev))
        return autotune_ragged_queue(msgs, offsets, lens, variants, out_lens, digests, n, stream, dev, nullptr,
                                     nullptr, nullptr);
    const size_t bytes = scratch_bytes(n, ntiles);
    uint8_t *scratch = static_cast<uint8_t *>(stream_scratch(stream, bytes, &err));
    if (!scratch) return err;
    const Buffers bf = carve(scratch, n, ntiles);
    const QueueConfig cfg = choose_config(n, dev);
    const uint64_t grid = queue_grid(cfg, n, dev);

    // Graph replay needs a capturable stream that is not already capturing.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool graphs = tuning_get(KB_TUNE_GRAPHS) != 0 && stream != nullptr &&
                        cudaStreamIsCapturing(stream, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone;
    if (!graphs) return issue(msgs, offsets, lens, variants, out_lens, digests, n, bf, ntiles, cfg, grid, stream, dev);

    GraphKey key{{msgs, offsets, lens, variants, out_lens, digests, scratch}, n, stream,
                 cfg.per_variant ? 100 : cfg.lanes ? -cfg.minb : cfg.minb, cfg.blocks_per_sm, dev.device};
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
            if (it->key == key) {
                g_graphs.splice(g_graphs.begin(), g_graphs, it);
                return cuda_status(cudaGraphLaunch(it->exec, stream));
            }
        }
    }
    // Capture once, instantiate, launch.
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return issue(msgs, offsets, lens, variants, out_lens, digests, n, bf, ntiles, cfg, grid, stream, dev);
    }
    const int rc = issue(msgs, offsets, lens, variants, out_lens, digests, n, bf, ntiles, cfg, grid, stream, dev);
    cudaGraph_t graph = nullptr;
    const cudaError_t end = cudaStreamEndCapture(stream, &graph);
    if (rc != KB_OK || end != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != KB_OK ? rc : KB_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t inst = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (inst != cudaSuccess) {
        cudaGetLastError();
        return issue(msgs, offsets, lens, variants, out_lens, digests, n, bf, ntiles, cfg, grid, stream, dev);
    }
    const int launched = cuda_status(cudaGraphLaunch(exec, stream));
    std::lock_guard<std::mutex> lk(g_graph_mu);
    g_graphs.push_front(GraphEntry{key, exec});
    while (g_graphs.size() > kGraphCacheSize) {
        cudaGraphExecDestroy(g_graphs.back().exec);
        g_graphs.pop_back();
    }
    return launched;
}

__global__ void k_compare(const uint8_t *__restrict__ a, const uint8_t *__restrict__ b, uint64_t bytes,
                          unsigned int *mismatch) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < bytes; i += step)
        if (a[i] != b[i]) {
            atomicOr(mismatch, 1u);
            return;
        }
}

// Autotuner: times every (register budget, blocks per SM) candidate on this
// batch, checks that each writes the same bytes as the first, and keeps the
// fastest for batches of the same size class on this device.  Synchronous;
// allocates a reference copy of the outputs for the duration of the call.
int autotune_ragged_queue(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                          const uint32_t *out_lens, uint8_t *digests, uint64_t n, cudaStream_t stream,
                          const DeviceInfo &dev, int64_t *best_minb, int64_t *best_bps, float *best_ms) {
    const uint64_t ntiles = digest_offsets_tiles(n);
    int err = KB_OK;
    const size_t bytes = scratch_bytes(n, ntiles);
    uint8_t *scratch = static_cast<uint8_t *>(stream_scratch(stream, bytes, &err));
    if (!scratch) return err;
    const Buffers bf = carve(scratch, n, ntiles);
    cudaEvent_t a = nullptr, b = nullptr;
    uint8_t *ref = nullptr;
    unsigned int *mismatch = nullptr;
    uint64_t total_out = 0;
    QueueConfig best;
    float best_t = 1e30f;
    int rc = KB_OK;
    bool have_ref = false;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess ||
        cudaMalloc(&mismatch, sizeof(unsigned int)) != cudaSuccess)
        rc = KB_ERR_CUDA;
    for (int minb : kMinBlocksChoices) {
        if (rc != KB_OK) break;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, queue_kernel(minb), kThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        for (int bps = per_sm; bps >= 1 && bps >= per_sm - 2 && rc == KB_OK; --bps) {
            QueueConfig cfg;
            cfg.minb = minb;
            cfg.blocks_per_sm = bps;
            const uint64_t grid = queue_grid(cfg, n, dev);
            // One untimed run, then the timed one.
            rc = issue(msgs, offsets, lens, variants, out_lens, digests, n, bf, ntiles, cfg, grid, stream, dev);
            if (rc == KB_OK) rc = cuda_status(cudaEventRecord(a, stream));
            if (rc == KB_OK) rc = issue(msgs, offsets, lens, variants, out_lens, digests, n, bf, ntiles, cfg, grid, stream, dev);
            if (rc == KB_OK) rc = cuda_status(cudaEventRecord(b, stream));
            if (rc == KB_OK) rc = cuda_status(cudaEventSynchronize(b));
            float ms = 0;
            if (rc == KB_OK) rc = cuda_status(cudaEventElapsedTime(&ms, a, b));
            if (rc != KB_OK) break;
            if (!have_ref) {
                // Output size: last digest offset + its length.
                uint64_t last_off = 0;
                uint32_t last_len = 0;
                if (cudaMemcpy(&last_off, bf.out_off + (n - 1), 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
                    cudaMemcpy(&last_len, out_lens + (n - 1), 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
                    rc = KB_ERR_CUDA;
                    break;
                }
                total_out = last_off + last_len;
                if (total_out && cudaMalloc(&ref, total_out) != cudaSuccess) {
                    cudaGetLastError();
                    rc = KB_ERR_NOMEM;
                    break;
                }
                if (total_out && cudaMemcpyAsync(ref, digests, total_out, cudaMemcpyDeviceToDevice, stream) != cudaSuccess) {
                    rc = KB_ERR_CUDA;
                    break;
                }
                have_ref = true;
            } else if (total_out) {
                unsigned int bad = 0;
                if (cudaMemsetAsync(mismatch, 0, sizeof bad, stream) != cudaSuccess) { rc = KB_ERR_CUDA; break; }
                k_compare<<<dev.sm_count * 8, 256, 0, stream>>>(ref, digests, total_out, mismatch);
                if (cudaMemcpyAsync(&bad, mismatch, sizeof bad, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                    cudaStreamSynchronize(stream) != cudaSuccess) {
                    rc = KB_ERR_CUDA;
                    break;
                }
                if (bad) continue;  // a configuration that changes the output is never chosen
            }
            if (ms < best_t) {
                best_t = ms;
                best = cfg;
            }
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (ref) cudaFree(ref);
    if (mismatch) cudaFree(mismatch);
    if (rc != KB_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_cache_locked(dev);
        for (auto it = g_tuned.begin(); it != g_tuned.end();)
            it = (it->device == dev.device && it->size_class == size_class(n)) ? g_tuned.erase(it) : std::next(it);
        g_tuned.push_front(TuneEntry{dev.device, size_class(n), best});
        save_cache_entry(dev, size_class(n), best);
    }
    // Leave the caller's digests from the chosen configuration.
    rc = issue(msgs, offsets, lens, variants, out_lens, digests, n, bf, ntiles, best, queue_grid(best, n, dev), stream,
               dev);
    if (best_minb) *best_minb = best.minb;
    if (best_bps) *best_bps = best.blocks_per_sm;
    if (best_ms) *best_ms = best_t;
    return rc;
}

void forget_tuning(int device) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto it = g_tuned.begin(); it != g_tuned.end();)
        it = (device < 0 || it->device == device) ? g_tuned.erase(it) : std::next(it);
    if (device < 0) g_cache_loaded.clear();
    else g_cache_loaded.erase(device);
}

void queue_config_for(uint64_t n, const DeviceInfo &dev, int64_t *min_blocks, int64_t *blocks_per_sm) {
    const QueueConfig cfg = choose_config(n, dev);
    if (min_blocks) *min_blocks = cfg.minb;
    if (blocks_per_sm) *blocks_per_sm = cfg.blocks_per_sm;
}

}  // namespace kb
