// sha3_queue.cu -- host side of the ragged-batch work queue (queue.cuh): the
// launch sequence, its CUDA-graph cache, the configuration choice and the
// autotuner, plus the direct-load instances of the queue kernel and the two
// control schedules.
//
// The five operations of a call (a memset and four kernels; six and a fork
// onto a side stream when the costliest messages run one warp each) are
// captured once per call signature into a CUDA graph and replayed afterwards.
// A control schedule groups the messages by variant instead and hashes each
// variant with its own launch (the plain per-variant form the queue is
// measured against).
//
// A configuration has four dimensions, all picked by the autotuner:
//   * register budget: the blocks of 128 threads per SM the queue kernel is
//     compiled for (2..8);
//   * blocks per SM of the persistent launch (at most that budget);
//   * staging: direct loads, or each thread's next block copied into shared
//     memory during the permutation (with the runtime-rate or the
//     rate-specialised absorb);
//   * threads per message: 1 for every message, or a hybrid in which the K
//     costliest messages run one warp each (the lane-parallel sponge) in a
//     kernel launched first on a side stream, concurrently with the queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include <unistd.h>

#include "queue.cuh"
#include "queue_host.h"

static_assert(kb::QueueConfig().stage == (kb::kStageRegs | kb::kLooped), "default queue stage");

namespace kb {

// One warp per message (lane-parallel sponge) over entries [0, limit) of the
// order, taken one at a time from *head.
__global__ void __launch_bounds__(kThreads)
    k_sha3_lanes(const uint8_t *__restrict__ msgs, const uint64_t *__restrict__ offsets,
                 const uint64_t *__restrict__ lens, const uint8_t *__restrict__ variants,
                 const uint32_t *__restrict__ out_lens, const uint64_t *__restrict__ out_off,
                 const uint32_t *__restrict__ order, uint8_t *__restrict__ digests, uint64_t limit,
                 unsigned long long *head, unsigned int *status) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(head, 1ull);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= limit) break;
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

namespace {

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
// The staged kernels exist for budgets 2..4 only.
const int kMinBlocksChoices[] = {2, 3, 4, 5, 6, 8};

const void *queue_kernel(int minb, int stage) {
    if (stage != kStageDirect) return queue_kernel_staged(minb, stage);
    switch (minb) {
        case 2: return reinterpret_cast<const void *>(&k_sha3_queue<2, kStageDirect>);
        case 3: return reinterpret_cast<const void *>(&k_sha3_queue<3, kStageDirect>);
        case 4: return reinterpret_cast<const void *>(&k_sha3_queue<4, kStageDirect>);
        case 5: return reinterpret_cast<const void *>(&k_sha3_queue<5, kStageDirect>);
        case 6: return reinterpret_cast<const void *>(&k_sha3_queue<6, kStageDirect>);
        case 8: return reinterpret_cast<const void *>(&k_sha3_queue<8, kStageDirect>);
        default: return nullptr;
    }
}

struct Buffers {
    uint64_t *out_off;
    uint64_t *tile_sums;
    uint32_t *order;
    Control *ctl;
};

Buffers carve(uint8_t *scratch, uint64_t n, uint64_t ntiles) {
    Buffers bf;
    bf.ctl = reinterpret_cast<Control *>(scratch);
    uint8_t *p = scratch + (sizeof(Control) + 255) / 256 * 256;
    bf.out_off = reinterpret_cast<uint64_t *>(p);
    bf.tile_sums = bf.out_off + n;
    bf.order = reinterpret_cast<uint32_t *>(bf.tile_sums + ntiles);
    return bf;
}

// Resident blocks per SM of a kernel of kThreads threads (occupancy API),
// cached per (kernel, device); 1 when the query fails.
int resident_blocks(const void *fn, int device) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(fn, device);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    cache[key] = per_sm;
    return per_sm;
}

// Blocks of the hashing launch for n messages.
uint64_t queue_grid(const QueueConfig &cfg, uint64_t n, int device, int sm_count) {
    const void *fn = cfg.per_variant ? reinterpret_cast<const void *>(&k_sha3_variant<1>)
                     : cfg.lanes     ? reinterpret_cast<const void *>(&k_sha3_lanes)
                                     : queue_kernel(cfg.minb, cfg.stage);
    uint64_t per_sm = uint64_t(resident_blocks(fn, device));
    if (!cfg.per_variant && !cfg.lanes && cfg.blocks_per_sm > 0) per_sm = std::min<uint64_t>(per_sm, cfg.blocks_per_sm);
    const uint64_t full = per_sm * uint64_t(sm_count > 0 ? sm_count : 1);
    const uint64_t threads_per_item = cfg.lanes ? 32 : 1;
    const uint64_t need = (n * threads_per_item + kThreads - 1) / kThreads;
    return std::max<uint64_t>(1, std::min(need, full));
}

}  // namespace

size_t queue_scratch_bytes(uint64_t n) { return queue_scratch_size(n); }

bool queue_config_valid(const QueueConfig &cfg) {
    if (cfg.per_variant || cfg.lanes) return true;
    return queue_kernel(cfg.minb, cfg.stage) != nullptr && cfg.blocks_per_sm >= 0 && cfg.warp_messages >= 0;
}

// Enqueues the whole ragged pipeline on `stream` (capturable: no allocation,
// no synchronisation, no occupancy queries once the grid is known).  A
// hybrid configuration forks onto aux->side and joins back.
int queue_issue(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                const uint32_t *out_lens, uint8_t *digests, uint64_t n, uint8_t *scratch, const QueueConfig &cfg,
                uint64_t grid, int sm_count, unsigned int *status, cudaStream_t stream, const AuxStream *aux) {
    const uint64_t ntiles = digest_offsets_tiles(n);
    const Buffers bf = carve(scratch, n, ntiles);
    if (cudaMemsetAsync(bf.ctl, 0, sizeof(Control), stream) != cudaSuccess) return KB_ERR_CUDA;
    if (cfg.per_variant) {
        k_prep<true><<<unsigned(ntiles), kScanThreads, 0, stream>>>(lens, variants, out_lens, n, bf.tile_sums, bf.ctl);
        k_plan<<<1, kScanThreads, 0, stream>>>(bf.tile_sums, ntiles, bf.ctl, 0);
        k_scatter<true><<<unsigned(ntiles), kScanThreads, 0, stream>>>(lens, variants, out_lens, n, bf.tile_sums,
                                                                       bf.out_off, bf.order, bf.ctl);
        const unsigned g = unsigned(grid);
        k_sha3_variant<0><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, status);
        k_sha3_variant<1><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, status);
        k_sha3_variant<2><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, status);
        k_sha3_variant<3><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, status);
        k_sha3_variant<4><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, status);
        k_sha3_variant<5><<<g, kThreads, 0, stream>>>(msgs, offsets, lens, out_lens, bf.out_off, bf.order, digests, bf.ctl, status);
        k_flag_invalid_variants<<<1, 1, 0, stream>>>(bf.ctl, status);
        return cuda_status(cudaGetLastError());
    }
    // The warp-per-message share: the K costliest messages (entries [0, K) of
    // the order); the queue kernel starts after them.
    const uint64_t k = cfg.lanes ? 0 : std::min<uint64_t>(uint64_t(cfg.warp_messages), n);
    if (k && !aux) return KB_ERR_INVALID;
    k_prep<false><<<unsigned(ntiles), kScanThreads, 0, stream>>>(lens, variants, out_lens, n, bf.tile_sums, bf.ctl);
    k_plan<<<1, kScanThreads, 0, stream>>>(bf.tile_sums, ntiles, bf.ctl, k);
    k_scatter<false><<<unsigned(ntiles), kScanThreads, 0, stream>>>(lens, variants, out_lens, n, bf.tile_sums,
                                                                    bf.out_off, bf.order, bf.ctl);
    if (k) {
        if (cudaEventRecord(aux->fork, stream) != cudaSuccess || cudaStreamWaitEvent(aux->side, aux->fork, 0) != cudaSuccess)
            return KB_ERR_CUDA;
        const uint64_t warps = std::min<uint64_t>(k, uint64_t(4) * uint64_t(sm_count > 0 ? sm_count : 1));
        k_sha3_lanes<<<unsigned((warps + 3) / 4), kThreads, 0, aux->side>>>(msgs, offsets, lens, variants, out_lens,
                                                                          bf.out_off, bf.order, digests, k,
                                                                          &bf.ctl->lane_head, status);
        if (cudaEventRecord(aux->join, aux->side) != cudaSuccess) return KB_ERR_CUDA;
    }
    if (k < n || cfg.lanes) {
        unsigned long long *head = &bf.ctl->head;
        const void *fn = cfg.lanes ? reinterpret_cast<const void *>(&k_sha3_lanes) : queue_kernel(cfg.minb, cfg.stage);
        if (!fn) return KB_ERR_INVALID;
        cudaError_t e;
        if (cfg.lanes) {
            uint64_t limit = n;
            void *args[] = {&msgs, &offsets, &lens, &variants, &out_lens, const_cast<uint64_t **>(&bf.out_off),
                            const_cast<uint32_t **>(&bf.order), &digests, &limit, &head, &status};
            e = cudaLaunchKernel(fn, dim3(unsigned(grid)), dim3(kThreads), args, 0, stream);
        } else {
            Control *ctl = bf.ctl;
            void *args[] = {&msgs, &offsets, &lens, &variants, &out_lens, const_cast<uint64_t **>(&bf.out_off),
                            const_cast<uint32_t **>(&bf.order), &digests, &n, &ctl, &status};
            e = cudaLaunchKernel(fn, dim3(unsigned(grid)), dim3(kThreads), args, 0, stream);
        }
        if (e != cudaSuccess) return KB_ERR_CUDA;
    }
    if (k && cudaStreamWaitEvent(stream, aux->join, 0) != cudaSuccess) return KB_ERR_CUDA;
    return cuda_status(cudaGetLastError());
}

uint64_t queue_grid_for(const QueueConfig &cfg, uint64_t n, int device, int sm_count) {
    return queue_grid(cfg, n, device, sm_count);
}

namespace {

// ---- side streams of the hybrid schedule, one per (device, stream) -----------

std::mutex g_aux_mu;
std::map<std::pair<int, cudaStream_t>, AuxStream> g_aux;

// The side stream of `stream`, created on first use (outside any capture).
const AuxStream *aux_for(int device, cudaStream_t stream, int *err) {
    std::lock_guard<std::mutex> lk(g_aux_mu);
    const auto key = std::make_pair(device, stream);
    auto it = g_aux.find(key);
    if (it != g_aux.end()) return &it->second;
    AuxStream a;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&a.side, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (a.side) cudaStreamDestroy(a.side);
        if (a.fork) cudaEventDestroy(a.fork);
        if (a.join) cudaEventDestroy(a.join);
        *err = KB_ERR_CUDA;
        return nullptr;
    }
    return &g_aux.emplace(key, a).first->second;
}

void drop_aux(int device) {
    std::lock_guard<std::mutex> lk(g_aux_mu);
    for (auto it = g_aux.begin(); it != g_aux.end();) {
        if (device < 0 || it->first.first == device) {
            cudaStreamSynchronize(it->second.side);
            cudaStreamDestroy(it->second.side);
            cudaEventDestroy(it->second.fork);
            cudaEventDestroy(it->second.join);
            it = g_aux.erase(it);
        } else {
            ++it;
        }
    }
}

// ---- graph cache --------------------------------------------------------------

struct GraphKey {
    const void *ptrs[7];
    uint64_t n;
    cudaStream_t stream;
    int minb, blocks_per_sm, stage, schedule, device;
    int64_t warp_messages;
    bool operator==(const GraphKey &o) const {
        return std::memcmp(ptrs, o.ptrs, sizeof ptrs) == 0 && n == o.n && stream == o.stream && minb == o.minb &&
               blocks_per_sm == o.blocks_per_sm && stage == o.stage && schedule == o.schedule &&
               device == o.device && warp_messages == o.warp_messages;
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
//    "blocks_per_sm": blocks per SM of the launch,
//    "staging": KB_QUEUE_STAGING_* value, "warp_messages": K}
// Lines without the last two fields (an older form) read as direct loads and
// K = 0.  Entries are matched on the GPU's name and SM count; lines that do
// not parse are ignored, and I/O failures leave the in-memory tuning as it is.

struct CacheLine {
    std::string gpu;
    int sms = 0, size_class = 0, minb = 0, bps = 0, staging = KB_QUEUE_STAGING_DIRECT;
    long long warp_messages = 0;
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
    "{\"gpu\": \"%s\", \"sms\": %d, \"size_class\": %d, \"min_blocks\": %d, \"blocks_per_sm\": %d, "
    "\"staging\": %d, \"warp_messages\": %lld}\n";

// KB_QUEUE_STAGING_* values 1..4 <-> kernel stage codes.
const int kStageCodes[] = {kStageDirect, kStageDirect | kLooped, kStageAsync | kLooped, kStageRegs | kLooped};
int stage_of(int staging) { return staging >= 1 && staging <= 4 ? kStageCodes[staging - 1] : kStageDirect; }
int staging_of(int stage) {
    for (int k = 0; k < 4; ++k)
        if (kStageCodes[k] == stage) return k + 1;
    return KB_QUEUE_STAGING_DIRECT;
}

bool valid_line(const CacheLine &c) {
    if (c.size_class < 0 || c.size_class > 63 || c.bps < 0 || c.bps > 32 || c.warp_messages < 0) return false;
    if (c.staging < KB_QUEUE_STAGING_DIRECT || c.staging > KB_QUEUE_STAGING_REGS) return false;
    return queue_kernel(c.minb, stage_of(c.staging)) != nullptr;
}

std::vector<CacheLine> read_cache(const char *path) {
    std::vector<CacheLine> out;
    FILE *f = std::fopen(path, "r");
    if (!f) return out;
    char buf[512];
    while (std::fgets(buf, sizeof buf, f)) {
        CacheLine c;
        char name[256];
        const int got = std::sscanf(buf,
                                    "{\"gpu\": \"%255[^\"]\", \"sms\": %d, \"size_class\": %d, \"min_blocks\": %d, "
                                    "\"blocks_per_sm\": %d, \"staging\": %d, \"warp_messages\": %lld}",
                                    name, &c.sms, &c.size_class, &c.minb, &c.bps, &c.staging, &c.warp_messages);
        if (got == 5) {  // the older form
            c.staging = KB_QUEUE_STAGING_DIRECT;
            c.warp_messages = 0;
        } else if (got != 7) {
            continue;
        }
        c.gpu = name;
        if (!valid_line(c)) continue;
        out.push_back(c);
    }
    std::fclose(f);
    return out;
}

std::set<int> g_cache_loaded;  // devices whose file entries are in g_tuned (under g_tune_mu)

QueueConfig config_of(const CacheLine &c) {
    QueueConfig cfg;
    cfg.minb = c.minb;
    cfg.blocks_per_sm = c.bps;
    cfg.stage = stage_of(c.staging);
    cfg.warp_messages = c.warp_messages;
    return cfg;
}

// Adds this GPU's entries of the file to g_tuned, once per device.
void load_cache_locked(int device, int sm_count) {
    if (g_cache_loaded.count(device)) return;
    g_cache_loaded.insert(device);
    const char *path = cache_path();
    if (!path) return;
    const std::string name = gpu_name(device);
    for (const CacheLine &c : read_cache(path)) {
        if (c.gpu != name || c.sms != sm_count) continue;
        bool have = false;
        for (const auto &t : g_tuned) have = have || (t.device == device && t.size_class == c.size_class);
        if (have) continue;
        g_tuned.push_back(TuneEntry{device, c.size_class, config_of(c)});
    }
}

// Writes one entry to the file, replacing an older one with the same key.
void save_cache_entry(int device, int sm_count, int sc, const QueueConfig &cfg) {
    const char *path = cache_path();
    if (!path) return;
    const std::string name = gpu_name(device);
    std::vector<CacheLine> lines = read_cache(path);
    lines.erase(std::remove_if(lines.begin(), lines.end(),
                               [&](const CacheLine &c) {
                                   return c.gpu == name && c.sms == sm_count && c.size_class == sc;
                               }),
                lines.end());
    CacheLine c;
    c.gpu = name;
    c.sms = sm_count;
    c.size_class = sc;
    c.minb = cfg.minb;
    c.bps = cfg.blocks_per_sm;
    c.staging = staging_of(cfg.stage);
    c.warp_messages = static_cast<long long>(cfg.warp_messages);
    lines.push_back(c);
    // A name of this process's own, so that processes saving at once do not
    // write into each other's file; the last rename wins.
    const std::string tmp = std::string(path) + ".tmp." + std::to_string(static_cast<long>(getpid()));
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const CacheLine &l : lines)
        std::fprintf(f, kCacheFormat, l.gpu.c_str(), l.sms, l.size_class, l.minb, l.bps, l.staging, l.warp_messages);
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
    load_cache_locked(dev.device, dev.sm_count);
    for (const auto &t : g_tuned)
        if (t.device == dev.device && t.size_class == size_class(n)) return true;
    return false;
}

QueueConfig choose_config(uint64_t n, const DeviceInfo &dev) {
    QueueConfig cfg;
    if (use_tuned()) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_cache_locked(dev.device, dev.sm_count);
        for (const auto &t : g_tuned)
            if (t.device == dev.device && t.size_class == size_class(n)) {
                cfg = t.cfg;
                break;
            }
    }
    apply_knobs(cfg);
    return cfg;
}

}  // namespace

// Knobs override the tuned or default configuration, dimension by dimension.
void apply_knobs(QueueConfig &cfg) {
    const int64_t regs = tuning_get(KB_TUNE_QUEUE_MIN_BLOCKS);
    const int64_t bps = tuning_get(KB_TUNE_QUEUE_BLOCKS_PER_SM);
    const int64_t staging = tuning_get(KB_TUNE_QUEUE_STAGING);
    const int64_t warp = tuning_get(KB_TUNE_QUEUE_WARP_MESSAGES);
    if (regs > 0) cfg.minb = int(regs);
    if (bps > 0) cfg.blocks_per_sm = int(bps);
    if (staging > 0) cfg.stage = stage_of(int(staging));
    if (warp >= 0) cfg.warp_messages = warp;
    // A register budget the chosen staging is not compiled for falls back to
    // direct loads.
    if (!queue_kernel(cfg.minb, cfg.stage)) cfg.stage = kStageDirect;
    if (!queue_kernel(cfg.minb, cfg.stage)) cfg.minb = QueueConfig().minb;
    cfg.lanes = tuning_get(KB_TUNE_RAGGED_SCHEDULE) == KB_SCHEDULE_LANE_PARALLEL;
    cfg.per_variant = tuning_get(KB_TUNE_RAGGED_SCHEDULE) == KB_SCHEDULE_PER_VARIANT;
}

void release_queue_graphs(int device) {
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        drop_graphs_locked(device);
    }
    drop_aux(device);
}

int launch_ragged_queue(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                        const uint32_t *out_lens, uint8_t *digests, uint64_t n, cudaStream_t stream,
                        const DeviceInfo &dev) {
    int err = KB_OK;
    // SHA3GB_TUNE=full: a size class seen for the first time is tuned here
    // (synchronously), which also leaves this batch's digests.
    cudaStreamCaptureStatus cap0 = cudaStreamCaptureStatusNone;
    if (tune_mode() == TuneMode::Full && use_tuned() && tuning_get(KB_TUNE_RAGGED_SCHEDULE) == KB_SCHEDULE_QUEUE &&
        tuning_get(KB_TUNE_QUEUE_MIN_BLOCKS) == 0 && tuning_get(KB_TUNE_QUEUE_BLOCKS_PER_SM) == 0 &&
        tuning_get(KB_TUNE_QUEUE_STAGING) == 0 && tuning_get(KB_TUNE_QUEUE_WARP_MESSAGES) < 0 &&
        cudaStreamIsCapturing(stream, &cap0) == cudaSuccess && cap0 == cudaStreamCaptureStatusNone &&
        !have_tuned(n, dev))
        return autotune_ragged_queue(msgs, offsets, lens, variants, out_lens, digests, n, stream, dev, nullptr);
    const size_t bytes = queue_scratch_bytes(n);
    uint8_t *scratch = static_cast<uint8_t *>(stream_scratch(stream, bytes, &err));
    if (!scratch) return err;
    const QueueConfig cfg = choose_config(n, dev);
    const uint64_t grid = queue_grid(cfg, n, dev.device, dev.sm_count);
    const AuxStream *aux = nullptr;
    if (!cfg.lanes && !cfg.per_variant && cfg.warp_messages > 0) {
        aux = aux_for(dev.device, stream, &err);
        if (!aux) return err;
    }
    auto run = [&] {
        return queue_issue(msgs, offsets, lens, variants, out_lens, digests, n, scratch, cfg, grid, dev.sm_count,
                           dev.d_status, stream, aux);
    };

    // Graph replay needs a capturable stream that is not already capturing.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool graphs = tuning_get(KB_TUNE_GRAPHS) != 0 && stream != nullptr &&
                        cudaStreamIsCapturing(stream, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone;
    if (!graphs) return run();

    GraphKey key{{msgs, offsets, lens, variants, out_lens, digests, scratch},
                 n, stream, cfg.minb, cfg.blocks_per_sm, cfg.stage,
                 cfg.per_variant ? 2 : cfg.lanes ? 1 : 0, dev.device, cfg.warp_messages};
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
        return run();
    }
    const int rc = run();
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
        return run();
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

namespace {

__global__ void k_compare(const uint8_t *__restrict__ a, const uint8_t *__restrict__ b, uint64_t bytes,
                          unsigned int *mismatch) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < bytes; i += step)
        if (a[i] != b[i]) {
            atomicOr(mismatch, 1u);
            return;
        }
}

// The candidates of the autotuner: every compiled (register budget, staging)
// pair at its largest resident block count and the two below it, with one
// thread per message; the hybrid split is tried afterwards on the best of
// those (tune_hybrid).
std::vector<QueueConfig> base_candidates(int device) {
    std::vector<QueueConfig> out;
    for (int stage : kStageCodes) {
        for (int minb : kMinBlocksChoices) {
            const void *fn = queue_kernel(minb, stage);
            if (!fn) continue;
            const int per_sm = resident_blocks(fn, device);
            for (int bps = per_sm; bps >= 1 && bps >= per_sm - 2; --bps) {
                QueueConfig cfg;
                cfg.minb = minb;
                cfg.blocks_per_sm = bps;
                cfg.stage = stage;
                cfg.warp_messages = 0;
                out.push_back(cfg);
            }
        }
    }
    return out;
}

}  // namespace

// Autotuner: times every candidate on this batch, checks that each writes
// the same bytes as the first, and keeps the fastest for batches of the same
// size class on this device.  Then tries the hybrid split (the K costliest
// messages one warp each, K in kHybridChoices) on the winner.  Synchronous;
// allocates a reference copy of the outputs for the duration of the call.
int autotune_ragged_queue(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens, const uint8_t *variants,
                          const uint32_t *out_lens, uint8_t *digests, uint64_t n, cudaStream_t stream,
                          const DeviceInfo &dev, QueueConfig *chosen) {
    int err = KB_OK;
    uint8_t *scratch = static_cast<uint8_t *>(stream_scratch(stream, queue_scratch_bytes(n), &err));
    if (!scratch) return err;
    const AuxStream *aux = aux_for(dev.device, stream, &err);
    if (!aux) return err;
    const Buffers bf = carve(scratch, n, digest_offsets_tiles(n));
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

    // Times one candidate (one untimed run, then the timed one) and keeps it
    // when it is the fastest so far and writes the reference bytes.
    auto trial = [&](const QueueConfig &cfg) {
        const uint64_t grid = queue_grid(cfg, n, dev.device, dev.sm_count);
        auto go = [&] {
            return queue_issue(msgs, offsets, lens, variants, out_lens, digests, n, scratch, cfg, grid, dev.sm_count,
                               dev.d_status, stream, aux);
        };
        rc = go();
        if (rc == KB_OK) rc = cuda_status(cudaEventRecord(a, stream));
        if (rc == KB_OK) rc = go();
        if (rc == KB_OK) rc = cuda_status(cudaEventRecord(b, stream));
        if (rc == KB_OK) rc = cuda_status(cudaEventSynchronize(b));
        float ms = 0;
        if (rc == KB_OK) rc = cuda_status(cudaEventElapsedTime(&ms, a, b));
        if (rc != KB_OK) return;
        if (!have_ref) {
            // Output size: last digest offset + its length.
            uint64_t last_off = 0;
            uint32_t last_len = 0;
            if (cudaMemcpy(&last_off, bf.out_off + (n - 1), 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(&last_len, out_lens + (n - 1), 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = KB_ERR_CUDA;
                return;
            }
            total_out = last_off + last_len;
            if (total_out && cudaMalloc(&ref, total_out) != cudaSuccess) {
                cudaGetLastError();
                rc = KB_ERR_NOMEM;
                return;
            }
            if (total_out && cudaMemcpyAsync(ref, digests, total_out, cudaMemcpyDeviceToDevice, stream) != cudaSuccess) {
                rc = KB_ERR_CUDA;
                return;
            }
            have_ref = true;
        } else if (total_out) {
            unsigned int bad = 0;
            if (cudaMemsetAsync(mismatch, 0, sizeof bad, stream) != cudaSuccess) {
                rc = KB_ERR_CUDA;
                return;
            }
            k_compare<<<dev.sm_count * 8, 256, 0, stream>>>(ref, digests, total_out, mismatch);
            if (cudaMemcpyAsync(&bad, mismatch, sizeof bad, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess) {
                rc = KB_ERR_CUDA;
                return;
            }
            if (bad) return;  // a configuration that changes the output is never chosen
        }
        if (ms < best_t) {
            best_t = ms;
            best = cfg;
        }
    };
    for (const QueueConfig &cfg : base_candidates(dev.device)) {
        if (rc != KB_OK) break;
        trial(cfg);
    }
    // Threads per message: the hybrid split on the best configuration.
    const QueueConfig base = best;
    for (int64_t k : kHybridChoices) {
        if (rc != KB_OK || uint64_t(k) >= n) break;
        QueueConfig cfg = base;
        cfg.warp_messages = k;
        trial(cfg);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (ref) cudaFree(ref);
    if (mismatch) cudaFree(mismatch);
    if (rc != KB_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_cache_locked(dev.device, dev.sm_count);
        for (auto it = g_tuned.begin(); it != g_tuned.end();)
            it = (it->device == dev.device && it->size_class == size_class(n)) ? g_tuned.erase(it) : std::next(it);
        g_tuned.push_front(TuneEntry{dev.device, size_class(n), best});
        save_cache_entry(dev.device, dev.sm_count, size_class(n), best);
    }
    // Leave the caller's digests from the chosen configuration.
    rc = queue_issue(msgs, offsets, lens, variants, out_lens, digests, n, scratch, best,
                     queue_grid(best, n, dev.device, dev.sm_count), dev.sm_count, dev.d_status, stream, aux);
    if (chosen) {
        *chosen = best;
        chosen->ms = best_t;
    }
    return rc;
}

void forget_tuning(int device) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto it = g_tuned.begin(); it != g_tuned.end();)
        it = (device < 0 || it->device == device) ? g_tuned.erase(it) : std::next(it);
    if (device < 0) g_cache_loaded.clear();
    else g_cache_loaded.erase(device);
}

QueueConfig queue_config_for(uint64_t n, const DeviceInfo &dev) { return choose_config(n, dev); }

int queue_staging_value(const QueueConfig &cfg) { return staging_of(cfg.stage); }

}  // namespace kb
