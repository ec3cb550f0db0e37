// serve.cu -- continuous-batching hash server: requests of any size and any
// of the six functions arrive one by one; the server batches whatever has
// arrived whenever a stream slot is free, admits requests against a fixed
// device-memory budget, keeps every message resident in that device arena
// while it is hashed, and reports per-request latency.
//
// Pipeline per batch (on the batch's stream slot):
//   1. the batch's request descriptors go host -> device in one copy;
//   2. k_gather copies each message from (page-locked, device-visible) host
//      memory into the batch's region of the arena, coalesced;
//   3. k_serve_hash hashes one request per thread, longest first, and writes
//      each output straight into the caller's host buffer; the thread then
//      posts the request id to a completion ring in host memory (system-scope
//      atomic), so a short request completes as soon as its own hash does,
//      not when the longest message of its batch does;
//   4. an event marks the batch done; its stream slot is reused.  A
//      short-lane batch holds one arena region until then; in the long lane
//      each request has its own region, given back as soon as its
//      completion arrives, so a finished request's bytes do not wait for the
//      longest chain of its batch.
// Host threads: the caller submits; a dispatcher forms and launches batches;
// a completer drains the completion ring and retires finished batches.  If
// the device lacks native host atomics, requests complete with their batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "arena_heap.h"
#include "keccak_core.cuh"
#include "lane_parallel.cuh"
#include "runtime.cuh"
#include "sponge.cuh"

namespace kb {
namespace {

using Clock = std::chrono::steady_clock;

struct ReqDesc {
    uint64_t src;         // host address of the message (device-visible)
    uint64_t len;         // message bytes
    uint64_t arena_off;   // where k_gather places it (16-byte aligned)
    uint64_t out;         // host address of the output (device-visible)
    uint64_t chunk_base;  // index of the request's first 16 KiB gather chunk
    uint32_t out_len;
    uint32_t id;          // request id + 1 (0 marks an empty ring slot)
    uint32_t variant;
    uint32_t pad;
};

constexpr uint64_t kGatherChunk = 16384;  // bytes per gather block
constexpr int kGatherThreads = 256;

constexpr uint64_t kRingSlots = 1u << 20;

struct CompletionRing {
    unsigned long long produced;  // written by the device (system-scope atomic)
    unsigned int pad[30];
    unsigned int slot[kRingSlots];
};

// Copies every message of the batch into the arena: each block handles one
// 16 KiB chunk of one request (found by binary search on chunk_base).
// Destination words are aligned; the source is read through the aligned
// 32-bit words that hold its bytes and funnel-shifted into place.
__global__ void __launch_bounds__(kGatherThreads)
    k_gather(const ReqDesc *__restrict__ d, uint32_t m, uint64_t total_chunks, uint8_t *__restrict__ arena) {
    for (uint64_t c = blockIdx.x; c < total_chunks; c += gridDim.x) {
        uint32_t lo = 0, hi = m - 1;  // last request with chunk_base <= c
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) / 2;
            if (d[mid].chunk_base <= c) lo = mid;
            else hi = mid - 1;
        }
        const uint64_t len = d[lo].len;
        const uint64_t begin = (c - d[lo].chunk_base) * kGatherChunk;
        if (begin >= len) continue;
        const uint64_t end = begin + kGatherChunk < len ? begin + kGatherChunk : len;
        const uint8_t *src = reinterpret_cast<const uint8_t *>(d[lo].src);
        uint8_t *dst = arena + d[lo].arena_off;
        const uint64_t nw_total = len / 4;  // whole words of the message
        const uintptr_t s0 = reinterpret_cast<uintptr_t>(src);
        const uint32_t sh = uint32_t(s0 & 3) * 8;
        const uint32_t *a = reinterpret_cast<const uint32_t *>(s0 & ~uintptr_t(3));
        uint32_t *dw = reinterpret_cast<uint32_t *>(dst);
        const uint64_t w_end = end / 4 < nw_total ? end / 4 : nw_total;
#pragma unroll 4
        for (uint64_t w = begin / 4 + threadIdx.x; w < w_end; w += kGatherThreads) {
            const uint32_t x = a[w];
            const uint32_t y = sh ? a[w + 1] : 0u;  // word w+1 holds byte 4w+3 when sh != 0
            dw[w] = __funnelshift_r(x, y, sh);
        }
        if (end == len)
            for (uint64_t b = nw_total * 4 + threadIdx.x; b < len; b += kGatherThreads) dst[b] = src[b];
    }
}

// One request per thread, in the order the host sorted them (longest first).
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_serve_hash(const ReqDesc *__restrict__ d, uint32_t m, const uint8_t *__restrict__ arena, CompletionRing *ring) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const ReqDesc q = d[r];
    sponge_rt<true, PlainRep>(arena + q.arena_off, q.len, int(q.variant), reinterpret_cast<uint8_t *>(q.out),
                              q.out_len);
    if (ring) {
        __threadfence_system();  // the output is visible before the completion
        const unsigned long long pos = atomicAdd_system(&ring->produced, 1ull);
        volatile unsigned int *slot = &ring->slot[pos & (kRingSlots - 1)];
        *slot = q.id;
    }
}

// Long requests: one warp per request (lane-parallel sponge).
__global__ void __launch_bounds__(kThreads)
    k_serve_hash_lanes(const ReqDesc *__restrict__ d, uint32_t m, const uint8_t *__restrict__ arena,
                       CompletionRing *ring) {
    const uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (r >= m) return;
    const ReqDesc q = d[r];
    lane_sponge<true>(arena + q.arena_off, q.len, int(q.variant), reinterpret_cast<uint8_t *>(q.out), q.out_len);
    __syncwarp();
    if (ring && (threadIdx.x & 31) == 0) {
        __threadfence_system();
        const unsigned long long pos = atomicAdd_system(&ring->produced, 1ull);
        volatile unsigned int *slot = &ring->slot[pos & (kRingSlots - 1)];
        *slot = q.id;
    }
}

struct Request {
    const uint8_t *msg = nullptr;
    uint64_t len = 0;
    uint8_t *out = nullptr;
    uint32_t out_len = 0;
    uint8_t variant = 0;
    int64_t t_arrive = 0;              // ns since the server started
    int64_t t_submit = 0;              // when submit() took it
    std::atomic<int64_t> t_launch{-1}; // when its batch was enqueued
    std::atomic<int64_t> t_done{-1};   // ns since the server started, -1 while pending
    uint64_t region = ~uint64_t(0);    // its own arena region in the long lane (under the lock); none: ~0
};

constexpr uint64_t kNoRegion = ~uint64_t(0);

// Request table: fixed array of chunk pointers, so readers need no lock.
constexpr uint32_t kChunk = 1u << 16;
constexpr uint32_t kMaxChunks = 1u << 12;

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    ReqDesc *h_desc = nullptr;  // page-locked
    ReqDesc *d_desc = nullptr;
    std::vector<uint32_t> ids;
    uint64_t region_start = 0, region_bytes = 0;
    bool busy = false;      // holds a batch (set by the dispatcher under the lock)
    bool launched = false;  // its completion event has been recorded
    bool per_request = false;  // each request has its own arena region (Request::region)
};

uint64_t align16(uint64_t v) { return (v + 15) & ~uint64_t(15); }

uint64_t request_cost(uint64_t len, int v, uint32_t out_len) {
    const uint64_t rate = uint64_t(variant_rate(v));
    return len / rate + 1 + (out_len > rate ? (out_len - 1) / rate : 0);
}

}  // namespace

// Requests travel in one of two lanes by cost (permutations): short ones
// never wait for a stream slot or arena space held by a long sponge chain.
struct Lane {
    std::deque<uint32_t> pending;
    std::vector<Slot> slots;
    ArenaHeap heap;         // offsets relative to `base`
    uint64_t base = 0;      // start of this lane's part of the device arena
    uint64_t max_len = 0;   // longest message the lane can hold
};

constexpr int kShortLane = 0, kLongLane = 1;

struct Server {
    kb_server_config cfg{};
    int device = -1;
    int sm_count = 1;
    uint8_t *arena = nullptr;
    CompletionRing *ring = nullptr;  // page-locked, device-visible
    bool ring_mode = false;
    uint64_t consumed = 0;
    uint64_t long_threshold = 64;     // cost (permutations) above which a request is long
    bool long_lanes_kernel = true;    // long lane: one warp per request
    Lane lanes[2];
    // Two locks, so that submitting never waits for batch formation: qmu
    // guards only the lanes' pending queues (submit pushes at the back, the
    // dispatcher alone takes from the front); mu guards the slots, the arena
    // heaps, Request::region and the stats.  Order: mu before qmu.
    std::mutex mu;
    std::mutex qmu;
    std::mutex chunk_mu;              // creation of request-table chunks
    std::condition_variable cv;
    std::unique_ptr<Request[]> chunks[kMaxChunks];
    std::atomic<uint32_t> n_requests{0};
    std::atomic<uint64_t> n_done{0};
    std::atomic<bool> stop{false};
    std::atomic<int> error{KB_OK};
    uint64_t batches = 0, max_batch_seen = 0, bytes_done = 0;
    std::atomic<uint64_t> rejected{0};
    Clock::time_point t0;
    std::thread dispatcher, completer;
    std::vector<uint32_t> candidates;  // the dispatcher's copy of a lane's oldest pending ids

    Request &req(uint32_t id) { return chunks[id / kChunk][id % kChunk]; }
    int64_t now_ns() const {
        return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
    }

    int submit(const uint8_t *msg, uint64_t len, int variant, uint32_t out_len, uint8_t *out, int64_t t_arrive,
               uint64_t *ticket) {
        if (variant < 0 || variant > 5) return KB_ERR_INVALID;
        const int dg = variant_digest(variant);
        if (dg && out_len != uint32_t(dg)) return KB_ERR_INVALID;
        if ((len && !msg) || (out_len && !out) || out_len > (1u << 20)) return KB_ERR_INVALID;
        const int lane = request_cost(len, variant, out_len) > long_threshold ? kLongLane : kShortLane;
        if (align16(len) > lanes[lane].max_len || align16(len) > cfg.max_batch_bytes) {
            rejected.fetch_add(1);
            return KB_ERR_TOO_LARGE;
        }
        const uint32_t id = n_requests.fetch_add(1);
        if (id / kChunk >= kMaxChunks) return KB_ERR_NOMEM;
        {
            std::lock_guard<std::mutex> lk(chunk_mu);
            if (!chunks[id / kChunk]) chunks[id / kChunk].reset(new Request[kChunk]);
        }
        Request &r = req(id);
        r.msg = msg;
        r.len = len;
        r.out = out;
        r.out_len = out_len;
        r.variant = uint8_t(variant);
        r.t_submit = now_ns();
        r.t_arrive = t_arrive >= 0 ? t_arrive : r.t_submit;
        r.t_launch.store(-1, std::memory_order_relaxed);
        r.t_done.store(-1);
        {
            std::lock_guard<std::mutex> lk(qmu);
            lanes[lane].pending.push_back(id);
        }
        cv.notify_all();
        if (ticket) *ticket = id;
        return KB_OK;
    }

    bool has_pending(const Lane &ln) {
        std::lock_guard<std::mutex> q(qmu);
        return !ln.pending.empty();
    }

    // Forms one batch into slot s from the lane's pending queue (mu held; qmu
    // is taken only to copy the oldest candidates and, at the end, to drop
    // the admitted ones from the front, which no other thread removes).
    // per_request: each request takes its own region of the lane's arena, in
    // arrival order while one fits, and gives it back as soon as its own
    // completion arrives (see complete_loop); otherwise the batch takes one
    // region, given back when the whole batch is done.
    bool form_batch(Lane &ln, Slot &s, bool per_request) {
        s.ids.clear();
        s.per_request = per_request;
        std::vector<uint32_t> &cand = candidates;
        {
            std::lock_guard<std::mutex> q(qmu);
            const size_t k = std::min<size_t>(ln.pending.size(), cfg.max_batch_requests);
            cand.assign(ln.pending.begin(), ln.pending.begin() + k);
        }
        auto pop_admitted = [&] {
            std::lock_guard<std::mutex> q(qmu);
            ln.pending.erase(ln.pending.begin(), ln.pending.begin() + s.ids.size());
        };
        uint64_t bytes = 0;
        if (per_request) {
            for (uint32_t id : cand) {
                Request &r = req(id);
                const uint64_t need = align16(r.len);
                if (s.ids.size() >= cfg.max_batch_requests || bytes + need > cfg.max_batch_bytes) break;
                uint64_t start = 0;
                if (!ln.heap.alloc(std::max<uint64_t>(need, 16), &start)) break;
                r.region = start;
                s.ids.push_back(id);
                bytes += need;
            }
            if (s.ids.empty()) return false;
            pop_admitted();
            s.region_start = ln.base;
            s.region_bytes = 0;
            return true;
        }
        for (uint32_t id : cand) {
            const Request &r = req(id);
            const uint64_t need = align16(r.len);
            if (s.ids.size() >= cfg.max_batch_requests || bytes + need > cfg.max_batch_bytes) break;
            s.ids.push_back(id);
            bytes += need;
        }
        if (s.ids.empty()) return false;
        uint64_t start = 0;
        // Admission: the whole batch must fit in the free part of the budget;
        // otherwise shrink it (the oldest requests stay first in line).
        while (!s.ids.empty() && !ln.heap.alloc(std::max<uint64_t>(bytes, 16), &start)) {
            bytes -= align16(req(s.ids.back()).len);
            s.ids.pop_back();
        }
        if (s.ids.empty()) return false;
        pop_admitted();
        s.region_start = ln.base + start;
        s.region_bytes = std::max<uint64_t>(bytes, 16);
        return true;
    }

    // Fills the slot's descriptors and enqueues its work (no lock held; the
    // slot is already marked busy, so no other thread touches it).  Long-lane
    // batches hash one request per warp, short-lane batches one per thread.
    int launch(Slot &s, bool lanes_kernel) {
        // Longest first, so that warps hold requests of similar cost.
        std::sort(s.ids.begin(), s.ids.end(), [&](uint32_t a, uint32_t b) {
            const Request &x = req(a), &y = req(b);
            return request_cost(x.len, x.variant, x.out_len) > request_cost(y.len, y.variant, y.out_len);
        });
        uint64_t off = s.region_start, chunks = 0;
        const int64_t t_launch = now_ns();
        for (size_t k = 0; k < s.ids.size(); ++k) {
            Request &r = req(s.ids[k]);
            r.t_launch.store(t_launch, std::memory_order_relaxed);
            ReqDesc &dsc = s.h_desc[k];
            dsc.src = reinterpret_cast<uint64_t>(r.msg);
            dsc.len = r.len;
            // (region_start is the lane's base for per-request regions)
            dsc.arena_off = s.per_request ? s.region_start + r.region : off;
            dsc.out = reinterpret_cast<uint64_t>(r.out);
            dsc.chunk_base = chunks;
            dsc.out_len = r.out_len;
            dsc.id = s.ids[k] + 1;
            dsc.variant = r.variant;
            dsc.pad = 0;
            off += align16(r.len);
            chunks += r.len ? (r.len + kGatherChunk - 1) / kGatherChunk : 1;
        }
        const uint32_t m = uint32_t(s.ids.size());
        NvtxRange range(lanes_kernel ? "kb_server batch (long lane)" : "kb_server batch (short lane)");
        cudaError_t e = cudaMemcpyAsync(s.d_desc, s.h_desc, sizeof(ReqDesc) * m, cudaMemcpyHostToDevice, s.stream);
        if (e == cudaSuccess) {
            const uint64_t gblocks = std::min<uint64_t>(chunks, uint64_t(sm_count) * 16);
            k_gather<<<unsigned(gblocks), kGatherThreads, 0, s.stream>>>(s.d_desc, m, chunks, arena);
            if (lanes_kernel)
                k_serve_hash_lanes<<<(m * 32 + kThreads - 1) / kThreads, kThreads, 0, s.stream>>>(
                    s.d_desc, m, arena, ring_mode ? ring : nullptr);
            else
                k_serve_hash<<<(m + kThreads - 1) / kThreads, kThreads, 0, s.stream>>>(s.d_desc, m, arena,
                                                                                       ring_mode ? ring : nullptr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
        return e == cudaSuccess ? KB_OK : KB_ERR_CUDA;
    }

    void dispatch_loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop.load()) {
            bool launched_any = false;
            for (int li = 0; li < 2; ++li) {
                Lane &ln = lanes[li];
                if (!has_pending(ln)) continue;
                Slot *slot = nullptr;
                for (auto &sl : ln.slots)
                    if (!sl.busy) {
                        slot = &sl;
                        break;
                    }
                if (!slot || !form_batch(ln, *slot, li == kLongLane && ring_mode)) continue;
                slot->busy = true;
                slot->launched = false;
                ++batches;
                max_batch_seen = std::max<uint64_t>(max_batch_seen, slot->ids.size());
                lk.unlock();
                const int rc = launch(*slot, li == kLongLane && long_lanes_kernel);
                lk.lock();
                if (rc != KB_OK) error.store(rc);
                slot->launched = true;
                launched_any = true;
            }
            if (!launched_any) cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }

    void complete(uint32_t id, int64_t t) {
        Request &r = req(id);
        if (r.t_done.load() < 0) {
            r.t_done.store(t);
            n_done.fetch_add(1);
        }
    }

    // Gives back the arena region of a request that has its own (lock held).
    void release_region(uint32_t id) {
        Request &r = req(id);
        if (r.region == kNoRegion) return;
        lanes[kLongLane].heap.free(r.region);
        r.region = kNoRegion;
    }

    void complete_loop() {
        cudaSetDevice(device);
        std::vector<uint32_t> finished;  // completed this pass, in ring order
        while (true) {
            bool progress = false;
            finished.clear();
            if (ring_mode) {
                volatile unsigned long long *prod = &ring->produced;
                const unsigned long long p = *prod;
                while (consumed < p) {
                    volatile unsigned int *slot = &ring->slot[consumed & (kRingSlots - 1)];
                    unsigned int v = 0;
                    for (int spin = 0; spin < (1 << 20) && (v = *slot) == 0; ++spin) {
                    }
                    if (v == 0) break;  // written late; pick it up next pass
                    *slot = 0;
                    complete(v - 1, now_ns());
                    finished.push_back(v - 1);
                    ++consumed;
                    progress = true;
                }
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                // A finished request's own region can take new messages at
                // once: its hashing has read them (the ring entry is posted
                // after the sponge), whatever the rest of its batch is doing.
                for (uint32_t id : finished) release_region(id);
                for (Lane &ln : lanes)
                for (auto &s : ln.slots) {
                    if (!s.busy || !s.launched) continue;
                    const cudaError_t q = cudaEventQuery(s.done);
                    if (q == cudaErrorNotReady) continue;
                    if (q != cudaSuccess) error.store(KB_ERR_CUDA);
                    const int64_t t = now_ns();
                    for (uint32_t id : s.ids) {
                        if (!ring_mode) complete(id, t);
                        bytes_done += req(id).len;
                    }
                    if (s.per_request) {
                        for (uint32_t id : s.ids) release_region(id);  // any whose entry is not read yet
                    } else {
                        ln.heap.free(s.region_start - ln.base);
                    }
                    s.busy = false;
                    progress = true;
                }
            }
            if (progress) cv.notify_all();
            if (stop.load()) {
                bool idle = true;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    for (Lane &ln : lanes)
                        for (auto &s : ln.slots) idle = idle && !s.busy;
                }
                const volatile unsigned long long *prod = &ring->produced;
                if (idle && (!ring_mode || consumed == *prod)) break;
            }
            if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(2));
        }
    }

    int drain(int timeout_ms) {
        const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 1 << 30 : timeout_ms);
        while (n_done.load() < n_requests.load()) {
            if (error.load() != KB_OK) return error.load();
            if (Clock::now() > deadline) return KB_ERR_TIMEOUT;
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        return error.load();
    }
};

}  // namespace kb

using namespace kb;

extern "C" {

kb_server *kb_server_create(const kb_server_config *cfg, int *status) {
    int st = KB_OK;
    Server *s = nullptr;
    do {
        if (!cfg || cfg->hbm_budget_bytes < 4096 || cfg->max_inflight < 1 || cfg->max_inflight > 64 ||
            cfg->max_batch_requests < 1 || cfg->max_batch_requests > 65536 || cfg->max_batch_bytes < 16) {
            st = KB_ERR_INVALID;
            break;
        }
        s = new Server();
        s->cfg = *cfg;
        s->cfg.max_batch_bytes = std::min(cfg->max_batch_bytes, cfg->hbm_budget_bytes);
        if (cudaGetDevice(&s->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
            st = KB_ERR_CUDA;
            break;
        }
        int native = 0;
        cudaDeviceGetAttribute(&native, cudaDevAttrHostNativeAtomicSupported, s->device);
        s->ring_mode = native != 0;
        if (cudaMalloc(&s->arena, cfg->hbm_budget_bytes) != cudaSuccess) {
            cudaGetLastError();
            st = KB_ERR_NOMEM;
            break;
        }
        // The short lane gets an eighth of the budget (short requests carry few
        // bytes), the long lane the rest.
        const uint64_t total = cfg->hbm_budget_bytes & ~uint64_t(255);
        const uint64_t short_bytes = (total / 8) & ~uint64_t(255);
        s->long_threshold = cfg->long_threshold_perms ? cfg->long_threshold_perms : 64;
        s->long_lanes_kernel = cfg->long_lane_kernel != KB_SERVER_LONG_THREAD_PER_REQUEST;
        s->lanes[kShortLane].base = 0;
        s->lanes[kShortLane].heap.reset(short_bytes);
        s->lanes[kShortLane].max_len = short_bytes;
        s->lanes[kLongLane].base = short_bytes;
        s->lanes[kLongLane].heap.reset(total - short_bytes);
        s->lanes[kLongLane].max_len = total - short_bytes;
        if (cudaHostAlloc(&s->ring, sizeof(CompletionRing), cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            st = KB_ERR_NOMEM;
            break;
        }
        std::memset(s->ring, 0, sizeof(CompletionRing));
        for (Lane &ln : s->lanes) ln.slots.resize(cfg->max_inflight);
        for (Lane &ln : s->lanes)
        for (auto &sl : ln.slots) {
            if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
                cudaHostAlloc(&sl.h_desc, sizeof(ReqDesc) * cfg->max_batch_requests, cudaHostAllocDefault) !=
                    cudaSuccess ||
                cudaMalloc(&sl.d_desc, sizeof(ReqDesc) * cfg->max_batch_requests) != cudaSuccess) {
                cudaGetLastError();
                st = KB_ERR_NOMEM;
                break;
            }
        }
        if (st != KB_OK) break;
        s->t0 = Clock::now();
        s->dispatcher = std::thread([s] { s->dispatch_loop(); });
        s->completer = std::thread([s] { s->complete_loop(); });
    } while (false);
    if (st != KB_OK && s) {
        kb_server_destroy(reinterpret_cast<kb_server *>(s));
        s = nullptr;
    }
    if (status) *status = st;
    return reinterpret_cast<kb_server *>(s);
}

void kb_server_destroy(kb_server *handle) {
    Server *s = reinterpret_cast<Server *>(handle);
    if (!s) return;
    if (s->dispatcher.joinable() || s->completer.joinable()) {
        s->drain(60000);
        s->stop.store(true);
        s->cv.notify_all();
        if (s->dispatcher.joinable()) s->dispatcher.join();
        if (s->completer.joinable()) s->completer.join();
    }
    for (Lane &ln : s->lanes)
    for (auto &sl : ln.slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
        if (sl.d_desc) cudaFree(sl.d_desc);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->ring) cudaFreeHost(s->ring);
    if (s->arena) cudaFree(s->arena);
    delete s;
}

int kb_server_submit(kb_server *handle, const uint8_t *msg, uint64_t len, int variant, uint32_t out_len,
                     uint8_t *out, uint64_t *ticket) {
    Server *s = reinterpret_cast<Server *>(handle);
    if (!s) return KB_ERR_INVALID;
    return s->submit(msg, len, variant, out_len, out, -1, ticket);
}

int kb_server_wait(kb_server *handle, uint64_t ticket, int timeout_ms) {
    Server *s = reinterpret_cast<Server *>(handle);
    if (!s || ticket >= s->n_requests.load()) return KB_ERR_INVALID;
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 1 << 30 : timeout_ms);
    while (s->req(uint32_t(ticket)).t_done.load() < 0) {
        if (s->error.load() != KB_OK) return s->error.load();
        if (Clock::now() > deadline) return KB_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    return KB_OK;
}

int kb_server_drain(kb_server *handle, int timeout_ms) {
    Server *s = reinterpret_cast<Server *>(handle);
    return s ? s->drain(timeout_ms) : KB_ERR_INVALID;
}

int kb_server_replay(kb_server *handle, const uint8_t *pool, const uint64_t *offsets, const uint64_t *lens,
                     const uint8_t *variants, const uint32_t *out_lens, const int64_t *arrival_ns, uint64_t n,
                     uint8_t *outputs, int64_t *latency_ns, kb_server_stats *stats) {
    Server *s = reinterpret_cast<Server *>(handle);
    if (!s || !offsets || !lens || !variants || !out_lens || !arrival_ns || (n && !outputs)) return KB_ERR_INVALID;
    if (n == 0) return KB_OK;
    const uint32_t first = s->n_requests.load();
    if (first + n > uint64_t(kChunk) * kMaxChunks) return KB_ERR_TOO_LARGE;
    std::vector<uint64_t> out_pos(n);
    uint64_t acc = 0;
    for (uint64_t i = 0; i < n; ++i) {
        out_pos[i] = acc;
        acc += out_lens[i];
    }
    const int64_t base = s->now_ns() + 1000000;  // first arrival 1 ms from now
    int rc = KB_OK;
    for (uint64_t i = 0; i < n && rc == KB_OK; ++i) {
        const int64_t target = base + arrival_ns[i];
        int64_t t;
        while ((t = s->now_ns()) < target) {
            if (target - t > 200000) std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        rc = s->submit(pool + offsets[i], lens[i], variants[i], out_lens[i], outputs + out_pos[i], target, nullptr);
    }
    if (rc != KB_OK) return rc;
    rc = s->drain(-1);
    if (rc != KB_OK) return rc;
    std::vector<int64_t> lat(n);
    int64_t last = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const Request &r = s->req(uint32_t(first + i));
        lat[i] = r.t_done.load() - r.t_arrive;
        last = std::max(last, r.t_done.load());
        if (latency_ns) latency_ns[i] = lat[i];
    }
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        std::vector<int64_t> sorted = lat;
        std::sort(sorted.begin(), sorted.end());
        auto pct = [&](double q) {
            const size_t k = std::min<size_t>(n - 1, size_t(q * double(n)));
            return double(sorted[k]) / 1e3;
        };
        double sum = 0;
        uint64_t bytes = 0;
        for (uint64_t i = 0; i < n; ++i) {
            sum += double(lat[i]);
            bytes += lens[i];
        }
        const double wall = double(last - (base + arrival_ns[0])) / 1e9;
        stats->requests = n;
        stats->message_bytes = bytes;
        stats->wall_s = wall;
        stats->throughput_rps = wall > 0 ? double(n) / wall : 0;
        stats->throughput_gbs = wall > 0 ? double(bytes) / wall / 1e9 : 0;
        stats->lat_mean_us = sum / double(n) / 1e3;
        stats->lat_p50_us = pct(0.50);
        stats->lat_p90_us = pct(0.90);
        stats->lat_p99_us = pct(0.99);
        stats->lat_p999_us = pct(0.999);
        stats->lat_max_us = double(sorted[n - 1]) / 1e3;
        // The latency's parts: submit lag, queue wait, service.
        std::vector<int64_t> part(n);
        auto pct_of = [&](auto get, double q) {
            for (uint64_t i = 0; i < n; ++i) part[i] = get(s->req(uint32_t(first + i)));
            const size_t k = std::min<size_t>(n - 1, size_t(q * double(n)));
            std::nth_element(part.begin(), part.begin() + k, part.end());
            return double(part[k]) / 1e3;
        };
        auto lag = [](const Request &r) { return r.t_submit - r.t_arrive; };
        auto wait = [](const Request &r) { return r.t_launch.load(std::memory_order_relaxed) - r.t_submit; };
        auto service = [](const Request &r) { return r.t_done.load() - r.t_launch.load(std::memory_order_relaxed); };
        stats->submit_lag_p50_us = pct_of(lag, 0.50);
        stats->submit_lag_p99_us = pct_of(lag, 0.99);
        stats->queue_wait_p50_us = pct_of(wait, 0.50);
        stats->queue_wait_p99_us = pct_of(wait, 0.99);
        stats->service_p50_us = pct_of(service, 0.50);
        stats->service_p99_us = pct_of(service, 0.99);
        std::lock_guard<std::mutex> lk(s->mu);
        stats->batches = s->batches;
        stats->max_batch_requests_seen = s->max_batch_seen;
        stats->peak_arena_bytes = s->lanes[0].heap.peak() + s->lanes[1].heap.peak();
        stats->rejected = s->rejected.load();
        stats->completion_ring = s->ring_mode ? 1 : 0;
    }
    return KB_OK;
}

}  // extern "C"
