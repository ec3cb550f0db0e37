// runtime.cu -- per-device state, per-stream scratch arenas and grid sizing.
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>
#include <utility>

#include "runtime.cuh"

namespace kb {
namespace {

struct Arena {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct DeviceSlot {
    DeviceInfo info;
    std::map<cudaStream_t, Arena> arenas;
    std::map<std::tuple<const void *, int, size_t>, int> occupancy;  // blocks/SM per (kernel, threads, smem)
};

std::mutex g_mu;
std::map<int, DeviceSlot> g_devices;

DeviceSlot *slot_for_current(int *err) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        *err = KB_ERR_CUDA;
        return nullptr;
    }
    auto it = g_devices.find(dev);
    if (it != g_devices.end()) return &it->second;
    DeviceSlot s;
    s.info.device = dev;
    if (cudaDeviceGetAttribute(&s.info.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaMalloc(&s.info.d_status, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(s.info.d_status, 0, sizeof(unsigned int)) != cudaSuccess) {
        *err = KB_ERR_CUDA;
        return nullptr;
    }
    return &g_devices.emplace(dev, std::move(s)).first->second;
}

}  // namespace

DeviceInfo *device_info(int *err) {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceSlot *s = slot_for_current(err);
    return s ? &s->info : nullptr;
}

void *stream_scratch(cudaStream_t stream, size_t bytes, int *err) {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceSlot *s = slot_for_current(err);
    if (!s) return nullptr;
    Arena &a = s->arenas[stream];
    if (a.bytes >= bytes && a.ptr) return a.ptr;
    if (a.ptr) {
        // Work already enqueued on this stream may still use the old block.
        if (cudaStreamSynchronize(stream) != cudaSuccess) {
            *err = KB_ERR_CUDA;
            return nullptr;
        }
        cudaFree(a.ptr);
        a.ptr = nullptr;
        a.bytes = 0;
    }
    size_t want = bytes < (size_t(1) << 20) ? (size_t(1) << 20) : bytes + bytes / 4;
    if (cudaMalloc(&a.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        a.ptr = nullptr;
        *err = KB_ERR_NOMEM;
        return nullptr;
    }
    a.bytes = want;
    return a.ptr;
}

void release_device() {
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    auto it = g_devices.find(dev);
    if (it == g_devices.end()) return;
    cudaDeviceSynchronize();
    for (auto &kv : it->second.arenas)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    if (it->second.info.d_status) cudaFree(it->second.info.d_status);
    g_devices.erase(it);
}

namespace {
constexpr int kTuneKeys = 10;
// Defaults: plain layout, cost-bucketed queue, graphs on, tuned configs used,
// register budget and blocks per SM from the tuner (or built-in defaults),
// host buffers staged through device memory, packed 64-byte messages staged
// through shared memory by bulk copies, queue staging and warp-per-message
// share from the tuner (or built-in defaults).
std::atomic<int64_t> g_tuning[kTuneKeys] = {{KB_REP_PLAIN}, {KB_SCHEDULE_QUEUE}, {1}, {1}, {0}, {0},
                                            {KB_HOST_PATH_AUTO}, {KB_STAGING_TMA}, {0}, {-1}};
}  // namespace

int64_t tuning_get(int key) { return (key >= 0 && key < kTuneKeys) ? g_tuning[key].load() : -1; }

int tuning_set(int key, int64_t value) {
    switch (key) {
        case KB_TUNE_REPRESENTATION:
            if (value != KB_REP_PLAIN && value != KB_REP_INTERLEAVED) return KB_ERR_INVALID;
            break;
        case KB_TUNE_RAGGED_SCHEDULE:
            if (value < KB_SCHEDULE_INPUT_ORDER || value > KB_SCHEDULE_PER_VARIANT) return KB_ERR_INVALID;
            break;
        case KB_TUNE_GRAPHS:
        case KB_TUNE_AUTOTUNE:
            if (value != 0 && value != 1) return KB_ERR_INVALID;
            break;
        case KB_TUNE_QUEUE_MIN_BLOCKS:
            if (value != 0 && (value < 2 || value > 6) && value != 8) return KB_ERR_INVALID;
            break;
        case KB_TUNE_QUEUE_BLOCKS_PER_SM:
            if (value < 0 || value > 32) return KB_ERR_INVALID;
            break;
        case KB_TUNE_HOST_PATH:
            if (value < KB_HOST_PATH_AUTO || value > KB_HOST_PATH_ZERO_COPY) return KB_ERR_INVALID;
            break;
        case KB_TUNE_STAGING:
            if (value != KB_STAGING_DIRECT && value != KB_STAGING_TMA) return KB_ERR_INVALID;
            break;
        case KB_TUNE_QUEUE_STAGING:
            if (value < 0 || value > KB_QUEUE_STAGING_REGS) return KB_ERR_INVALID;
            break;
        case KB_TUNE_QUEUE_WARP_MESSAGES:
            if (value < -1 || value > int64_t(UINT32_MAX)) return KB_ERR_INVALID;
            break;
        default:
            return KB_ERR_INVALID;
    }
    g_tuning[key].store(value);
    return KB_OK;
}

// Resident blocks of `threads` per SM for kernel `fn` (occupancy API, cached).
static int blocks_per_sm(const void *fn, int threads, size_t smem, const DeviceInfo &dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto &slot = g_devices[dev.device];
    const auto key = std::make_tuple(fn, threads, smem);
    auto it = slot.occupancy.find(key);
    if (it != slot.occupancy.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    slot.occupancy[key] = per_sm;
    return per_sm;
}

uint64_t persistent_grid(const void *fn, int threads, size_t smem, uint64_t work_items,
                         const DeviceInfo &dev) {
    const int per_sm = blocks_per_sm(fn, threads, smem, dev);
    const uint64_t full = uint64_t(per_sm) * uint64_t(dev.sm_count);
    const uint64_t need = (work_items + threads - 1) / threads;
    uint64_t g = need < full ? need : full;
    return g < 1 ? 1 : g;
}

}  // namespace kb
