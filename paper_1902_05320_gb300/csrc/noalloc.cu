// noalloc.cu -- keccak_batch_noalloc: the ragged batch entry point for callers
// that must not allocate device memory.
//
// keccak_batch keeps its scratch (the queue's control block, the digest
// offsets and the work order) in arenas it allocates with cudaMalloc on first
// use and when a larger batch arrives.  Some callers cannot let that happen:
// a serving process that reserves all device memory up front under a fixed
// budget, a plugin or real-time host whose rules forbid cudaMalloc (it can
// synchronise the whole device and stall unrelated work), or code that must
// know its memory footprint before it runs.  This entry point runs the same
// cost-bucketed queue (its prep, plan, scatter and hashing kernels, in the
// built-in configuration, one thread per message, launched directly without
// a graph) with the scratch in a fixed, file-scope device array instead:
// every GPU that loads the library holds that array until the process exits,
// and no call here allocates or frees device memory.
//
// The array is shared by every call: each call overwrites it, so calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race and must be serialised by the caller.  The control block and the
// status word are cleared at the start of each call; the other parts are
// written before they are read.  Its device address is looked up with
// cudaGetSymbolAddress on the first call in each CUDA context (with that
// context current); that first call should therefore come before any stream
// capture.
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "queue.cuh"
#include "queue_host.h"

namespace kb {
namespace {

constexpr uint64_t kMaxMessages = KB_NOALLOC_MAX_MESSAGES;
constexpr size_t kStatusBytes = 256;
constexpr size_t kQueueBytes = queue_scratch_size(kMaxMessages);
constexpr size_t kScratchBytes = kStatusBytes + kQueueBytes;
static_assert(kScratchBytes == KB_NOALLOC_SCRATCH_BYTES, "the header's stated size must match the array");

// Layout: [status word (256 B) | the queue's scratch for kMaxMessages].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Setup {
    unsigned char *scratch = nullptr;  // device address of the array in this context
    int sms = 0, device = -1;
};

std::mutex g_mu;
std::map<CUcontext, Setup> g_setup;  // per CUDA context (a module's globals live per context)

using CtxGetCurrent = CUresult (*)(CUcontext *);

CUcontext current_context() {
    static CtxGetCurrent fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        cudaGetLastError();
        return reinterpret_cast<CtxGetCurrent>(p);
    }();
    CUcontext ctx = nullptr;
    if (!fn || fn(&ctx) != CUDA_SUCCESS) return nullptr;
    return ctx;
}

// First call in the current context: look up the array's device address.
int setup(Setup *out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return KB_ERR_CUDA;
    CUcontext ctx = current_context();
    if (!ctx) {
        // No context is current on this thread yet: make the device's primary
        // context current (cudaSetDevice initialises it; nothing is allocated).
        if (cudaSetDevice(dev) != cudaSuccess) return KB_ERR_CUDA;
        ctx = current_context();
        if (!ctx) return KB_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_setup.find(ctx);
    if (it != g_setup.end() && it->second.device == dev) {
        *out = it->second;
        return KB_OK;
    }
    Setup s;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return KB_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return KB_ERR_CUDA;
    }
    s.scratch = static_cast<unsigned char *>(p);
    s.device = dev;
    g_setup[ctx] = s;
    *out = s;
    return KB_OK;
}

}  // namespace

// Forgets every cached address (keccak_release), so the next call looks it
// up again, e.g. after cudaDeviceReset.
void forget_noalloc_setup() {
    std::lock_guard<std::mutex> lk(g_mu);
    g_setup.clear();
}

}  // namespace kb

using namespace kb;

extern "C" int keccak_batch_noalloc(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                                    const uint8_t *variant, const uint32_t *out_lens, uint8_t *digests,
                                    uint64_t n, void *stream) {
    if (n == 0) return KB_OK;
    if (n > kMaxMessages) return KB_ERR_TOO_LARGE;
    if (!msgs || !offsets || !lens || !variant || !out_lens || !digests) return KB_ERR_INVALID;
    Setup s;
    int err = setup(&s);
    if (err != KB_OK) return err;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int *status = reinterpret_cast<unsigned int *>(s.scratch);
    uint8_t *queue_scratch = s.scratch + kStatusBytes;
    // Built-in configuration, one thread per message (no side stream needed).
    QueueConfig cfg;
    cfg.warp_messages = 0;
    // The status word must start at zero; the control block is cleared by
    // queue_issue itself.
    if (cudaMemsetAsync(status, 0, sizeof(unsigned int), st) != cudaSuccess) return KB_ERR_CUDA;
    const uint64_t grid = queue_grid_for(cfg, n, s.device, s.sms);
    return queue_issue(msgs, offsets, lens, variant, out_lens, digests, n, queue_scratch, cfg, grid, s.sms, status,
                       st, nullptr);
}
