// noalloc.cu -- keccak_batch_noalloc: the ragged batch entry point for callers
// that must not allocate device memory.
//
// keccak_batch keeps its scratch (the digest offsets of the messages) in
// arenas it allocates with cudaMalloc on first use and when a larger batch
// arrives.  Some callers cannot let that happen: a serving process that
// reserves all device memory up front under a fixed budget, a plugin or
// real-time host whose rules forbid cudaMalloc (it can synchronise the whole
// device and stall unrelated work), or code that must know its memory
// footprint before it runs.  This entry point gives them the same kernels
// with the scratch in a fixed, file-scope device array instead: every GPU
// that loads the library holds that array until the process exits, and no
// call here allocates or frees device memory.
//
// The array is shared by every call: each call overwrites it, so calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race and must be serialised by the caller.  Its device address is looked up
// with cudaGetSymbolAddress on the first call on each device (with that
// device current); that first call should therefore come before any stream
// capture.
#include <cuda_runtime.h>

#include <mutex>

#include "runtime.cuh"

namespace kb {
namespace {

constexpr uint64_t kMaxMessages = KB_NOALLOC_MAX_MESSAGES;
// The digest-offset scan uses tiles of at least 1024 messages.
constexpr uint64_t kMaxTiles = (kMaxMessages + 1023) / 1024;
constexpr size_t kStatusBytes = 256;
constexpr size_t kScratchBytes = kStatusBytes + 8 * kMaxMessages + 8 * kMaxTiles;

// Layout: [status word | out_off[kMaxMessages] | tile_sums[kMaxTiles]].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch[kMaxDevices];  // device address of the array, per device
int g_sms[kMaxDevices];

// First call on `dev` (current): look up the array's device address.
int setup(int dev, unsigned char **scratch, int *sms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return KB_ERR_CUDA;
        }
        int count = 0;
        if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return KB_ERR_CUDA;
        }
        g_sms[dev] = count;
        g_scratch[dev] = static_cast<unsigned char *>(p);
    }
    *scratch = g_scratch[dev];
    *sms = g_sms[dev];
    return KB_OK;
}

}  // namespace
}  // namespace kb

using namespace kb;

extern "C" int keccak_batch_noalloc(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                                    const uint8_t *variant, const uint32_t *out_lens, uint8_t *digests,
                                    uint64_t n, void *stream) {
    if (n == 0) return KB_OK;
    if (n > kMaxMessages) return KB_ERR_TOO_LARGE;
    if (!msgs || !offsets || !lens || !variant || !out_lens || !digests) return KB_ERR_INVALID;
    if (digest_offsets_tiles(n) > kMaxTiles) return KB_ERR_TOO_LARGE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KB_ERR_CUDA;
    unsigned char *scratch = nullptr;
    int sms = 0;
    int err = setup(dev, &scratch, &sms);
    if (err != KB_OK) return err;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned int *status = reinterpret_cast<unsigned int *>(scratch);
    uint64_t *out_off = reinterpret_cast<uint64_t *>(scratch + kStatusBytes);
    uint64_t *tile_sums = out_off + kMaxMessages;
    // The status word is the only part that must start at zero.
    if (cudaMemsetAsync(status, 0, sizeof(unsigned int), s) != cudaSuccess) return KB_ERR_CUDA;
    return launch_ragged_external(msgs, offsets, lens, variant, out_lens, digests, n, out_off, tile_sums, status,
                                  sms, s);
}
