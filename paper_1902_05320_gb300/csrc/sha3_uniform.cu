// sha3_uniform.cu -- fixed-stride batch kernel: one thread per message
// (the paper's granularity of a thread per message, Section 4.1), every
// message the same length and variant (Section 4.3).
//
// Specialisations: for each variant, a compile-time 64-byte message read with
// four 16-byte loads (one rate block: the padding folds into constants and
// round 0 runs on mostly-zero lanes), a runtime length below the rate (one
// block, round 0 on zero capacity lanes), and a general runtime length; the
// runtime forms with 8-byte aligned loads or at any alignment.  The state representation is
// a template parameter: plain 32-bit halves by default, bit-interleaved
// halves as the measured control for SHA3-256.  A grid of (occupancy x SMs)
// blocks strides over the messages.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "keccak_core.cuh"
#include "keccak_interleaved.cuh"
#include "runtime.cuh"
#include "sponge.cuh"
#include "tma.cuh"

namespace kb {
namespace {

// LEN >= 0: compile-time message length; -1: runtime; -2: runtime, below the
// rate, with at most one block of output.  A8: base and stride are multiples
// of 8 (16 when LEN == 64).
template <int V, int LEN, bool A8, class Rep>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_sha3_uniform(const uint8_t *__restrict__ msgs, uint64_t stride, uint64_t len_rt,
                   uint8_t *__restrict__ out, uint32_t out_len, uint64_t n) {
    using P = Variant<V>;
    const uint64_t len = LEN >= 0 ? uint64_t(LEN) : len_rt;
    const uint32_t dlen = P::digest ? uint32_t(P::digest) : out_len;
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t m = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; m < n; m += step) {
        const uint8_t *p = msgs + m * stride;
        uint8_t *dst = out + m * dlen;
        if constexpr (LEN == 64) {
            static_assert(64 < P::rate, "a 64-byte message is one block for every variant");
            uint32_t A[25], B[25];
#pragma unroll
            for (int i = 0; i < 25; ++i) A[i] = B[i] = 0;
            const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint4 v = __ldg(q + j);
                Rep::set_word(A[2 * j], B[2 * j], v.x, v.y);
                Rep::set_word(A[2 * j + 1], B[2 * j + 1], v.z, v.w);
            }
            // Domain byte at offset 64 (lane 8, byte 0); 0x80 at byte rate-1.
            A[8] ^= Rep::word_a(uint64_t(P::domain));
            B[8] ^= Rep::word_b(uint64_t(P::domain));
            constexpr uint64_t kEnd = uint64_t(0x80) << 56;
            A[P::rate / 8 - 1] ^= Rep::word_a(kEnd);
            B[P::rate / 8 - 1] ^= Rep::word_b(kEnd);
            const uint32_t nsq = dlen > uint32_t(P::rate) ? (dlen - 1) / P::rate : 0;
            for (uint32_t i = 0; i <= nsq; ++i) {
                if (i > 0) squeeze<P::rate, Rep>(A, B, dst + uint64_t(i - 1) * P::rate, P::rate);
                Rep::template permute<true>(A, B);
            }
            squeeze<P::rate, Rep>(A, B, dst + uint64_t(nsq) * P::rate, dlen - nsq * P::rate);
        } else if constexpr (LEN == -2) {
            // A runtime length below the rate and at most one output block:
            // the message is the padded last block and one permutation,
            // with round 0 on the known-zero capacity lanes folded.
            uint32_t A[25], B[25];
#pragma unroll
            for (int i = 0; i < 25; ++i) A[i] = B[i] = 0;
            absorb_last<P::rate, P::domain, A8, Rep>(A, B, p, uint32_t(len));
            Rep::template permute<true>(A, B);
            squeeze<P::rate, Rep>(A, B, dst, dlen);
        } else {
            sponge<P::rate, P::domain, A8, Rep>(p, len, dst, dlen);
        }
    }
}

// The 64-byte form with its messages staged through shared memory by bulk
// asynchronous copies (cp.async.bulk, completed on an mbarrier): a block takes
// tiles of kThreads consecutive messages (8 KiB, one copy issued by thread 0),
// two buffers deep, so the next tile arrives while the current one is hashed.
// Each thread reads its message from shared memory; once every thread has
// read the buffer (a proxy fence, then a block barrier) thread 0 refills it
// with the tile after next, and the hashing runs while that copy is in
// flight.  Needs stride 64 and a 16-byte aligned base in device memory.  A
// wait that outlasts kWaitNs sets KB_DEV_TIMEOUT; the block then waits
// (bounded) for its copies in flight and stops without writing the rest of
// its digests.
constexpr uint32_t kTileBytes = kThreads * 64;  // 8 KiB
constexpr uint64_t kWaitNs = 1000000000ull;     // 1 s

template <int V, class Rep>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_sha3_uniform64_tma(const uint8_t *__restrict__ msgs, uint8_t *__restrict__ out, uint32_t out_len, uint64_t n,
                         unsigned int *status) {
    using P = Variant<V>;
    static_assert(64 < P::rate, "a 64-byte message is one block for every variant");
    __shared__ __align__(128) uint8_t buf[2][kTileBytes];
    __shared__ __align__(8) uint64_t bar[2];
    const uint64_t ntiles = (n + kThreads - 1) / kThreads;
    const uint32_t dlen = P::digest ? uint32_t(P::digest) : out_len;
    const uint64_t stride = gridDim.x;
    // Thread 0 issues the copies; uses[b] counts the copies issued into buffer b.
    uint32_t uses[2] = {0, 0};
    auto issue = [&](uint64_t tile, int b) {
        const uint64_t first = tile * kThreads;
        const uint32_t bytes = uint32_t(n - first < kThreads ? n - first : uint64_t(kThreads)) * 64;
        mbar_arrive_expect_tx(&bar[b], bytes);
        bulk_copy_g2s(buf[b], msgs + first * 64, bytes, &bar[b]);
        ++uses[b];
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blockIdx.x < ntiles) issue(blockIdx.x, 0);
        if (blockIdx.x + stride < ntiles) issue(blockIdx.x + stride, 1);
    }
    uint32_t k = 0;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += stride, ++k) {
        const int b = int(k & 1);
        const bool ok = mbar_wait_bounded(&bar[b], (k >> 1) & 1, kWaitNs);
        const uint64_t m = tile * kThreads + threadIdx.x;
        uint32_t A[25], B[25];
#pragma unroll
        for (int i = 0; i < 25; ++i) A[i] = B[i] = 0;
        if (ok && m < n) {
            const uint4 *q = reinterpret_cast<const uint4 *>(buf[b] + threadIdx.x * 64);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint4 v = q[j];
                Rep::set_word(A[2 * j], B[2 * j], v.x, v.y);
                Rep::set_word(A[2 * j + 1], B[2 * j + 1], v.z, v.w);
            }
        }
        // Every thread has read buffer b (or timed out): refill it, or stop.
        // The proxy fence orders this thread's reads of b before the bulk
        // copy's writes into it.
        fence_proxy_async_smem();
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(status, KB_DEV_TIMEOUT);
                // A buffer holds at most one copy beyond the phases consumed
                // before this tile; wait (bounded) for it to land.
                for (int c = 0; c < 2; ++c) {
                    const uint32_t consumed = (k + 1 - uint32_t(c)) / 2;
                    if (uses[c] > consumed) mbar_wait_bounded(&bar[c], consumed & 1, kWaitNs);
                }
            }
            return;
        }
        if (threadIdx.x == 0 && tile + 2 * stride < ntiles) issue(tile + 2 * stride, b);
        if (m < n) {
            A[8] ^= Rep::word_a(uint64_t(P::domain));
            B[8] ^= Rep::word_b(uint64_t(P::domain));
            constexpr uint64_t kEnd = uint64_t(0x80) << 56;
            A[P::rate / 8 - 1] ^= Rep::word_a(kEnd);
            B[P::rate / 8 - 1] ^= Rep::word_b(kEnd);
            uint8_t *dst = out + m * dlen;
            const uint32_t nsq = dlen > uint32_t(P::rate) ? (dlen - 1) / P::rate : 0;
            for (uint32_t i = 0; i <= nsq; ++i) {
                if (i > 0) squeeze<P::rate, Rep>(A, B, dst + uint64_t(i - 1) * P::rate, P::rate);
                Rep::template permute<true>(A, B);
            }
            squeeze<P::rate, Rep>(A, B, dst + uint64_t(nsq) * P::rate, dlen - nsq * P::rate);
        }
    }
}

template <int V, int LEN, bool A8, class Rep>
int launch_one(const uint8_t *msgs, uint64_t stride, uint64_t len, uint32_t out_len, uint8_t *digests,
               uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    const void *fn = reinterpret_cast<const void *>(&k_sha3_uniform<V, LEN, A8, Rep>);
    // One-block messages: a grid of (occupancy x SMs) blocks strides over
    // them.  Longer messages: one message per thread and as many blocks as
    // that takes, so the block scheduler balances the last wave dynamically.
    const uint64_t need = (n + kThreads - 1) / kThreads;
    const uint64_t grid = len < uint64_t(Variant<V>::rate) ? persistent_grid(fn, kThreads, 0, n, dev)
                                                           : std::min<uint64_t>(need, uint64_t(INT32_MAX));
    k_sha3_uniform<V, LEN, A8, Rep><<<unsigned(grid), kThreads, 0, stream>>>(msgs, stride, len, digests,
                                                                              out_len, n);
    return cuda_status(cudaGetLastError());
}

template <int V>
int launch_tma(const uint8_t *msgs, uint32_t out_len, uint8_t *digests, uint64_t n, cudaStream_t stream,
               const DeviceInfo &dev) {
    const void *fn = reinterpret_cast<const void *>(&k_sha3_uniform64_tma<V, PlainRep>);
    const uint64_t grid = persistent_grid(fn, kThreads, 0, n, dev);
    k_sha3_uniform64_tma<V, PlainRep><<<unsigned(grid), kThreads, 0, stream>>>(msgs, digests, out_len, n,
                                                                                 dev.d_status);
    return cuda_status(cudaGetLastError());
}

// True when p is device memory of this device (not host-mapped, not a peer's).
bool device_resident(const void *p, int device) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

template <int V>
int launch_variant(const uint8_t *msgs, uint64_t stride, uint64_t len, uint32_t out_len, uint8_t *digests,
                   uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    const uintptr_t base = reinterpret_cast<uintptr_t>(msgs);
    const bool a16 = ((base | stride) & 15) == 0;
    const bool a8 = ((base | stride) & 7) == 0;
    if constexpr (V == 1) {
        // The bit-interleaved control, selected through the tuning interface.
        if (tuning_get(KB_TUNE_REPRESENTATION) == KB_REP_INTERLEAVED) {
            if (len == 64 && a16)
                return launch_one<V, 64, true, InterleavedRep>(msgs, stride, len, out_len, digests, n, stream, dev);
            if (a8) return launch_one<V, -1, true, InterleavedRep>(msgs, stride, len, out_len, digests, n, stream, dev);
        }
    }
    if (len == 64 && stride == 64 && a16 && tuning_get(KB_TUNE_STAGING) == KB_STAGING_TMA &&
        device_resident(msgs, dev.device))
        return launch_tma<V>(msgs, out_len, digests, n, stream, dev);
    if (len == 64 && a16) return launch_one<V, 64, true, PlainRep>(msgs, stride, len, out_len, digests, n, stream, dev);
    constexpr int rate = Variant<V>::rate;
    if (len < uint64_t(rate) && (Variant<V>::digest || out_len <= uint32_t(rate))) {
        if (a8) return launch_one<V, -2, true, PlainRep>(msgs, stride, len, out_len, digests, n, stream, dev);
        return launch_one<V, -2, false, PlainRep>(msgs, stride, len, out_len, digests, n, stream, dev);
    }
    if (a8) return launch_one<V, -1, true, PlainRep>(msgs, stride, len, out_len, digests, n, stream, dev);
    return launch_one<V, -1, false, PlainRep>(msgs, stride, len, out_len, digests, n, stream, dev);
}

}  // namespace

int launch_uniform(const uint8_t *msgs, uint64_t stride, uint64_t len, int variant, uint32_t out_len,
                   uint8_t *digests, uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    switch (variant) {
        case 0: return launch_variant<0>(msgs, stride, len, out_len, digests, n, stream, dev);
        case 1: return launch_variant<1>(msgs, stride, len, out_len, digests, n, stream, dev);
        case 2: return launch_variant<2>(msgs, stride, len, out_len, digests, n, stream, dev);
        case 3: return launch_variant<3>(msgs, stride, len, out_len, digests, n, stream, dev);
        case 4: return launch_variant<4>(msgs, stride, len, out_len, digests, n, stream, dev);
        case 5: return launch_variant<5>(msgs, stride, len, out_len, digests, n, stream, dev);
        default: return KB_ERR_INVALID;
    }
}

}  // namespace kb
