// stream.cu -- incremental (streaming) hashing of many messages at once: each
// message has a sponge state in device memory that absorbs pieces of any
// length across calls and is finalised into its digest.  The state is the
// sponge of Section 3.2 paused between absorbed blocks: the 25 lanes plus the
// bytes of a block not yet complete.
//
// State layout (KB_STATE_BYTES = 384 bytes per message, 8-byte aligned):
//   [0, 200)    25 lanes, little-endian 64-bit words (lane x + 5y)
//   [200, 368)  pending bytes of the current block (at most rate - 1)
//   368         u32 number of pending bytes
//   372         u8 variant
//   373         u8 1 after keccak_stream_final (further absorbs are refused)
//   376         u64 total bytes absorbed
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "keccak_core.cuh"
#include "runtime.cuh"
#include "sponge.cuh"

namespace kb {
namespace {

constexpr uint32_t kStateBytes = KB_STATE_BYTES;
constexpr uint32_t kBufOff = 200, kNbufOff = 368, kVarOff = 372, kDoneOff = 373, kTotalOff = 376;

__device__ __forceinline__ void load_lanes(const uint8_t *st, uint32_t (&A)[25], uint32_t (&B)[25]) {
    const uint2 *w = reinterpret_cast<const uint2 *>(st);
#pragma unroll
    for (int i = 0; i < 25; ++i) {
        const uint2 v = w[i];
        A[i] = v.x;
        B[i] = v.y;
    }
}

__device__ __forceinline__ void store_lanes(uint8_t *st, const uint32_t (&A)[25], const uint32_t (&B)[25]) {
    uint2 *w = reinterpret_cast<uint2 *>(st);
#pragma unroll
    for (int i = 0; i < 25; ++i) w[i] = make_uint2(A[i], B[i]);
}

__global__ void __launch_bounds__(kThreads) k_stream_init(uint8_t *states, const uint8_t *variants, uint64_t n,
                                                          unsigned int *status) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
        uint8_t *st = states + i * kStateBytes;
        uint2 *w = reinterpret_cast<uint2 *>(st);
        for (uint32_t k = 0; k < kStateBytes / 8; ++k) w[k] = make_uint2(0, 0);
        const uint8_t v = variants[i];
        st[kVarOff] = v;
        if (v > 5) atomicOr(status, KB_DEV_BAD_VARIANT);
    }
}

// Appends message i's chunk to its state: completes the pending block first,
// then absorbs whole blocks straight from the chunk, then keeps the rest.
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_stream_absorb(uint8_t *states, const uint8_t *__restrict__ msgs, const uint64_t *__restrict__ offsets,
                    const uint64_t *__restrict__ lens, uint64_t n, unsigned int *status) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
        uint8_t *st = states + i * kStateBytes;
        const int v = st[kVarOff];
        uint64_t len = lens[i];
        if (v > 5 || st[kDoneOff]) {
            if (len) atomicOr(status, v > 5 ? KB_DEV_BAD_VARIANT : KB_DEV_BAD_OUTLEN);
            continue;
        }
        if (len == 0) continue;
        const uint32_t rate = uint32_t(variant_rate(v));
        const int nwords = int(rate / 8);
        const uint8_t *p = msgs + offsets[i];
        uint8_t *buf = st + kBufOff;
        uint32_t nbuf = *reinterpret_cast<uint32_t *>(st + kNbufOff);
        *reinterpret_cast<uint64_t *>(st + kTotalOff) += len;
        uint32_t A[25], B[25];
        load_lanes(st, A, B);
        bool dirty = false;
        if (nbuf) {  // top up the pending block
            const uint32_t take = len < rate - nbuf ? uint32_t(len) : rate - nbuf;
            for (uint32_t k = 0; k < take; ++k) buf[nbuf + k] = p[k];
            nbuf += take;
            p += take;
            len -= take;
            if (nbuf == rate) {
                absorb_full_rt<true, PlainRep>(A, B, buf, nwords);
                PlainRep::permute<false>(A, B);
                nbuf = 0;
                dirty = true;
            }
        }
        while (len >= rate) {
            absorb_full_rt<false, PlainRep>(A, B, p, nwords);
            PlainRep::permute<false>(A, B);
            p += rate;
            len -= rate;
            dirty = true;
        }
        for (uint32_t k = 0; k < uint32_t(len); ++k) buf[nbuf + k] = p[k];
        nbuf += uint32_t(len);
        *reinterpret_cast<uint32_t *>(st + kNbufOff) = nbuf;
        if (dirty) store_lanes(st, A, B);
    }
}

__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_stream_final(uint8_t *states, const uint32_t *__restrict__ out_lens, const uint64_t *__restrict__ out_off,
                   uint8_t *__restrict__ digests, uint64_t n, unsigned int *status) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
        uint8_t *st = states + i * kStateBytes;
        const int v = st[kVarOff];
        const uint32_t dlen = out_lens[i];
        if (v > 5) {
            atomicOr(status, KB_DEV_BAD_VARIANT);
            continue;
        }
        if (st[kDoneOff] || (v < 4 && dlen != uint32_t(variant_digest(v)))) {
            atomicOr(status, KB_DEV_BAD_OUTLEN);
            continue;
        }
        const uint32_t rate = uint32_t(variant_rate(v));
        const int nwords = int(rate / 8);
        const uint32_t nbuf = *reinterpret_cast<const uint32_t *>(st + kNbufOff);
        uint32_t A[25], B[25];
        load_lanes(st, A, B);
        absorb_last_rt<true, PlainRep>(A, B, st + kBufOff, nbuf, nwords, rt_domain(v));
        PlainRep::permute<false>(A, B);
        uint8_t *dst = digests + out_off[i];
        const uint32_t nsq = dlen > rate ? (dlen - 1) / rate : 0;
        for (uint32_t j = 0; j < nsq; ++j) {
            squeeze_rt<PlainRep>(A, B, dst + uint64_t(j) * rate, rate);
            PlainRep::permute<false>(A, B);
        }
        if (dlen > nsq * rate) squeeze_rt<PlainRep>(A, B, dst + uint64_t(nsq) * rate, dlen - nsq * rate);
        st[kDoneOff] = 1;
    }
}

// One thread per message and as many blocks as that takes (the block
// scheduler balances the last wave; a grid-stride split would give some
// threads one message more than others).
uint64_t grid_for(const void *, uint64_t n, const DeviceInfo &) {
    return std::min<uint64_t>((n + kThreads - 1) / kThreads, uint64_t(INT32_MAX));
}

}  // namespace

int launch_stream_init(uint8_t *states, const uint8_t *variants, uint64_t n, cudaStream_t stream,
                       const DeviceInfo &dev) {
    const uint64_t g = grid_for(reinterpret_cast<const void *>(&k_stream_init), n, dev);
    k_stream_init<<<unsigned(g), kThreads, 0, stream>>>(states, variants, n, dev.d_status);
    return cuda_status(cudaGetLastError());
}

int launch_stream_absorb(uint8_t *states, const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                         uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    const uint64_t g = grid_for(reinterpret_cast<const void *>(&k_stream_absorb), n, dev);
    k_stream_absorb<<<unsigned(g), kThreads, 0, stream>>>(states, msgs, offsets, lens, n, dev.d_status);
    return cuda_status(cudaGetLastError());
}

int launch_stream_final(uint8_t *states, const uint32_t *out_lens, uint8_t *digests, uint64_t n,
                        cudaStream_t stream, const DeviceInfo &dev) {
    const uint64_t ntiles = digest_offsets_tiles(n);
    int err = KB_OK;
    uint64_t *out_off = static_cast<uint64_t *>(stream_scratch(stream, size_t(8 * (n + ntiles)), &err));
    if (!out_off) return err;
    if ((err = launch_digest_offsets(out_lens, n, out_off, out_off + n, stream)) != KB_OK) return err;
    const uint64_t g = grid_for(reinterpret_cast<const void *>(&k_stream_final), n, dev);
    k_stream_final<<<unsigned(g), kThreads, 0, stream>>>(states, out_lens, out_off, digests, n, dev.d_status);
    return cuda_status(cudaGetLastError());
}

}  // namespace kb
