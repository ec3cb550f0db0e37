// stream.cu -- incremental (streaming) hashing of many messages at once: each
// message has a sponge state in device memory that absorbs pieces of any
// length across calls and is finalised into its digest.  The state is the
// sponge of Section 3.2 paused between absorbed blocks: the 25 lanes plus the
// bytes of a block not yet complete.
//
// One kernel template does every step: a call may start from fresh states
// (INIT: the first piece is absorbed in the same launch as the
// initialisation) and may end with the padding and squeeze (FINAL: the last
// piece is absorbed in the same launch), so a message fed in k pieces takes k
// launches.  Whole blocks are absorbed straight from the piece with the next
// block's words loaded into registers during the permutation (cut into rate
// segments, as in the ragged queue), and the permutation is the looped form.
//
// State layout (KB_STATE_BYTES = 384 bytes per message, 8-byte aligned):
//   [0, 200)    25 lanes, little-endian 64-bit words (lane x + 5y)
//   [200, 368)  pending bytes of the current block (at most rate - 1)
//   368         u32 number of pending bytes
//   372         u8 variant
//   373         u8 1 after the final step (further absorbs are refused)
//   376         u64 total bytes absorbed
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "keccak_core.cuh"
#include "runtime.cuh"
#include "sponge.cuh"
#include "sponge_staged.cuh"

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

// One step of message i: absorbs its piece (msgs + offsets[i], lens[i]
// bytes), completing the pending block first, then whole blocks straight from
// the piece, then keeping the rest as pending bytes.
// INIT: the state starts empty for variants[i] (nothing is read from it).
// FINAL: the state is then padded, permuted and squeezed into out_lens[i]
// bytes at digests + out_off[i], and marked finalised.
template <bool INIT, bool FINAL>
__global__ void __launch_bounds__(kThreads, 3)
    k_stream_step(uint8_t *states, const uint8_t *__restrict__ init_variants, const uint8_t *__restrict__ msgs,
                  const uint64_t *__restrict__ offsets, const uint64_t *__restrict__ lens,
                  const uint32_t *__restrict__ out_lens, const uint64_t *__restrict__ out_off,
                  uint8_t *__restrict__ digests, uint64_t n, unsigned int *status) {
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t *st = states + i * kStateBytes;
    int v;
    uint32_t nbuf = 0;
    uint32_t A[25], B[25];
    if constexpr (INIT) {
        // Only the counters and flags need a value: pending bytes are always
        // written before they are read.
        v = init_variants[i];
        *reinterpret_cast<uint32_t *>(st + kNbufOff) = 0;
        st[kVarOff] = uint8_t(v);
        st[kDoneOff] = 0;
        *reinterpret_cast<uint64_t *>(st + kTotalOff) = 0;
#pragma unroll
        for (int k = 0; k < 25; ++k) A[k] = B[k] = 0;
        if (v > 5) {
            atomicOr(status, KB_DEV_BAD_VARIANT);
            store_lanes(st, A, B);
            return;
        }
    } else {
        v = st[kVarOff];
        if (v > 5 || st[kDoneOff]) {
            if (lens[i] || FINAL) atomicOr(status, v > 5 ? KB_DEV_BAD_VARIANT : KB_DEV_BAD_OUTLEN);
            return;
        }
        nbuf = *reinterpret_cast<const uint32_t *>(st + kNbufOff);
        load_lanes(st, A, B);
    }
    uint32_t dlen = 0;
    if constexpr (FINAL) {
        dlen = out_lens[i];
        if (v < 4 && dlen != uint32_t(variant_digest(v))) {
            atomicOr(status, KB_DEV_BAD_OUTLEN);
            if constexpr (INIT) store_lanes(st, A, B);
            return;
        }
    }
    const uint32_t rate = uint32_t(variant_rate(v));
    const int nwords = int(rate / 8);
    uint64_t len = lens[i];
    const uint8_t *p = msgs + offsets[i];
    uint8_t *buf = st + kBufOff;
    *reinterpret_cast<uint64_t *>(st + kTotalOff) += len;
    bool dirty = INIT;
    if (nbuf && len) {  // top up the pending block
        const uint32_t take = len < rate - nbuf ? uint32_t(len) : rate - nbuf;
        for (uint32_t k = 0; k < take; ++k) buf[nbuf + k] = p[k];
        nbuf += take;
        p += take;
        len -= take;
        if (nbuf == rate) {
            absorb_full_rt<true, PlainRep>(A, B, buf, nwords);
            permute_plain<true>(A, B);
            nbuf = 0;
            dirty = true;
        }
    }
    const uint64_t nblk = len / rate;
    if (nblk) {
        const uint32_t sh = uint32_t(reinterpret_cast<uintptr_t>(p) & 3) * 8;
        const bool un = sh != 0;
        uint32_t w[kStageWords];
#pragma unroll
        for (int k = 0; k < kStageWords; ++k) w[k] = 0;
        fetch_full_seg(w, p, nwords, un);
        for (uint64_t b = 0; b < nblk; ++b) {
            absorb_full_seg<PlainRep>(A, B, w, sh, nwords);
            if (b + 1 < nblk) fetch_full_seg(w, p + (b + 1) * rate, nwords, un);
            permute_plain<true>(A, B);
        }
        p += nblk * rate;
        len -= nblk * rate;
        dirty = true;
    }
    // The rest of the piece joins the pending bytes.
    for (uint32_t k = 0; k < uint32_t(len); ++k) buf[nbuf + k] = p[k];
    nbuf += uint32_t(len);
    if constexpr (FINAL) {
        absorb_last_rt<true, PlainRep>(A, B, buf, nbuf, nwords, rt_domain(v));
        permute_plain<true>(A, B);
        uint8_t *dst = digests + out_off[i];
        const uint32_t nsq = dlen > rate ? (dlen - 1) / rate : 0;
        for (uint32_t j = 0; j < nsq; ++j) {
            squeeze_rt<PlainRep>(A, B, dst + uint64_t(j) * rate, rate);
            permute_plain<true>(A, B);
        }
        if (dlen > nsq * rate) squeeze_rt<PlainRep>(A, B, dst + uint64_t(nsq) * rate, dlen - nsq * rate);
        st[kDoneOff] = 1;  // the lanes of a finalised state are never read again
        return;
    }
    *reinterpret_cast<uint32_t *>(st + kNbufOff) = nbuf;
    if (dirty) store_lanes(st, A, B);
}

// One thread per message and as many blocks as that takes (the block
// scheduler balances the last wave; a grid-stride split would give some
// threads one message more than others).
unsigned grid_for(uint64_t n) { return unsigned(std::min<uint64_t>((n + kThreads - 1) / kThreads, uint64_t(INT32_MAX))); }

}  // namespace

int launch_stream_init(uint8_t *states, const uint8_t *variants, uint64_t n, cudaStream_t stream,
                       const DeviceInfo &dev) {
    k_stream_init<<<grid_for(n), kThreads, 0, stream>>>(states, variants, n, dev.d_status);
    return cuda_status(cudaGetLastError());
}

int launch_stream_step(bool init, bool final_, uint8_t *states, const uint8_t *variants, const uint8_t *msgs,
                       const uint64_t *offsets, const uint64_t *lens, const uint32_t *out_lens, uint8_t *digests,
                       uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    uint64_t *out_off = nullptr;
    uint64_t *zeros = nullptr;
    if (final_) {
        // Digest offsets: the exclusive scan of out_lens.  A final step
        // without a piece reads a zeroed array as its offsets and lengths.
        const uint64_t ntiles = digest_offsets_tiles(n);
        int err = KB_OK;
        const uint64_t extra = msgs ? 0 : n;
        out_off = static_cast<uint64_t *>(stream_scratch(stream, size_t(8 * (n + ntiles + extra)), &err));
        if (!out_off) return err;
        if (!msgs) {
            zeros = out_off + n + ntiles;
            if (cudaMemsetAsync(zeros, 0, size_t(8 * n), stream) != cudaSuccess) return KB_ERR_CUDA;
            msgs = reinterpret_cast<const uint8_t *>(zeros);
            offsets = lens = zeros;
        }
        if ((err = launch_digest_offsets(out_lens, n, out_off, out_off + n, stream)) != KB_OK) return err;
    }
    const unsigned g = grid_for(n);
    if (init && final_) return KB_ERR_INVALID;  // one whole message per state: keccak_batch
    if (init)
        k_stream_step<true, false><<<g, kThreads, 0, stream>>>(states, variants, msgs, offsets, lens, out_lens,
                                                               out_off, digests, n, dev.d_status);
    else if (final_)
        k_stream_step<false, true><<<g, kThreads, 0, stream>>>(states, variants, msgs, offsets, lens, out_lens,
                                                               out_off, digests, n, dev.d_status);
    else
        k_stream_step<false, false><<<g, kThreads, 0, stream>>>(states, variants, msgs, offsets, lens, out_lens,
                                                                out_off, digests, n, dev.d_status);
    return cuda_status(cudaGetLastError());
}

int launch_stream_absorb(uint8_t *states, const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                         uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    return launch_stream_step(false, false, states, nullptr, msgs, offsets, lens, nullptr, nullptr, n, stream, dev);
}

int launch_stream_final(uint8_t *states, const uint32_t *out_lens, uint8_t *digests, uint64_t n,
                        cudaStream_t stream, const DeviceInfo &dev) {
    return launch_stream_step(false, true, states, nullptr, nullptr, nullptr, nullptr, out_lens, digests, n, stream,
                              dev);
}

}  // namespace kb
