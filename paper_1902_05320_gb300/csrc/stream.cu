// stream.cu -- incremental (streaming) hashing of many messages at once: each
// message has a sponge state in device memory that absorbs pieces of any
// length across calls and is finalised into its digest.  The state is the
// sponge of Section 3.2 paused between absorbed bytes: the 25 lanes, with
// the bytes of a block not yet complete already XORed into them, and the
// count of those bytes.
//
// One kernel template does every step: a call may start from fresh states
// (INIT: the first piece is absorbed in the same launch as the
// initialisation) and may end with the padding and squeeze (FINAL: the last
// piece is absorbed in the same launch), so a message fed in k pieces takes k
// launches.  A piece is XORed into the lanes where it lands: its head tops up
// the open block at byte offset `pending`, whole blocks follow with the next
// block's words loaded into registers during the permutation (cut into rate
// segments, as in the ragged queue), and its tail opens the next block.  No
// byte is copied to or from a buffer, and one loop around a single call site
// of the (looped) permutation covers the completed block, the whole blocks,
// the padded block and the squeeze blocks.
//
// State layout (KB_STATE_BYTES = 384 bytes per message, 8-byte aligned):
//   [0, 200)    25 lanes, little-endian 64-bit words (lane x + 5y), with the
//               pending bytes of the open block XORed in
//   200         u32 number of pending bytes (bytes of the open block, < rate)
//   204         u8 variant
//   205         u8 1 after the final step (further absorbs are refused)
//   208         u64 total bytes absorbed
//   [216, 384)  reserved
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
constexpr uint32_t kNbufOff = 200, kVarOff = 204, kDoneOff = 205, kTotalOff = 208, kUsedBytes = 216;
static_assert(kUsedBytes <= kStateBytes, "state fields exceed KB_STATE_BYTES");

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

// Bits [0, min(x, 32)) set; none for x <= 0.
__device__ __forceinline__ uint32_t low_bits(int x) { return __funnelshift_lc(0xFFFFFFFFu, 0u, uint32_t(max(x, 0))); }

// XORs the n bytes at p (n >= 1, off + n <= 8 * nwords) into state bytes
// [off, off + n): state byte s takes piece byte s - off.  State 32-bit word j
// is the funnel shift of the aligned words at (p - off) + 4j and + 4j + 4, of
// which only those holding a byte of the piece are loaded (the others read
// as zero), and the bits outside [8 off, 8 (off + n)) are masked off.  So the
// piece is read only through aligned 32-bit words that hold one of its
// bytes.  Predicated over the largest rate, so every state index is a
// register.
__device__ __forceinline__ void xor_bytes_at(uint32_t (&A)[25], uint32_t (&B)[25], const uint8_t *p, uint32_t n,
                                             uint32_t off, int nwords) {
    const uintptr_t pa = reinterpret_cast<uintptr_t>(p);
    const uintptr_t q = pa - off;  // where state byte 0 would sit
    const uintptr_t qa = q & ~uintptr_t(3);
    const uint32_t sh = uint32_t(q & 3) * 8;
    const uint32_t t0 = uint32_t(((pa & ~uintptr_t(3)) - qa) >> 2);            // first word holding a piece byte
    const uint32_t t1 = uint32_t((((pa + n - 1) & ~uintptr_t(3)) - qa) >> 2);  // last one
    auto word = [&](uint32_t t) -> uint32_t {
        return (t >= t0 && t <= t1) ? __ldg(reinterpret_cast<const uint32_t *>(qa + 4 * uintptr_t(t))) : 0u;
    };
    const int b0 = int(8 * off), b1 = int(8 * (off + n));
    uint32_t prev = word(0);
#pragma unroll
    for (int k = 0; k < 21; ++k) {
        if (k < nwords) {
            const uint32_t w1 = word(uint32_t(2 * k + 1));
            const uint32_t w2 = word(uint32_t(2 * k + 2));
            uint32_t lo = __funnelshift_r(prev, w1, sh);
            uint32_t hi = __funnelshift_r(w1, w2, sh);
            prev = w2;
            lo &= low_bits(b1 - 64 * k) & ~low_bits(b0 - 64 * k);
            hi &= low_bits(b1 - 64 * k - 32) & ~low_bits(b0 - 64 * k - 32);
            PlainRep::xor_word(A[k], B[k], lo, hi);
        }
    }
}

// The padding of the open block: the domain byte (suffix bits and the first
// 1 of pad10*1) at byte `pending`, and 0x80 (the last 1) into byte rate - 1.
__device__ __forceinline__ void pad_open_block(uint32_t (&A)[25], uint32_t (&B)[25], uint32_t pending, int nwords,
                                               uint32_t domain) {
    int rb = int(8 * pending);
#pragma unroll
    for (int k = 0; k < 21; ++k) {
        if (k < nwords) {
            uint32_t lo = 0, hi = 0;
            if (uint32_t(rb) < 32u) lo = domain << rb;
            else if (uint32_t(rb - 32) < 32u) hi = domain << (rb - 32);
            if (k == nwords - 1) hi ^= 0x80000000u;
            rb -= 64;
            PlainRep::xor_word(A[k], B[k], lo, hi);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_stream_init(uint8_t *states, const uint8_t *variants, uint64_t n,
                                                          unsigned int *status) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
        uint8_t *st = states + i * kStateBytes;
        uint2 *w = reinterpret_cast<uint2 *>(st);
        for (uint32_t k = 0; k < kUsedBytes / 8; ++k) w[k] = make_uint2(0, 0);
        const uint8_t v = variants[i];
        st[kVarOff] = v;
        if (v > 5) atomicOr(status, KB_DEV_BAD_VARIANT);
    }
}

// One step of message i: absorbs its piece (msgs + offsets[i], lens[i]
// bytes) into the lanes: the head completes the open block, whole blocks
// follow, the tail opens the next block.
// INIT: the state starts empty for variants[i] (nothing is read from it).
// FINAL: the open block is then padded and the state permuted and squeezed
// into out_lens[i] bytes at digests + out_off[i], and marked finalised.
template <bool INIT, bool FINAL>
__global__ void __launch_bounds__(kThreads, 3)
    k_stream_step(uint8_t *states, const uint8_t *__restrict__ init_variants, const uint8_t *__restrict__ msgs,
                  const uint64_t *__restrict__ offsets, const uint64_t *__restrict__ lens,
                  const uint32_t *__restrict__ out_lens, const uint64_t *__restrict__ out_off,
                  uint8_t *__restrict__ digests, uint64_t n, unsigned int *status) {
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t *st = states + i * kStateBytes;
    uint32_t *pending_field = reinterpret_cast<uint32_t *>(st + kNbufOff);
    uint64_t *total_field = reinterpret_cast<uint64_t *>(st + kTotalOff);
    int v;
    uint32_t pending = 0;
    uint64_t total_in = 0;
    uint32_t A[25], B[25];
    if constexpr (INIT) {
        v = init_variants[i];
        st[kVarOff] = uint8_t(v);
        st[kDoneOff] = 0;
#pragma unroll
        for (int k = 0; k < 25; ++k) A[k] = B[k] = 0;
        if (v > 5) {
            atomicOr(status, KB_DEV_BAD_VARIANT);
            *pending_field = 0;
            *total_field = 0;
            store_lanes(st, A, B);
            return;
        }
    } else {
        v = st[kVarOff];
        if (v > 5 || st[kDoneOff]) {
            if (lens[i] || FINAL) atomicOr(status, v > 5 ? KB_DEV_BAD_VARIANT : KB_DEV_BAD_OUTLEN);
            return;
        }
        pending = *pending_field;
        total_in = *total_field;
        load_lanes(st, A, B);
    }
    uint32_t dlen = 0;
    if constexpr (FINAL) {
        dlen = out_lens[i];
        if (v < 4 && dlen != uint32_t(variant_digest(v))) {
            atomicOr(status, KB_DEV_BAD_OUTLEN);
            if constexpr (INIT) {
                *pending_field = 0;
                *total_field = 0;
                store_lanes(st, A, B);
            }
            return;
        }
    }
    const uint32_t rate = uint32_t(variant_rate(v));
    const int nwords = int(rate / 8);
    uint64_t len = lens[i];
    const uint8_t *p = msgs + offsets[i];
    *total_field = total_in + len;
    // Head: completes the open block as far as the piece reaches.
    if (pending && len) {
        const uint32_t take = len < rate - pending ? uint32_t(len) : rate - pending;
        xor_bytes_at(A, B, p, take, pending, nwords);
        pending += take;
        p += take;
        len -= take;
    }
    const uint32_t closed = pending == rate ? 1u : 0u;  // the open block is now complete
    if (closed) pending = 0;
    const uint64_t nblk = len / rate;
    const uint32_t tail = uint32_t(len - nblk * rate);  // > 0 only when pending == 0
    // The fields are written before the permutations, so that nothing but
    // the lanes and the block loop stays live across them.
    uint32_t pad_at = 0, domain = 0;
    if constexpr (FINAL) {
        pad_at = pending + tail;
        domain = rt_domain(v);
        st[kDoneOff] = 1;  // the lanes of a finalised state are never read again
    } else {
        *pending_field = pending + tail;
    }
    // Permutations: the completed block, the whole blocks, and for FINAL the
    // padded block.
    const uint64_t steps = closed + nblk + (FINAL ? 1 : 0);
    const uint32_t sh = uint32_t(reinterpret_cast<uintptr_t>(p) & 3) * 8;  // the same for every whole block
    const bool un = sh != 0;
    uint32_t w[kStageWords];
#pragma unroll
    for (int k = 0; k < kStageWords; ++k) w[k] = 0;
    if (nblk) fetch_full_seg(w, p, nwords, un);
    for (uint64_t s = 0; s < steps; ++s) {
        if (s >= closed) {
            const uint64_t b = s - closed;
            if (b < nblk) {
                absorb_full_seg<PlainRep>(A, B, w, sh, nwords);
                if (b + 1 < nblk) fetch_full_seg(w, p + (b + 1) * rate, nwords, un);
            } else if constexpr (FINAL) {  // b == nblk: the tail, then the padding
                if (tail) xor_bytes_at(A, B, p + nblk * rate, tail, 0, nwords);
                pad_open_block(A, B, pad_at, nwords, domain);
            }
        }
        permute_plain<true>(A, B);
    }
    if constexpr (FINAL) {
        // Squeeze: out_lens[i] bytes, one permutation between rate-sized blocks.
        const uint32_t dlen = out_lens[i];
        uint8_t *dst = digests + out_off[i];
        const uint32_t nsq = dlen > rate ? (dlen - 1) / rate : 0;
        for (uint32_t j = 0; j < nsq; ++j) {
            squeeze_rt<PlainRep>(A, B, dst + uint64_t(j) * rate, rate);
            permute_plain<true>(A, B);
        }
        if (dlen > nsq * rate) squeeze_rt<PlainRep>(A, B, dst + uint64_t(nsq) * rate, dlen - nsq * rate);
        return;
    }
    // Tail: opens the next block (pending is 0 whenever there is a tail).
    if (tail) xor_bytes_at(A, B, p + nblk * rate, tail, 0, nwords);
    if (INIT || lens[i]) store_lanes(st, A, B);
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
