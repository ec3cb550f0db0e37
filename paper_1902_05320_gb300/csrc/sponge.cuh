// sponge.cuh -- absorb / pad / squeeze of the Keccak[c] sponge (Section 3.2,
// Eq. 11-18) on a register state of keccak_core.cuh, generic over the state
// representation (PlainRep or InterleavedRep).
//
// Byte form of the padding: for a message of len bytes and rate r bytes, the
// last block holds the len mod r remaining bytes, then the domain byte (the
// suffix bits plus the first "1" of pad10*1, LSB-first: 0x06 for SHA3, 0x1F
// for SHAKE) at position len mod r, zeros, and 0x80 (the final "1") XORed
// into byte r-1.  When len mod r = r-1 both land in one byte (0x86 / 0x9F).
//
// Memory access rule: a message is read only through naturally aligned 4- or
// 8-byte words that contain at least one of its bytes, so no access can leave
// the page (or allocation granule) that holds the message.
#pragma once

#include <cstdint>

#include "../../include/sha3gb.h"
#include "keccak_core.cuh"

namespace kb {

// Little-endian 64-bit word of 8 valid bytes at an 8-byte aligned address.
__device__ __forceinline__ void ld_word_a8(const uint8_t *p, uint32_t &lo, uint32_t &hi) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
    lo = v.x;
    hi = v.y;
}

// Bytes [p, p + nvalid) as a little-endian 64-bit word, 1 <= nvalid <= 8, any
// alignment; bytes past nvalid read as zero.  Loads only the aligned 32-bit
// words that hold a valid byte.
__device__ __forceinline__ void ld_word_any(const uint8_t *p, uint32_t nvalid, uint32_t &lo, uint32_t &hi) {
    const uintptr_t start = reinterpret_cast<uintptr_t>(p);
    const uint32_t *a = reinterpret_cast<const uint32_t *>(start & ~uintptr_t(3));
    const uint32_t sh = uint32_t(start & 3) * 8;
    const uintptr_t last = start + nvalid - 1;
    const uint32_t nw = uint32_t(((last & ~uintptr_t(3)) - (start & ~uintptr_t(3))) >> 2) + 1;
    const uint32_t w0 = __ldg(a);
    const uint32_t w1 = nw > 1 ? __ldg(a + 1) : 0u;
    const uint32_t w2 = nw > 2 ? __ldg(a + 2) : 0u;
    lo = __funnelshift_r(w0, w1, sh);
    hi = __funnelshift_r(w1, w2, sh);
    if (nvalid < 8) {
        const uint64_t mask = (uint64_t(1) << (8 * nvalid)) - 1;
        lo &= uint32_t(mask);
        hi &= uint32_t(mask >> 32);
    }
}

// Absorbs one full block of RATE bytes at p (p 8-byte aligned when A8).
template <int RATE, bool A8, class Rep>
__device__ __forceinline__ void absorb_full(uint32_t (&A)[25], uint32_t (&B)[25], const uint8_t *p) {
    if constexpr (A8) {
#pragma unroll
        for (int k = 0; k < RATE / 8; ++k) {
            uint32_t lo, hi;
            ld_word_a8(p + 8 * k, lo, hi);
            Rep::xor_word(A[k], B[k], lo, hi);
        }
    } else {
        // RATE/4 aligned words cover the block; one more when p is unaligned.
        const uintptr_t start = reinterpret_cast<uintptr_t>(p);
        const uint32_t *a = reinterpret_cast<const uint32_t *>(start & ~uintptr_t(3));
        const uint32_t sh = uint32_t(start & 3) * 8;
        uint32_t prev = __ldg(a);
#pragma unroll
        for (int k = 0; k < RATE / 8; ++k) {
            const uint32_t w1 = __ldg(a + 2 * k + 1);
            const uint32_t w2 = (2 * k + 2 < RATE / 4 || sh != 0) ? __ldg(a + 2 * k + 2) : 0u;
            const uint32_t lo = __funnelshift_r(prev, w1, sh);
            const uint32_t hi = __funnelshift_r(w1, w2, sh);
            prev = w2;
            Rep::xor_word(A[k], B[k], lo, hi);
        }
    }
}

// Writes bytes [0, nbytes) of the rate part of the state to dst
// (nbytes <= RATE), with the widest stores dst's alignment allows.
template <int RATE, class Rep>
__device__ __forceinline__ void squeeze(const uint32_t (&A)[25], const uint32_t (&B)[25], uint8_t *dst,
                                        uint32_t nbytes) {
    const uintptr_t d = reinterpret_cast<uintptr_t>(dst);
    if ((d & 15) == 0 && (nbytes & 15) == 0) {
#pragma unroll
        for (int k = 0; k + 1 < RATE / 8; k += 2) {
            if (uint32_t(8 * k) < nbytes) {
                uint4 v;
                Rep::get_word(A[k], B[k], v.x, v.y);
                Rep::get_word(A[k + 1], B[k + 1], v.z, v.w);
                *reinterpret_cast<uint4 *>(dst + 8 * k) = v;
            }
        }
    } else if ((d & 7) == 0 && (nbytes & 7) == 0) {
#pragma unroll
        for (int k = 0; k < RATE / 8; ++k) {
            if (uint32_t(8 * k) < nbytes) {
                uint2 v;
                Rep::get_word(A[k], B[k], v.x, v.y);
                *reinterpret_cast<uint2 *>(dst + 8 * k) = v;
            }
        }
    } else if ((d & 3) == 0 && (nbytes & 3) == 0) {
#pragma unroll
        for (int k = 0; k < RATE / 8; ++k) {
            if (uint32_t(8 * k) < nbytes) {
                uint32_t lo, hi;
                Rep::get_word(A[k], B[k], lo, hi);
                *reinterpret_cast<uint32_t *>(dst + 8 * k) = lo;
                if (uint32_t(8 * k + 4) < nbytes) *reinterpret_cast<uint32_t *>(dst + 8 * k + 4) = hi;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < RATE / 8; ++k) {
            if (uint32_t(8 * k) < nbytes) {
                uint32_t lo, hi;
                Rep::get_word(A[k], B[k], lo, hi);
                const uint64_t w = (uint64_t(hi) << 32) | lo;
                const uint32_t nb = nbytes - 8 * k < 8 ? nbytes - 8 * k : 8;
                for (uint32_t b = 0; b < nb; ++b) dst[8 * k + b] = uint8_t(w >> (8 * b));
            }
        }
    }
}

// ---- runtime-rate sponge (ragged batches: the variant varies per message) ----

__device__ __forceinline__ uint32_t rt_domain(int v) { return v < 4 ? 0x06u : 0x1Fu; }

// XORs the first nwords 64-bit words of the block at p into the state.  The
// loop runs over the largest rate (21 words, SHAKE128) with a predicate, so
// every state index stays a compile-time register.
template <bool A8, class Rep>
__device__ __forceinline__ void absorb_full_rt(uint32_t (&A)[25], uint32_t (&B)[25], const uint8_t *p, int nwords) {
    if constexpr (A8) {
#pragma unroll
        for (int k = 0; k < 21; ++k) {
            if (k < nwords) {
                uint32_t lo, hi;
                ld_word_a8(p + 8 * k, lo, hi);
                Rep::xor_word(A[k], B[k], lo, hi);
            }
        }
    } else {
        // 2*nwords aligned 32-bit words cover the block, one more when p is
        // unaligned; each 64-bit word is two funnel shifts.
        const uintptr_t start = reinterpret_cast<uintptr_t>(p);
        const uint32_t *a = reinterpret_cast<const uint32_t *>(start & ~uintptr_t(3));
        const uint32_t sh = uint32_t(start & 3) * 8;
        uint32_t prev = __ldg(a);
#pragma unroll
        for (int k = 0; k < 21; ++k) {
            if (k < nwords) {
                const uint32_t w1 = __ldg(a + 2 * k + 1);
                const uint32_t w2 = (2 * k + 2 < 2 * nwords || sh != 0) ? __ldg(a + 2 * k + 2) : 0u;
                const uint32_t lo = __funnelshift_r(prev, w1, sh);
                const uint32_t hi = __funnelshift_r(w1, w2, sh);
                prev = w2;
                Rep::xor_word(A[k], B[k], lo, hi);
            }
        }
    }
}

// Absorbs the final, padded block for a runtime rate of nwords 64-bit words:
// rem (0 <= rem < 8*nwords) message bytes at p, the domain byte at rem and
// 0x80 XORed into byte 8*nwords-1.  The block is read as the aligned 32-bit
// words that hold at least one message byte, funnel-shifted into place; the
// bytes of the last such word that lie past the message are masked off.
template <bool A8, class Rep>
__device__ __forceinline__ void absorb_last_rt(uint32_t (&A)[25], uint32_t (&B)[25], const uint8_t *p, uint32_t rem,
                                               int nwords, uint32_t domain) {
    const uintptr_t start = reinterpret_cast<uintptr_t>(p);
    const uint32_t *a = reinterpret_cast<const uint32_t *>(A8 ? start : start & ~uintptr_t(3));
    const uint32_t sh = A8 ? 0u : uint32_t(start & 3) * 8;
    // Aligned words 0 .. nw-1 overlap the rem message bytes.
    const uint32_t nw = rem ? uint32_t(((start + rem - 1) >> 2) - (start >> 2)) + 1 : 0u;
    int rb = int(8 * rem);  // message bits still to come, from the current 64-bit word on
    uint32_t prev = nw ? __ldg(a) : 0u;
#pragma unroll
    for (int k = 0; k < 21; ++k) {
        if (k < nwords) {
            const uint32_t w1 = uint32_t(2 * k + 1) < nw ? __ldg(a + 2 * k + 1) : 0u;
            const uint32_t w2 = uint32_t(2 * k + 2) < nw ? __ldg(a + 2 * k + 2) : 0u;
            uint32_t lo = __funnelshift_r(prev, w1, sh);
            uint32_t hi = __funnelshift_r(w1, w2, sh);
            prev = w2;
            // Keep max(rb, 0) low bits (clamped to 32 per half); the domain
            // byte goes right after the message's last bit.
            lo &= __funnelshift_lc(0xFFFFFFFFu, 0u, uint32_t(max(rb, 0)));
            hi &= __funnelshift_lc(0xFFFFFFFFu, 0u, uint32_t(max(rb - 32, 0)));
            if (uint32_t(rb) < 32u) lo ^= domain << rb;
            else if (uint32_t(rb - 32) < 32u) hi ^= domain << (rb - 32);
            if (k == nwords - 1) hi ^= 0x80000000u;
            rb -= 64;
            Rep::xor_word(A[k], B[k], lo, hi);
        }
    }
}

// The final block for a compile-time rate and domain byte (one instance of
// the runtime-rate form above, with its word loop bounds folded).
template <int RATE, int DOMAIN, bool A8, class Rep>
__device__ __forceinline__ void absorb_last(uint32_t (&A)[25], uint32_t (&B)[25], const uint8_t *p, uint32_t rem) {
    absorb_last_rt<A8, Rep>(A, B, p, rem, RATE / 8, uint32_t(DOMAIN));
}

// One complete sponge for a message of len bytes at p, writing dlen output
// bytes to dst.  The permutation has a single call site, so its code appears
// once.
template <int RATE, int DOMAIN, bool A8, class Rep>
__device__ __forceinline__ void sponge(const uint8_t *p, uint64_t len, uint8_t *dst, uint32_t dlen) {
    uint32_t A[25], B[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) A[i] = B[i] = 0;
    const uint64_t nfull = len / RATE;
    const uint32_t rem = uint32_t(len - nfull * RATE);
    const uint32_t nsq = dlen > uint32_t(RATE) ? (dlen - 1) / RATE : 0;  // extra squeeze permutations
    const uint64_t total = nfull + 1 + nsq;
    for (uint64_t i = 0; i < total; ++i) {
        if (i < nfull) absorb_full<RATE, A8, Rep>(A, B, p + i * RATE);
        else if (i == nfull) absorb_last<RATE, DOMAIN, A8, Rep>(A, B, p + nfull * RATE, rem);
        else squeeze<RATE, Rep>(A, B, dst + (i - nfull - 1) * RATE, RATE);
        Rep::template permute<false>(A, B);
    }
    squeeze<RATE, Rep>(A, B, dst + uint64_t(nsq) * RATE, dlen - nsq * RATE);
}

// Writes bytes [0, nbytes) of the rate part of the state (0 < nbytes <= 168)
// to dst at any alignment.  Output byte b lands in the aligned 32-bit word
// (b + o) / 4, o = dst mod 4, so aligned word j is a funnel shift of state
// words j-1 and j.  Words wholly inside the output take one 32-bit store;
// the partial words at either end are written byte by byte, so no byte
// outside [dst, dst + nbytes) is touched.
template <class Rep>
__device__ __forceinline__ void squeeze_rt(const uint32_t (&A)[25], const uint32_t (&B)[25], uint8_t *dst,
                                           uint32_t nbytes) {
    const uintptr_t d = reinterpret_cast<uintptr_t>(dst);
    const uint32_t o = uint32_t(d & 3);
    uint32_t *al = reinterpret_cast<uint32_t *>(d & ~uintptr_t(3));
    const uint32_t sh = 8 * o;
    const uint32_t end = nbytes + o;    // output end, in bytes from al
    const uint32_t jl = (end - 1) >> 2;  // last aligned word touched
    const uint32_t jfull_lo = o ? 1u : 0u;
    const uint32_t jfull_hi = (end & 3) ? jl : jl + 1;  // full words: [jfull_lo, jfull_hi)
    uint32_t prev = 0, first = 0, last = 0;
#pragma unroll
    for (int j = 0; j <= 42; ++j) {
        if (uint32_t(j) > jl) break;
        uint32_t s = 0;
        if (j < 42) {
            uint32_t lo, hi;
            Rep::get_word(A[j / 2], B[j / 2], lo, hi);
            s = (j & 1) ? hi : lo;
        }
        const uint32_t v = __funnelshift_l(prev, s, sh);
        prev = s;
        if (uint32_t(j) >= jfull_lo && uint32_t(j) < jfull_hi) al[j] = v;
        if (j == 0) first = v;
        if (uint32_t(j) == jl) last = v;
    }
    uint8_t *b = reinterpret_cast<uint8_t *>(al);
    if (o) {  // head: bytes o .. min(4, end) - 1 of word 0
        const uint32_t hend = end < 4 ? end : 4u;
        for (uint32_t i = o; i < hend; ++i) b[i] = uint8_t(first >> (8 * i));
    }
    if ((end & 3) && !(jl == 0 && o)) {  // tail: bytes 0 .. (end & 3) - 1 of word jl
        for (uint32_t i = 0; i < (end & 3); ++i) b[4 * jl + i] = uint8_t(last >> (8 * i));
    }
}

template <bool A8, class Rep>
__device__ __forceinline__ void sponge_rt(const uint8_t *p, uint64_t len, int variant, uint8_t *dst, uint32_t dlen) {
    const int rate = variant_rate(variant);
    const int nwords = rate / 8;
    const uint32_t domain = rt_domain(variant);
    uint32_t A[25], B[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) A[i] = B[i] = 0;
    const uint64_t nfull = len / uint64_t(rate);
    const uint32_t rem = uint32_t(len - nfull * uint64_t(rate));
    const uint32_t nsq = dlen > uint32_t(rate) ? (dlen - 1) / uint32_t(rate) : 0;
    const uint64_t total = nfull + 1 + nsq;
    for (uint64_t i = 0; i < total; ++i) {
        if (i < nfull) absorb_full_rt<A8, Rep>(A, B, p + i * rate, nwords);
        else if (i == nfull) absorb_last_rt<A8, Rep>(A, B, p + nfull * rate, rem, nwords, domain);
        else squeeze_rt<Rep>(A, B, dst + (i - nfull - 1) * rate, uint32_t(rate));
        Rep::template permute<false>(A, B);
    }
    if (dlen > nsq * uint32_t(rate)) squeeze_rt<Rep>(A, B, dst + uint64_t(nsq) * rate, dlen - nsq * uint32_t(rate));
}

// One message of a ragged batch: checks its descriptor, then hashes it.
// Bad descriptors set a bit in *status and leave the output untouched.
__device__ __forceinline__ void hash_ragged_message(const uint8_t *msgs, const uint64_t *offsets,
                                                    const uint64_t *lens, const uint8_t *variants,
                                                    const uint32_t *out_lens, const uint64_t *out_off,
                                                    uint8_t *digests, uint64_t i, unsigned int *status) {
    const int v = variants[i];
    const uint32_t dlen = out_lens[i];
    if (v > 5) {
        atomicOr(status, KB_DEV_BAD_VARIANT);
        return;
    }
    if (v < 4 && dlen != uint32_t(variant_digest(v))) {
        atomicOr(status, KB_DEV_BAD_OUTLEN);
        return;
    }
    sponge_rt<false, PlainRep>(msgs + offsets[i], lens[i], v, digests + out_off[i], dlen);
}

}  // namespace kb
