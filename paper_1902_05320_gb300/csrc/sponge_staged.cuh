// sponge_staged.cuh -- the runtime-rate sponge of a ragged batch with each
// thread's next message block fetched into shared memory while the current
// permutation runs (Section 4.3's plaintext allocation, done per thread and
// asynchronously).
//
// Without staging, a thread that finishes a permutation loads its next block
// word by word and waits for DRAM before it can absorb it; with few warps per
// SM sub-partition (the queue kernel runs long chains of permutations, which
// progress fastest when few warps share the ALU pipe) nothing hides that wait.
// Here the block after the one being absorbed is requested with cp.async
// (4-byte copies of the aligned 32-bit words that hold its bytes, the same
// words the direct loads read, so no access leaves the message's page) before
// the permutation, and has arrived by the time the permutation ends.
//
// Shared-memory layout per block of kThreads threads: two buffers per thread
// of kStageWords words, word-major ([buffer][word][thread]), so a warp reading
// word k of its 32 threads' buffers touches 32 consecutive banks.  A buffer is
// refilled one permutation after it was read, and that permutation consumed
// the words read from it, so a copy never overwrites words not yet read.
#pragma once

#include <cstdint>

#include "keccak_core.cuh"
#include "sponge.cuh"

namespace kb {

// Aligned 32-bit words that can hold one block: 168 bytes (SHAKE128's rate)
// starting at any byte offset cover at most 43 of them.
constexpr int kStageWords = 43;
// Bytes of shared memory a block of `threads` threads needs for its stages.
constexpr int stage_bytes(int threads) { return 2 * kStageWords * threads * 4; }

__device__ __forceinline__ void cp_async4(uint32_t saddr, const void *gaddr) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(gaddr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One thread's two stage buffers.  `s` is the shared-state address and `g`
// the generic pointer of word 0 of buffer 0; word k of buffer b sits
// (b * kStageWords + k) * kThreads words further.
struct Stage {
    uint32_t s;
    const uint32_t *g;
};

__device__ __forceinline__ Stage make_stage(uint32_t *smem) {
    Stage st;
    st.g = smem + threadIdx.x;
    st.s = static_cast<uint32_t>(__cvta_generic_to_shared(st.g));
    return st;
}

constexpr uint32_t kStageStride = 4u * 128u;  // bytes between consecutive words of one thread (kThreads = 128)

// Requests the nw aligned 32-bit words starting at a (nw <= kStageWords) into
// buffer b; commits them as one group.
__device__ __forceinline__ void stage_words(const Stage &st, int b, const uint32_t *a, uint32_t nw) {
    const uint32_t base = st.s + uint32_t(b) * kStageWords * kStageStride;
#pragma unroll
    for (int k = 0; k < kStageWords; ++k)
        if (uint32_t(k) < nw) cp_async4(base + uint32_t(k) * kStageStride, a + k);
    cp_async_commit();
}

// The aligned words that hold the rem bytes at p (none when rem = 0).
__device__ __forceinline__ uint32_t last_block_words(const uint8_t *p, uint32_t rem) {
    const uintptr_t start = reinterpret_cast<uintptr_t>(p);
    return rem ? uint32_t(((start + rem - 1) >> 2) - (start >> 2)) + 1 : 0u;
}

__device__ __forceinline__ void stage_last(const Stage &st, int b, const uint8_t *p, uint32_t rem) {
    const uintptr_t start = reinterpret_cast<uintptr_t>(p);
    stage_words(st, b, reinterpret_cast<const uint32_t *>(start & ~uintptr_t(3)), last_block_words(p, rem));
}

// Runtime-rate full block: 2*nwords words (+1 when unaligned).
__device__ __forceinline__ void stage_full_rt(const Stage &st, int b, const uint8_t *p, int nwords) {
    const uintptr_t start = reinterpret_cast<uintptr_t>(p);
    stage_words(st, b, reinterpret_cast<const uint32_t *>(start & ~uintptr_t(3)),
                uint32_t(2 * nwords) + ((start & 3) ? 1u : 0u));
}

// XORs a staged full block into the state: nwords 64-bit words, sh = 8 *
// (p mod 4); a staged word the block does not reach is shifted out (sh = 0).
// Predicated over the largest rate so every state index is a register.
template <class Rep>
__device__ __forceinline__ void absorb_staged_full_rt(uint32_t (&A)[25], uint32_t (&B)[25], const uint32_t *w,
                                                      uint32_t sh, int nwords) {
    uint32_t prev = w[0];
#pragma unroll
    for (int k = 0; k < 21; ++k) {
        if (k < nwords) {
            const uint32_t w1 = w[(2 * k + 1) * 128];
            const uint32_t w2 = w[(2 * k + 2) * 128];
            const uint32_t lo = __funnelshift_r(prev, w1, sh);
            const uint32_t hi = __funnelshift_r(w1, w2, sh);
            prev = w2;
            Rep::xor_word(A[k], B[k], lo, hi);
        }
    }
}

// The staged final block: rem message bytes (nw aligned words staged), the
// domain byte at rem, 0x80 into byte 8*nwords-1 (as absorb_last_rt).
template <class Rep>
__device__ __forceinline__ void absorb_staged_last(uint32_t (&A)[25], uint32_t (&B)[25], const uint32_t *w,
                                                   uint32_t sh, uint32_t rem, uint32_t nw, int nwords,
                                                   uint32_t domain) {
    int rb = int(8 * rem);
    uint32_t prev = nw ? w[0] : 0u;
#pragma unroll
    for (int k = 0; k < 21; ++k) {
        if (k < nwords) {
            const uint32_t w1 = uint32_t(2 * k + 1) < nw ? w[(2 * k + 1) * 128] : 0u;
            const uint32_t w2 = uint32_t(2 * k + 2) < nw ? w[(2 * k + 2) * 128] : 0u;
            uint32_t lo = __funnelshift_r(prev, w1, sh);
            uint32_t hi = __funnelshift_r(w1, w2, sh);
            prev = w2;
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

// Keccak-f[1600] with all 24 rounds in a loop of four (constants from the
// __constant__ table): half the code of the form with an unrolled tail,
// for kernels whose instruction footprint matters more than the immediates.
__device__ __forceinline__ void keccak_f1600_looped(uint32_t (&L)[25], uint32_t (&H)[25]) {
#pragma unroll 1
    for (int r = 0; r < 24; r += 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j) plain_round_rt(L, H, r + j);
    }
}

template <bool LOOPED>
__device__ __forceinline__ void permute_plain(uint32_t (&A)[25], uint32_t (&B)[25]) {
    if constexpr (LOOPED) keccak_f1600_looped(A, B);
    else keccak_f1600_plain<false>(A, B);
}

// One whole sponge of a message of len bytes at p with variant `variant`
// (valid), dlen output bytes to dst, the next block staged in shared memory.
// The permutation has one call site.
template <bool LOOPED>
__device__ __forceinline__ void sponge_rt_staged(const Stage &st, const uint8_t *p, uint64_t len, int variant,
                                                 uint8_t *dst, uint32_t dlen) {
    using Rep = PlainRep;
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
    const uint8_t *last = p + nfull * uint64_t(rate);
    const uint32_t sh = uint32_t(reinterpret_cast<uintptr_t>(p) & 3) * 8;  // same for every block when rate % 4 == 0
    const uint32_t nw_last = last_block_words(last, rem);
    // Block 0 into buffer 0.
    if (nfull) {
        stage_full_rt(st, 0, p, nwords);
    } else {
        stage_last(st, 0, last, rem);
    }
    for (uint64_t i = 0; i < total; ++i) {
        if (i <= nfull) {
            const int b = int(i & 1);
            cp_async_wait_all();
            const uint32_t *w = st.g + b * kStageWords * 128;
            if (i < nfull) {
                absorb_staged_full_rt<Rep>(A, B, w, sh, nwords);
                // The next block goes into the other buffer while this permutation runs.
                if (i + 1 < nfull) {
                    stage_full_rt(st, b ^ 1, p + (i + 1) * uint64_t(rate), nwords);
                } else {
                    stage_last(st, b ^ 1, last, rem);
                }
            } else {
                absorb_staged_last<Rep>(A, B, w, sh, rem, nw_last, nwords, domain);
            }
        } else {
            squeeze_rt<Rep>(A, B, dst + (i - nfull - 1) * uint64_t(rate), uint32_t(rate));
        }
        permute_plain<LOOPED>(A, B);
    }
    if (dlen > nsq * uint32_t(rate)) squeeze_rt<Rep>(A, B, dst + uint64_t(nsq) * rate, dlen - nsq * uint32_t(rate));
}

// sponge_rt (direct loads) with the permutation form chosen by LOOPED.
template <bool LOOPED>
__device__ __forceinline__ void sponge_rt_direct(const uint8_t *p, uint64_t len, int variant, uint8_t *dst,
                                                 uint32_t dlen) {
    using Rep = PlainRep;
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
        if (i < nfull) absorb_full_rt<false, Rep>(A, B, p + i * rate, nwords);
        else if (i == nfull) absorb_last_rt<false, Rep>(A, B, p + nfull * rate, rem, nwords, domain);
        else squeeze_rt<Rep>(A, B, dst + (i - nfull - 1) * rate, uint32_t(rate));
        permute_plain<LOOPED>(A, B);
    }
    if (dlen > nsq * uint32_t(rate)) squeeze_rt<Rep>(A, B, dst + uint64_t(nsq) * rate, dlen - nsq * uint32_t(rate));
}

// The next full block's aligned words into w[0 .. 2*nwords] (the last one only
// when p is unaligned, i.e. when it holds bytes of the block).  The rates'
// word counts are 9, 13, 17, 18 and 21, so the loads are cut into segments
// at those counts and each segment is skipped by a branch; in a warp of one
// rate the branches do not diverge, and no predicated-off work is issued.
__device__ __forceinline__ void fetch_full_seg(uint32_t (&w)[kStageWords], const uint8_t *q, int nwords, bool un) {
    const uint32_t *a = reinterpret_cast<const uint32_t *>(reinterpret_cast<uintptr_t>(q) & ~uintptr_t(3));
#pragma unroll
    for (int k = 0; k < 18; ++k) w[k] = __ldg(a + k);
    if (nwords > 9 || un) w[18] = __ldg(a + 18);
    if (nwords > 9) {
#pragma unroll
        for (int k = 19; k < 26; ++k) w[k] = __ldg(a + k);
        if (nwords > 13 || un) w[26] = __ldg(a + 26);
        if (nwords > 13) {
#pragma unroll
            for (int k = 27; k < 34; ++k) w[k] = __ldg(a + k);
            if (nwords > 17 || un) w[34] = __ldg(a + 34);
            if (nwords > 17) {
                w[35] = __ldg(a + 35);
                if (nwords > 18 || un) w[36] = __ldg(a + 36);
                if (nwords > 18) {
#pragma unroll
                    for (int k = 37; k < 42; ++k) w[k] = __ldg(a + k);
                    if (un) w[42] = __ldg(a + 42);
                }
            }
        }
    }
}

// XORs 64-bit words [K0, K1) of a fetched block into the state.
template <int K0, int K1, class Rep>
__device__ __forceinline__ void absorb_words(uint32_t (&A)[25], uint32_t (&B)[25], const uint32_t (&w)[kStageWords],
                                             uint32_t sh) {
#pragma unroll
    for (int k = K0; k < K1; ++k) {
        const uint32_t lo = __funnelshift_r(w[2 * k], w[2 * k + 1], sh);
        const uint32_t hi = __funnelshift_r(w[2 * k + 1], w[2 * k + 2], sh);
        Rep::xor_word(A[k], B[k], lo, hi);
    }
}

// A fetched full block into the state, in the same segments.
template <class Rep>
__device__ __forceinline__ void absorb_full_seg(uint32_t (&A)[25], uint32_t (&B)[25], const uint32_t (&w)[kStageWords],
                                                uint32_t sh, int nwords) {
    absorb_words<0, 9, Rep>(A, B, w, sh);
    if (nwords > 9) {
        absorb_words<9, 13, Rep>(A, B, w, sh);
        if (nwords > 13) {
            absorb_words<13, 17, Rep>(A, B, w, sh);
            if (nwords > 17) {
                absorb_words<17, 18, Rep>(A, B, w, sh);
                if (nwords > 18) absorb_words<18, 21, Rep>(A, B, w, sh);
            }
        }
    }
}

// The runtime-rate sponge with the next block's aligned words loaded into
// registers before the permutation (plain loads, consumed after it): the
// load latency is hidden as with the shared-memory stage, without its copies
// and reads, at 43 more registers live across the permutation.  Full blocks
// use the segmented fetch and absorb above; the final block (once per
// message) the predicated form.
template <bool LOOPED>
__device__ __forceinline__ void sponge_rt_prefetch(const uint8_t *p, uint64_t len, int variant, uint8_t *dst,
                                                   uint32_t dlen) {
    using Rep = PlainRep;
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
    const uint8_t *last = p + nfull * uint64_t(rate);
    const uint32_t sh = uint32_t(reinterpret_cast<uintptr_t>(p) & 3) * 8;  // the same for every block (rate % 4 == 0)
    const bool un = sh != 0;
    const uint32_t nw_last = last_block_words(last, rem);
    uint32_t w[kStageWords];
#pragma unroll
    for (int k = 0; k < kStageWords; ++k) w[k] = 0;
    // The final block: its nw_last words, the rest zero.
    auto fetch_last = [&] {
        const uint32_t *a = reinterpret_cast<const uint32_t *>(reinterpret_cast<uintptr_t>(last) & ~uintptr_t(3));
#pragma unroll
        for (int k = 0; k < kStageWords; ++k) w[k] = uint32_t(k) < nw_last ? __ldg(a + k) : 0u;
    };
    if (nfull) fetch_full_seg(w, p, nwords, un);
    else fetch_last();
    for (uint64_t i = 0; i < total; ++i) {
        if (i <= nfull) {
            if (i < nfull) {
                absorb_full_seg<Rep>(A, B, w, sh, nwords);
                // The next block's words are requested before the permutation.
                if (i + 1 < nfull) fetch_full_seg(w, p + (i + 1) * uint64_t(rate), nwords, un);
                else fetch_last();
            } else {
                int rb = int(8 * rem);
                uint32_t prev = w[0];
#pragma unroll
                for (int k = 0; k < 21; ++k) {
                    if (k < nwords) {
                        uint32_t lo = __funnelshift_r(prev, w[2 * k + 1], sh);
                        uint32_t hi = __funnelshift_r(w[2 * k + 1], w[2 * k + 2], sh);
                        prev = w[2 * k + 2];
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
        } else {
            squeeze_rt<Rep>(A, B, dst + (i - nfull - 1) * uint64_t(rate), uint32_t(rate));
        }
        permute_plain<LOOPED>(A, B);
    }
    if (dlen > nsq * uint32_t(rate)) squeeze_rt<Rep>(A, B, dst + uint64_t(nsq) * rate, dlen - nsq * uint32_t(rate));
}

}  // namespace kb
