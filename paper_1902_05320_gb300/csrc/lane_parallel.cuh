// lane_parallel.cuh -- one message per warp: the 25 lanes of the Keccak state
// are spread over threads 0..24 (thread t holds lane t = x + 5y as its low and
// high 32-bit words), and the round's cross-lane steps become warp shuffles.
// A sponge then advances about twice as fast as in one thread, at several
// times the instructions per permutation; it serves long messages whose
// sequential chain of permutations, not the throughput of the machine, sets
// their latency.
//
// Per round and thread (Eq. 10), 18 shuffles in three dependent stages:
//   theta: the column parity C[x] from the four other lanes of the column
//          (8 shuffles), then C[x-1] and C[x+1] from the neighbouring columns
//          (4 shuffles), rot(C[x+1], 1) and the XOR into the lane;
//   rho:   the thread's own rotation amount (a per-thread register): two
//          selects and two funnel shifts;
//   pi+chi: B[x,y], B[x+1,y] and B[x+2,y] taken straight from the threads
//          whose rotated lanes pi sends there (6 shuffles), one LOP3 per word;
//   iota:  thread 0 XORs the round constant.
// A warp issues a shuffle only every dozen cycles or so, so the round's length
// follows the shuffle count: gathering C[x-1] and C[x+1] in one stage (20
// shuffles instead of 12) measured slower, and so did exchanges through shared
// memory once several such warps share an SM.  Threads 25..31 take part in
// every shuffle and their results are ignored.  Message blocks are read as
// one 8-byte word per thread (coalesced), the next block's word while the
// permutation runs, and digests written the same way.
#pragma once

#include <cstdint>

#include "keccak_core.cuh"
#include "sponge.cuh"

namespace kb {

struct LaneCtx {
    int t;                       // lane index x + 5y (threads >= 25 idle)
    int col[4];                  // the other four threads of this column
    int left, right;             // a thread of column x-1 / x+1 (same row)
    int pi0, pi1, pi2;           // threads whose rotated lanes become B[x,y], B[x+1,y], B[x+2,y]
    uint32_t rot_swap, rot_amt;  // rho: swap halves when the offset >= 32; shift
    uint32_t is_lane0;           // all ones on thread 0, else zero
};

// Eq. 6: B[x,y] = rho(A)[(x+3y) mod 5, x], so B[x,y] is the rotated lane of
// thread ((x+3y) mod 5) + 5x.
__device__ __forceinline__ int pi_source(int x, int y) { return (x + 3 * y) % 5 + 5 * x; }

__device__ __forceinline__ LaneCtx lane_ctx() {
    LaneCtx c;
    const int t = int(threadIdx.x & 31);
    c.t = t;
    const int x = t % 5, y = (t / 5) % 5;  // idle threads map onto some lane
    for (int k = 1; k <= 4; ++k) c.col[k - 1] = x + 5 * ((y + k) % 5);
    c.left = (x + 4) % 5 + 5 * y;
    c.right = (x + 1) % 5 + 5 * y;
    c.pi0 = pi_source(x, y);
    c.pi1 = pi_source((x + 1) % 5, y);
    c.pi2 = pi_source((x + 2) % 5, y);
    const int n = rho_offset(x + 5 * y);
    c.rot_swap = n >= 32 ? 0xffffffffu : 0u;
    c.rot_amt = uint32_t(n & 31);
    c.is_lane0 = t == 0 ? 0xffffffffu : 0u;
    return c;
}

__device__ __forceinline__ uint32_t shfl(uint32_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Upper 32 bits of (hi:lo) << (s mod 32), s in a register.
__device__ __forceinline__ uint32_t funnel_l_var(uint32_t lo, uint32_t hi, uint32_t s) {
    uint32_t d;
    asm("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(lo), "r"(hi), "r"(s));
    return d;
}

__device__ __forceinline__ void lane_round(const LaneCtx &c, uint32_t &lo, uint32_t &hi, int ir) {
    // theta (Eq. 2-4)
    const uint32_t cl = xor3(xor3(lo, shfl(lo, c.col[0]), shfl(lo, c.col[1])), shfl(lo, c.col[2]), shfl(lo, c.col[3]));
    const uint32_t ch = xor3(xor3(hi, shfl(hi, c.col[0]), shfl(hi, c.col[1])), shfl(hi, c.col[2]), shfl(hi, c.col[3]));
    const uint32_t ml = shfl(cl, c.left), mh = shfl(ch, c.left);    // C[x-1]
    const uint32_t pl = shfl(cl, c.right), ph = shfl(ch, c.right);  // C[x+1]
    lo = xor3(lo, ml, funnel_l<1>(ph, pl));  // rot(C[x+1], 1), low word
    hi = xor3(hi, mh, funnel_l<1>(pl, ph));  // high word
    // rho (Eq. 5 as FIPS 202 Algorithm 2): rotate left by this lane's offset
    const uint32_t a = (lo & ~c.rot_swap) | (hi & c.rot_swap);
    const uint32_t b = (hi & ~c.rot_swap) | (lo & c.rot_swap);
    const uint32_t rh = funnel_l_var(a, b, c.rot_amt);
    const uint32_t rl = funnel_l_var(b, a, c.rot_amt);
    // pi (Eq. 6) and chi (Eq. 7): B[x,y], B[x+1,y], B[x+2,y] from their sources
    lo = chi3(shfl(rl, c.pi0), shfl(rl, c.pi1), shfl(rl, c.pi2));
    hi = chi3(shfl(rh, c.pi0), shfl(rh, c.pi1), shfl(rh, c.pi2));
    // iota (Eq. 8-9)
    lo ^= c_rc.w[2 * ir] & c.is_lane0;
    hi ^= c_rc.w[2 * ir + 1] & c.is_lane0;
}

__device__ __forceinline__ void lane_permute(const LaneCtx &c, uint32_t &lo, uint32_t &hi) {
#pragma unroll 2
    for (int ir = 0; ir < 24; ++ir) lane_round(c, lo, hi, ir);
}

// This thread's 8-byte word of absorbed block i (the padded last block when
// i == nfull), or zeros when its lane is outside the rate.
template <bool A8>
__device__ __forceinline__ void lane_block_word(const LaneCtx &c, const uint8_t *p, uint64_t i, uint64_t nfull,
                                                uint32_t rem, int rate, int nwords, uint32_t domain, uint32_t &wl,
                                                uint32_t &wh) {
    wl = wh = 0;
    if (c.t >= nwords) return;
    const uint8_t *q = p + i * uint64_t(rate) + 8 * c.t;
    if (i < nfull) {
        if constexpr (A8) ld_word_a8(q, wl, wh);
        else ld_word_any(q, 8, wl, wh);
        return;
    }
    if (8u * c.t + 8 <= rem) {
        if constexpr (A8) ld_word_a8(q, wl, wh);
        else ld_word_any(q, 8, wl, wh);
    } else if (8u * c.t < rem) {
        ld_word_any(q, rem - 8 * c.t, wl, wh);
    }
    if (uint32_t(c.t) == rem / 8) {
        const uint32_t sh = (rem % 8) * 8;
        if (sh < 32) wl ^= domain << sh;
        else wh ^= domain << (sh - 32);
    }
    if (c.t == nwords - 1) wh ^= 0x80000000u;
}

// One whole sponge for the message at p (8-byte aligned when A8), executed by
// the full warp; output written to dst.  All threads of the warp must call it
// with the same arguments.
template <bool A8>
__device__ __forceinline__ void lane_sponge(const uint8_t *p, uint64_t len, int variant, uint8_t *dst, uint32_t dlen) {
    const LaneCtx c = lane_ctx();
    const int rate = variant_rate(variant);
    const int nwords = rate / 8;
    const uint32_t domain = variant < 4 ? 0x06u : 0x1Fu;
    uint32_t lo = 0, hi = 0;
    const uint64_t nfull = len / uint64_t(rate);
    const uint32_t rem = uint32_t(len - nfull * uint64_t(rate));
    const uint32_t nsq = dlen > uint32_t(rate) ? (dlen - 1) / uint32_t(rate) : 0;
    uint32_t wl, wh;
    lane_block_word<A8>(c, p, 0, nfull, rem, rate, nwords, domain, wl, wh);
    for (uint64_t i = 0; i <= nfull; ++i) {
        lo ^= wl;
        hi ^= wh;
        // The next block's word is loaded while this permutation runs.
        if (i < nfull) lane_block_word<A8>(c, p, i + 1, nfull, rem, rate, nwords, domain, wl, wh);
        lane_permute(c, lo, hi);
    }
    // Squeeze: thread t writes bytes [8t, 8t+8) of each output block.
    for (uint32_t j = 0; j <= nsq; ++j) {
        const uint32_t base = j * uint32_t(rate);
        const uint32_t take = dlen - base < uint32_t(rate) ? dlen - base : uint32_t(rate);
        if (8u * c.t < take) {
            uint8_t *o = dst + base + 8 * c.t;
            const uint32_t nb = take - 8 * c.t < 8 ? take - 8 * c.t : 8;
            if (nb == 8 && (reinterpret_cast<uintptr_t>(o) & 7) == 0) {
                *reinterpret_cast<uint2 *>(o) = make_uint2(lo, hi);
            } else {
                const uint64_t w = (uint64_t(hi) << 32) | lo;
                for (uint32_t k = 0; k < nb; ++k) o[k] = uint8_t(w >> (8 * k));
            }
        }
        if (j < nsq) lane_permute(c, lo, hi);
    }
}

}  // namespace kb
