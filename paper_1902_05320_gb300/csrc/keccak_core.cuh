// keccak_core.cuh -- device primitives of the batch SHA-3 library (sm_103a).
//
// The 1600-bit state is 25 lanes of 64 bits, lane index i = x + 5y (Eq. 1:
// lane bit z is state bit 64(5y+x)+z).  It lives in registers as 50 32-bit
// words, in one of two representations chosen at compile time:
//
//  * PlainRep (the default): lane i is (L[i], H[i]) = its low and high 32-bit
//    halves, i.e. the little-endian message words themselves.  A 64-bit
//    rotation by n is two SHF funnel shifts (none for n = 0, a register swap
//    for n = 32).
//  * InterleavedRep: lane i is (E[i], O[i]) = its even and odd bits.  A 64-bit
//    rotation becomes two 32-bit rotations, which saves 6 SHF per round
//    (theta's rotation by 1 and rho's offset-1 lane need one SHF instead of
//    two), but every absorbed or squeezed 64-bit word costs 26 instructions of
//    bit interleaving.  On sm_103a's half-rate integer pipe the conversion
//    outweighs the saving for every message size, so this form is kept as the
//    measured control.
//
// Round function (Eq. 10), per 32-bit word, written as LOP3 and SHF:
//   theta (Eq. 2-4): column parities C (two 3-input XORs per word), the
//     rotated parity rot(C[x+1], 1), then A ^ C[x-1] ^ rot(C[x+1], 1) in one
//     3-input LOP3 per word;
//   rho (Eq. 5, as FIPS 202 Algorithm 2) + pi (Eq. 6): constant funnel shifts
//     and a compile-time renaming of registers (pi costs nothing);
//   chi (Eq. 7): a ^ (~b & c), one LOP3 per word;
//   iota (Eq. 8-9, the paper's "zeta"): XOR of the round constant into lane 0.
// Plain form: 20 + 10 + 50 + 48 + 50 + 2 = 180 instructions per round.
//
// Round structure: the first rounds run in a loop of four rounds per
// iteration that reads the round constants from a __constant__ table (the
// placement Section 4.2 uses) -- a fully unrolled 24-round body is larger
// than the instruction cache serves well; the last four rounds are unrolled
// with the constants as immediates, so when only a few output lanes are used
// the compiler drops the rest of the final round.  Round 0 can be peeled the
// same way when most of the input state is known to be zero.
#pragma once

#include <cstdint>
#include <utility>

namespace kb {

// ---- compile-time constants -------------------------------------------------

// rc(t) of Definition 5: FIPS 202 Algorithm 5, with the 8-bit register packed
// into an integer (bit k = R[k]); one step is "prepend 0, fold R[8] into
// bits 0, 4, 5, 6, drop R[8]".
__host__ __device__ constexpr int rc_bit(int t) {
    int tm = ((t % 255) + 255) % 255;
    unsigned R = 1;
    for (int i = 0; i < tm; ++i) {
        R <<= 1;
        if (R & 0x100u) R ^= 0x100u | 0x1u | 0x10u | 0x20u | 0x40u;
    }
    return int(R & 1u);
}

// RC lane of round i_r for w = 64 (l = 6): bit 2^j - 1 is rc(j + 7 i_r).
__host__ __device__ constexpr uint64_t round_constant(int ir) {
    uint64_t v = 0;
    for (int j = 0; j <= 6; ++j)
        if (rc_bit(j + 7 * ir)) v |= uint64_t(1) << ((1 << j) - 1);
    return v;
}

// rho offset of lane i = x + 5y: (t+1)(t+2)/2 mod 64 at step t of the walk
// (x, y) <- (y, 2x + 3y mod 5) that starts at (1, 0); 0 for lane (0, 0).
__host__ __device__ constexpr int rho_offset(int lane) {
    if (lane == 0) return 0;
    int x = 1, y = 0;
    for (int t = 0; t < 24; ++t) {
        if (x + 5 * y == lane) return ((t + 1) * (t + 2) / 2) % 64;
        int nx = y, ny = (2 * x + 3 * y) % 5;
        x = nx;
        y = ny;
    }
    return -1;
}

// Even / odd bits of a 64-bit value (interleaved representation).
__host__ __device__ constexpr uint32_t even_half(uint64_t v) {
    uint32_t r = 0;
    for (int k = 0; k < 32; ++k) r |= uint32_t((v >> (2 * k)) & 1) << k;
    return r;
}
__host__ __device__ constexpr uint32_t odd_half(uint64_t v) {
    uint32_t r = 0;
    for (int k = 0; k < 32; ++k) r |= uint32_t((v >> (2 * k + 1)) & 1) << k;
    return r;
}

// The round constants as (low, high) 32-bit words, for the looped rounds.
struct RcTable {
    uint32_t w[48];
};
__host__ __device__ constexpr RcTable make_rc_table() {
    RcTable t{};
    for (int i = 0; i < 24; ++i) {
        t.w[2 * i] = uint32_t(round_constant(i));
        t.w[2 * i + 1] = uint32_t(round_constant(i) >> 32);
    }
    return t;
}
static __constant__ RcTable c_rc = make_rc_table();

// ---- instruction wrappers -----------------------------------------------------

__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// a ^ (~b & c): the chi row function.
__device__ __forceinline__ uint32_t chi3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xD2;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Upper 32 bits of (hi:lo) << N, 0 < N < 32 (one SHF).
template <int N>
__device__ __forceinline__ uint32_t funnel_l(uint32_t lo, uint32_t hi) {
    uint32_t d;
    asm("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(lo), "r"(hi), "n"(N));
    return d;
}

template <int N>
__device__ __forceinline__ uint32_t rotl32(uint32_t x) {
    if constexpr ((N & 31) == 0) return x;
    else return funnel_l<(N & 31)>(x, x);
}

// ---- plain representation: 64-bit rotation of (lo, hi) ------------------------

template <int N>
__device__ __forceinline__ void rotl64(uint32_t lo, uint32_t hi, uint32_t &nl, uint32_t &nh) {
    if constexpr (N == 0) {
        nl = lo;
        nh = hi;
    } else if constexpr (N == 32) {
        nl = hi;
        nh = lo;
    } else if constexpr (N < 32) {
        nh = funnel_l<N>(lo, hi);
        nl = funnel_l<N>(hi, lo);
    } else {
        nh = funnel_l<N - 32>(hi, lo);
        nl = funnel_l<N - 32>(lo, hi);
    }
}

// theta's column terms for the source lane of (X, Y), then rho; pi is the
// choice of source: Eq. 6, A'[x,y] = A[(x+3y) mod 5, x].
template <int X, int Y>
__device__ __forceinline__ void plain_theta_rho_pi(const uint32_t (&L)[25], const uint32_t (&H)[25],
                                                   const uint32_t (&CL)[5], const uint32_t (&CH)[5],
                                                   const uint32_t (&RL)[5], const uint32_t (&RH)[5],
                                                   uint32_t &bl, uint32_t &bh) {
    constexpr int SX = (X + 3 * Y) % 5;
    constexpr int SRC = SX + 5 * X;
    // Eq. 4 with D[x] = C[x-1] ^ rot(C[x+1], 1) (Eq. 3).
    const uint32_t tl = xor3(L[SRC], CL[(SX + 4) % 5], RL[(SX + 1) % 5]);
    const uint32_t th = xor3(H[SRC], CH[(SX + 4) % 5], RH[(SX + 1) % 5]);
    rotl64<rho_offset(SRC)>(tl, th, bl, bh);
}

template <int Y>
__device__ __forceinline__ void plain_row(const uint32_t (&L)[25], const uint32_t (&H)[25], const uint32_t (&CL)[5],
                                          const uint32_t (&CH)[5], const uint32_t (&RL)[5], const uint32_t (&RH)[5],
                                          uint32_t (&NL)[25], uint32_t (&NH)[25]) {
    uint32_t BL[5], BH[5];
    plain_theta_rho_pi<0, Y>(L, H, CL, CH, RL, RH, BL[0], BH[0]);
    plain_theta_rho_pi<1, Y>(L, H, CL, CH, RL, RH, BL[1], BH[1]);
    plain_theta_rho_pi<2, Y>(L, H, CL, CH, RL, RH, BL[2], BH[2]);
    plain_theta_rho_pi<3, Y>(L, H, CL, CH, RL, RH, BL[3], BH[3]);
    plain_theta_rho_pi<4, Y>(L, H, CL, CH, RL, RH, BL[4], BH[4]);
#pragma unroll
    for (int x = 0; x < 5; ++x) {  // Eq. 7
        NL[x + 5 * Y] = chi3(BL[x], BL[(x + 1) % 5], BL[(x + 2) % 5]);
        NH[x + 5 * Y] = chi3(BH[x], BH[(x + 1) % 5], BH[(x + 2) % 5]);
    }
}

// One round without iota; the caller XORs the round constant into lane 0.
__device__ __forceinline__ void plain_round_body(uint32_t (&L)[25], uint32_t (&H)[25], uint32_t (&NL)[25],
                                                 uint32_t (&NH)[25]) {
    uint32_t CL[5], CH[5], RL[5], RH[5];
#pragma unroll
    for (int x = 0; x < 5; ++x) {  // Eq. 2
        CL[x] = xor3(xor3(L[x], L[x + 5], L[x + 10]), L[x + 15], L[x + 20]);
        CH[x] = xor3(xor3(H[x], H[x + 5], H[x + 10]), H[x + 15], H[x + 20]);
    }
#pragma unroll
    for (int x = 0; x < 5; ++x) rotl64<1>(CL[x], CH[x], RL[x], RH[x]);
    plain_row<0>(L, H, CL, CH, RL, RH, NL, NH);
    plain_row<1>(L, H, CL, CH, RL, RH, NL, NH);
    plain_row<2>(L, H, CL, CH, RL, RH, NL, NH);
    plain_row<3>(L, H, CL, CH, RL, RH, NL, NH);
    plain_row<4>(L, H, CL, CH, RL, RH, NL, NH);
}

// Round i_r with its constant read from the __constant__ table.
__device__ __forceinline__ void plain_round_rt(uint32_t (&L)[25], uint32_t (&H)[25], int ir) {
    uint32_t NL[25], NH[25];
    plain_round_body(L, H, NL, NH);
    NL[0] ^= c_rc.w[2 * ir];  // Eq. 9
    NH[0] ^= c_rc.w[2 * ir + 1];
#pragma unroll
    for (int i = 0; i < 25; ++i) {
        L[i] = NL[i];
        H[i] = NH[i];
    }
}

// Round IR with its constant as an immediate.
template <int IR>
__device__ __forceinline__ void plain_round_ct(uint32_t (&L)[25], uint32_t (&H)[25]) {
    constexpr uint64_t RC = round_constant(IR);
    uint32_t NL[25], NH[25];
    plain_round_body(L, H, NL, NH);
    if constexpr (uint32_t(RC) != 0) NL[0] ^= uint32_t(RC);
    if constexpr (uint32_t(RC >> 32) != 0) NH[0] ^= uint32_t(RC >> 32);
#pragma unroll
    for (int i = 0; i < 25; ++i) {
        L[i] = NL[i];
        H[i] = NH[i];
    }
}

template <int FIRST, int... K>
__device__ __forceinline__ void plain_rounds_ct(uint32_t (&L)[25], uint32_t (&H)[25],
                                                std::integer_sequence<int, K...>) {
    (plain_round_ct<FIRST + K>(L, H), ...);
}

// Keccak-f[1600] = Keccak-p[1600, 24] (Eq. 10, i_r = 0..23).  PEEL0 runs
// round 0 with an immediate constant so that known-zero input lanes fold.
template <bool PEEL0>
__device__ __forceinline__ void keccak_f1600_plain(uint32_t (&L)[25], uint32_t (&H)[25]) {
    constexpr int kLoopUnroll = 4;
    constexpr int kFirst = PEEL0 ? 1 : 0;
    constexpr int kTail = PEEL0 ? 21 : 20;  // rounds [kTail, 24) unrolled
    if constexpr (PEEL0) plain_round_ct<0>(L, H);
#pragma unroll 1
    for (int r = kFirst; r < kTail; r += kLoopUnroll) {
#pragma unroll
        for (int j = 0; j < kLoopUnroll; ++j) plain_round_rt(L, H, r + j);
    }
    plain_rounds_ct<kTail>(L, H, std::make_integer_sequence<int, 24 - kTail>{});
}

// ---- representations ------------------------------------------------------------

struct PlainRep {
    static constexpr const char *name = "plain";
    // 64-bit little-endian word (lo, hi) <-> the lane's two state words.
    __device__ __forceinline__ static void xor_word(uint32_t &a, uint32_t &b, uint32_t lo, uint32_t hi) {
        a ^= lo;
        b ^= hi;
    }
    __device__ __forceinline__ static void set_word(uint32_t &a, uint32_t &b, uint32_t lo, uint32_t hi) {
        a = lo;
        b = hi;
    }
    __device__ __forceinline__ static void get_word(uint32_t a, uint32_t b, uint32_t &lo, uint32_t &hi) {
        lo = a;
        hi = b;
    }
    // A compile-time 64-bit lane value in this representation.
    __host__ __device__ static constexpr uint32_t word_a(uint64_t v) { return uint32_t(v); }
    __host__ __device__ static constexpr uint32_t word_b(uint64_t v) { return uint32_t(v >> 32); }
    template <bool PEEL0>
    __device__ __forceinline__ static void permute(uint32_t (&A)[25], uint32_t (&B)[25]) {
        keccak_f1600_plain<PEEL0>(A, B);
    }
};

// ---- variants -----------------------------------------------------------------

// Rate in bytes, digest size (0 = caller-chosen, SHAKE) and the domain byte:
// the suffix bits "01" (SHA3) or "1111" (SHAKE) of Eq. 13-18 followed by the
// first padding bit of pad10*1, packed LSB-first (0x06 and 0x1F).
template <int V> struct Variant;
template <> struct Variant<0> { static constexpr int rate = 144, digest = 28, domain = 0x06; };
template <> struct Variant<1> { static constexpr int rate = 136, digest = 32, domain = 0x06; };
template <> struct Variant<2> { static constexpr int rate = 104, digest = 48, domain = 0x06; };
template <> struct Variant<3> { static constexpr int rate = 72, digest = 64, domain = 0x06; };
template <> struct Variant<4> { static constexpr int rate = 168, digest = 0, domain = 0x1F; };
template <> struct Variant<5> { static constexpr int rate = 136, digest = 0, domain = 0x1F; };

__host__ __device__ constexpr int variant_rate(int v) {
    return v == 0 ? 144 : v == 1 ? 136 : v == 2 ? 104 : v == 3 ? 72 : v == 4 ? 168 : v == 5 ? 136 : 0;
}
__host__ __device__ constexpr int variant_digest(int v) {
    return v == 0 ? 28 : v == 1 ? 32 : v == 2 ? 48 : v == 3 ? 64 : 0;
}

}  // namespace kb
