// keccak_core.cuh -- device primitives of the batch SHA-3 library (sm_103a).
//
// State representation.  The 1600-bit state is 25 lanes of 64 bits, lane
// index i = x + 5y (Eq. 1, lane bit z = state bit 64(5y+x)+z).  Each lane is
// held in registers as two 32-bit halves in bit-interleaved form: E holds the
// lane's even bits (bit 2k of the lane is bit k of E), O its odd bits.  A
// 64-bit rotation by n then becomes two 32-bit rotations (one SHF each, none
// when the amount is 0): by n/2 on both halves for even n; for odd n the
// halves swap, E' = rotl(O, (n+1)/2) and O' = rotl(E, (n-1)/2).
//
// Round function (Eq. 10), per 32-bit half:
//   theta (Eq. 2-4): column parities C (two 3-input XOR LOP3s per half), the
//     rotated parity rot(C[x+1], 1) (one SHF per column: the odd-half part of
//     a rotation by 1 is a plain register rename), then each half-lane gets
//     A ^ C[x-1] ^ rot(C[x+1],1) in one 3-input LOP3.
//   rho (Eq. 5, as FIPS 202 Algorithm 2) + pi (Eq. 6): constant SHF amounts
//     and a compile-time renaming of registers; pi costs no instruction.
//   chi (Eq. 7): a ^ (~b & c), one LOP3 per half-lane.
//   iota (Eq. 8-9, the paper's "zeta"): XOR of compile-time immediates into
//     lane (0,0); a half whose constant is 0 costs nothing.
// That is at most 20 + 5 + 50 + 47 + 50 + 2 = 174 integer instructions per
// round.
//
// Round constants and rho offsets are computed at compile time by constexpr
// restatements of FIPS 202 Algorithm 5 (the LFSR rc) and of the rho walk, so
// the kernels carry them as instruction immediates (the paper kept them in
// constant memory, Section 4.2).
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

// Even / odd bits of a 64-bit constant, for interleaving immediates.
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

template <int N>
__device__ __forceinline__ uint32_t rotl32(uint32_t x) {
    if constexpr ((N & 31) == 0) {
        return x;
    } else {
        uint32_t d;
        asm("shf.l.wrap.b32 %0, %1, %1, %2;" : "=r"(d) : "r"(x), "n"(N & 31));
        return d;
    }
}

__device__ __forceinline__ uint32_t rotl32_1(uint32_t x) { return rotl32<1>(x); }

// ---- bit interleaving ---------------------------------------------------------

// Gathers the even bits of x into its low 16 bits and the odd bits into its
// high 16 bits (an inverse perfect shuffle made of four delta swaps).
__host__ __device__ __forceinline__ uint32_t unshuffle32(uint32_t x) {
    uint32_t t;
    t = (x ^ (x >> 1)) & 0x22222222u; x ^= t ^ (t << 1);
    t = (x ^ (x >> 2)) & 0x0C0C0C0Cu; x ^= t ^ (t << 2);
    t = (x ^ (x >> 4)) & 0x00F000F0u; x ^= t ^ (t << 4);
    t = (x ^ (x >> 8)) & 0x0000FF00u; x ^= t ^ (t << 8);
    return x;
}

// Inverse of unshuffle32.
__host__ __device__ __forceinline__ uint32_t shuffle32(uint32_t x) {
    uint32_t t;
    t = (x ^ (x >> 8)) & 0x0000FF00u; x ^= t ^ (t << 8);
    t = (x ^ (x >> 4)) & 0x00F000F0u; x ^= t ^ (t << 4);
    t = (x ^ (x >> 2)) & 0x0C0C0C0Cu; x ^= t ^ (t << 2);
    t = (x ^ (x >> 1)) & 0x22222222u; x ^= t ^ (t << 1);
    return x;
}

// 64-bit little-endian lane (lo = bytes 0..3, hi = bytes 4..7) -> (E, O).
__device__ __forceinline__ void to_interleaved(uint32_t lo, uint32_t hi, uint32_t &e, uint32_t &o) {
    lo = unshuffle32(lo);
    hi = unshuffle32(hi);
    e = __byte_perm(lo, hi, 0x5410);
    o = __byte_perm(lo, hi, 0x7632);
}

// (E, O) -> 64-bit little-endian lane halves.
__device__ __forceinline__ void from_interleaved(uint32_t e, uint32_t o, uint32_t &lo, uint32_t &hi) {
    lo = shuffle32(__byte_perm(e, o, 0x5410));
    hi = shuffle32(__byte_perm(e, o, 0x7632));
}

// ---- the permutation ------------------------------------------------------------

// theta's column terms for one source lane, then rho: writes the rotated
// half-lanes that pi places at (x, y).  SX is the source column.
template <int X, int Y>
__device__ __forceinline__ void theta_rho_pi(const uint32_t (&E)[25], const uint32_t (&O)[25],
                                             const uint32_t (&CE)[5], const uint32_t (&CO)[5],
                                             const uint32_t (&RE)[5], uint32_t &be, uint32_t &bo) {
    constexpr int SX = (X + 3 * Y) % 5;  // Eq. 6: A'[x,y] = A[(x+3y) mod 5, x]
    constexpr int SRC = SX + 5 * X;
    constexpr int N = rho_offset(SRC);
    // Eq. 4 with D[x] = C[x-1] ^ rot(C[x+1], 1); in interleaved form the even
    // half of rot(C,1) is rotl(C_odd, 1) and its odd half is C_even.
    const uint32_t te = xor3(E[SRC], CE[(SX + 4) % 5], RE[(SX + 1) % 5]);
    const uint32_t to = xor3(O[SRC], CO[(SX + 4) % 5], CE[(SX + 1) % 5]);
    if constexpr ((N & 1) == 0) {
        be = rotl32<N / 2>(te);
        bo = rotl32<N / 2>(to);
    } else {
        be = rotl32<(N + 1) / 2>(to);
        bo = rotl32<(N - 1) / 2>(te);
    }
}

template <int Y>
__device__ __forceinline__ void round_row(const uint32_t (&E)[25], const uint32_t (&O)[25],
                                          const uint32_t (&CE)[5], const uint32_t (&CO)[5],
                                          const uint32_t (&RE)[5], uint32_t (&NE)[25],
                                          uint32_t (&NO)[25]) {
    uint32_t BE[5], BO[5];
    theta_rho_pi<0, Y>(E, O, CE, CO, RE, BE[0], BO[0]);
    theta_rho_pi<1, Y>(E, O, CE, CO, RE, BE[1], BO[1]);
    theta_rho_pi<2, Y>(E, O, CE, CO, RE, BE[2], BO[2]);
    theta_rho_pi<3, Y>(E, O, CE, CO, RE, BE[3], BO[3]);
    theta_rho_pi<4, Y>(E, O, CE, CO, RE, BE[4], BO[4]);
#pragma unroll
    for (int x = 0; x < 5; ++x) {
        NE[x + 5 * Y] = chi3(BE[x], BE[(x + 1) % 5], BE[(x + 2) % 5]);
        NO[x + 5 * Y] = chi3(BO[x], BO[(x + 1) % 5], BO[(x + 2) % 5]);
    }
}

template <int IR>
__device__ __forceinline__ void keccak_round(uint32_t (&E)[25], uint32_t (&O)[25]) {
    uint32_t CE[5], CO[5], RE[5];
#pragma unroll
    for (int x = 0; x < 5; ++x) {
        CE[x] = xor3(xor3(E[x], E[x + 5], E[x + 10]), E[x + 15], E[x + 20]);
        CO[x] = xor3(xor3(O[x], O[x + 5], O[x + 10]), O[x + 15], O[x + 20]);
    }
#pragma unroll
    for (int x = 0; x < 5; ++x) RE[x] = rotl32_1(CO[x]);
    uint32_t NE[25], NO[25];
    round_row<0>(E, O, CE, CO, RE, NE, NO);
    round_row<1>(E, O, CE, CO, RE, NE, NO);
    round_row<2>(E, O, CE, CO, RE, NE, NO);
    round_row<3>(E, O, CE, CO, RE, NE, NO);
    round_row<4>(E, O, CE, CO, RE, NE, NO);
    constexpr uint64_t RC = round_constant(IR);
    constexpr uint32_t RCE = even_half(RC), RCO = odd_half(RC);
    if constexpr (RCE != 0) NE[0] ^= RCE;
    if constexpr (RCO != 0) NO[0] ^= RCO;
#pragma unroll
    for (int i = 0; i < 25; ++i) {
        E[i] = NE[i];
        O[i] = NO[i];
    }
}

template <int... IR>
__device__ __forceinline__ void keccak_rounds(uint32_t (&E)[25], uint32_t (&O)[25],
                                              std::integer_sequence<int, IR...>) {
    (keccak_round<IR>(E, O), ...);
}

// Keccak-f[1600] = Keccak-p[1600, 24], rounds i_r = 0..23, fully unrolled.
__device__ __forceinline__ void keccak_f1600(uint32_t (&E)[25], uint32_t (&O)[25]) {
    keccak_rounds(E, O, std::make_integer_sequence<int, 24>{});
}

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
