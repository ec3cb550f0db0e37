// keccak_interleaved.cuh -- the bit-interleaved representation of the state
// (lane i held as its even bits E[i] and odd bits O[i]), kept as the measured
// control for the plain representation of keccak_core.cuh.
//
// A 64-bit rotation by n becomes two 32-bit rotations: by n/2 on both halves
// for even n; for odd n the halves swap, E' = rotl(O, (n+1)/2) and
// O' = rotl(E, (n-1)/2).  theta's rotation by 1 and rho's offset-1 lane then
// need one SHF instead of two, so a round is 174 instructions instead of 180,
// at the price of 26 instructions per absorbed or squeezed 64-bit word.  The
// 24 rounds are fully unrolled with immediate round constants.
#pragma once

#include "keccak_core.cuh"

namespace kb {

// Gathers the even bits of x into bytes 0 and 2 and the odd bits into bytes
// 1 and 3 (three delta swaps of an inverse perfect shuffle).
__device__ __forceinline__ uint32_t unshuffle_bytes(uint32_t x) {
    uint32_t t;
    t = (x ^ (x >> 1)) & 0x22222222u; x ^= t ^ (t << 1);
    t = (x ^ (x >> 2)) & 0x0C0C0C0Cu; x ^= t ^ (t << 2);
    t = (x ^ (x >> 4)) & 0x00F000F0u; x ^= t ^ (t << 4);
    return x;
}

// Inverse of unshuffle_bytes.
__device__ __forceinline__ uint32_t shuffle_bytes(uint32_t x) {
    uint32_t t;
    t = (x ^ (x >> 4)) & 0x00F000F0u; x ^= t ^ (t << 4);
    t = (x ^ (x >> 2)) & 0x0C0C0C0Cu; x ^= t ^ (t << 2);
    t = (x ^ (x >> 1)) & 0x22222222u; x ^= t ^ (t << 1);
    return x;
}

// 64-bit little-endian word (lo = bytes 0..3, hi = bytes 4..7) -> (E, O).
__device__ __forceinline__ void to_interleaved(uint32_t lo, uint32_t hi, uint32_t &e, uint32_t &o) {
    lo = unshuffle_bytes(lo);
    hi = unshuffle_bytes(hi);
    e = __byte_perm(lo, hi, 0x6420);
    o = __byte_perm(lo, hi, 0x7531);
}

// (E, O) -> 64-bit little-endian word halves.
__device__ __forceinline__ void from_interleaved(uint32_t e, uint32_t o, uint32_t &lo, uint32_t &hi) {
    lo = shuffle_bytes(__byte_perm(e, o, 0x5140));
    hi = shuffle_bytes(__byte_perm(e, o, 0x7362));
}

template <int X, int Y>
__device__ __forceinline__ void il_theta_rho_pi(const uint32_t (&E)[25], const uint32_t (&O)[25],
                                                const uint32_t (&CE)[5], const uint32_t (&CO)[5],
                                                const uint32_t (&RE)[5], uint32_t &be, uint32_t &bo) {
    constexpr int SX = (X + 3 * Y) % 5;
    constexpr int SRC = SX + 5 * X;
    constexpr int N = rho_offset(SRC);
    // The even half of rot(C, 1) is rotl(C_odd, 1); its odd half is C_even.
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
__device__ __forceinline__ void il_row(const uint32_t (&E)[25], const uint32_t (&O)[25], const uint32_t (&CE)[5],
                                       const uint32_t (&CO)[5], const uint32_t (&RE)[5], uint32_t (&NE)[25],
                                       uint32_t (&NO)[25]) {
    uint32_t BE[5], BO[5];
    il_theta_rho_pi<0, Y>(E, O, CE, CO, RE, BE[0], BO[0]);
    il_theta_rho_pi<1, Y>(E, O, CE, CO, RE, BE[1], BO[1]);
    il_theta_rho_pi<2, Y>(E, O, CE, CO, RE, BE[2], BO[2]);
    il_theta_rho_pi<3, Y>(E, O, CE, CO, RE, BE[3], BO[3]);
    il_theta_rho_pi<4, Y>(E, O, CE, CO, RE, BE[4], BO[4]);
#pragma unroll
    for (int x = 0; x < 5; ++x) {
        NE[x + 5 * Y] = chi3(BE[x], BE[(x + 1) % 5], BE[(x + 2) % 5]);
        NO[x + 5 * Y] = chi3(BO[x], BO[(x + 1) % 5], BO[(x + 2) % 5]);
    }
}

template <int IR>
__device__ __forceinline__ void il_round(uint32_t (&E)[25], uint32_t (&O)[25]) {
    uint32_t CE[5], CO[5], RE[5];
#pragma unroll
    for (int x = 0; x < 5; ++x) {
        CE[x] = xor3(xor3(E[x], E[x + 5], E[x + 10]), E[x + 15], E[x + 20]);
        CO[x] = xor3(xor3(O[x], O[x + 5], O[x + 10]), O[x + 15], O[x + 20]);
    }
#pragma unroll
    for (int x = 0; x < 5; ++x) RE[x] = rotl32<1>(CO[x]);
    uint32_t NE[25], NO[25];
    il_row<0>(E, O, CE, CO, RE, NE, NO);
    il_row<1>(E, O, CE, CO, RE, NE, NO);
    il_row<2>(E, O, CE, CO, RE, NE, NO);
    il_row<3>(E, O, CE, CO, RE, NE, NO);
    il_row<4>(E, O, CE, CO, RE, NE, NO);
    constexpr uint64_t RC = round_constant(IR);
    if constexpr (even_half(RC) != 0) NE[0] ^= even_half(RC);
    if constexpr (odd_half(RC) != 0) NO[0] ^= odd_half(RC);
#pragma unroll
    for (int i = 0; i < 25; ++i) {
        E[i] = NE[i];
        O[i] = NO[i];
    }
}

template <int... IR>
__device__ __forceinline__ void il_rounds(uint32_t (&E)[25], uint32_t (&O)[25], std::integer_sequence<int, IR...>) {
    (il_round<IR>(E, O), ...);
}

struct InterleavedRep {
    static constexpr const char *name = "interleaved";
    __device__ __forceinline__ static void xor_word(uint32_t &a, uint32_t &b, uint32_t lo, uint32_t hi) {
        uint32_t e, o;
        to_interleaved(lo, hi, e, o);
        a ^= e;
        b ^= o;
    }
    __device__ __forceinline__ static void set_word(uint32_t &a, uint32_t &b, uint32_t lo, uint32_t hi) {
        to_interleaved(lo, hi, a, b);
    }
    __device__ __forceinline__ static void get_word(uint32_t a, uint32_t b, uint32_t &lo, uint32_t &hi) {
        from_interleaved(a, b, lo, hi);
    }
    __host__ __device__ static constexpr uint32_t word_a(uint64_t v) { return even_half(v); }
    __host__ __device__ static constexpr uint32_t word_b(uint64_t v) { return odd_half(v); }
    template <bool PEEL0>
    __device__ __forceinline__ static void permute(uint32_t (&A)[25], uint32_t (&B)[25]) {
        il_rounds(A, B, std::make_integer_sequence<int, 24>{});
    }
};

}  // namespace kb
