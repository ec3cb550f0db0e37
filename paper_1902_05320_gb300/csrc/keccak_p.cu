// keccak_p.cu -- the permutation alone: Keccak-p[b, n_r] (Section 3.1, Table 1
// widths, Eq. 10) applied in place to a batch of raw states, for every width
// b = 25w (w = 1, 2, 4, ..., 64) and any number of rounds n_r, with the round
// indices of FIPS 202 Algorithm 7 (the last n_r of 12 + 2l).  This is the
// tool for reduced-round and small-width experiments; the hashing entry
// points use the fixed Keccak-f[1600].
//
// The round constant of width w is the 64-bit one truncated to w bits (its
// bits sit at 2^j - 1 for j <= l), and rc has period 255, so one table of 255
// lanes serves all widths and all round indices.
#include <cuda_runtime.h>

#include "keccak_core.cuh"
#include "runtime.cuh"

namespace kb {
namespace {

struct Rc255 {
    uint64_t v[255];
};
__host__ __device__ constexpr Rc255 make_rc255() {
    int seq[255] = {};
    unsigned R = 1;  // rc(t) for t = 0..254, the register stepped once per t
    for (int t = 0; t < 255; ++t) {
        seq[t] = int(R & 1u);
        R <<= 1;
        if (R & 0x100u) R ^= 0x100u | 0x1u | 0x10u | 0x20u | 0x40u;
    }
    Rc255 out{};
    for (int ir = 0; ir < 255; ++ir) {
        uint64_t v = 0;
        for (int j = 0; j <= 6; ++j)
            if (seq[(j + 7 * ir) % 255]) v |= uint64_t(1) << ((1 << j) - 1);
        out.v[ir] = v;
    }
    return out;
}
static __constant__ Rc255 c_rc255 = make_rc255();

template <int W>
__device__ __forceinline__ uint32_t rotw(uint32_t x, int n) {
    constexpr uint32_t mask = W == 32 ? 0xffffffffu : ((1u << W) - 1u);
    n %= W;
    if (n == 0) return x;
    return ((x << n) | (x >> (W - n))) & mask;
}

// Widths up to 32: one 32-bit word per lane.
template <int W>
__device__ __forceinline__ void small_round(uint32_t (&A)[25], int ir) {
    uint32_t C[5], D[5], Bv[25];
#pragma unroll
    for (int x = 0; x < 5; ++x) C[x] = A[x] ^ A[x + 5] ^ A[x + 10] ^ A[x + 15] ^ A[x + 20];
#pragma unroll
    for (int x = 0; x < 5; ++x) D[x] = C[(x + 4) % 5] ^ rotw<W>(C[(x + 1) % 5], 1);
#pragma unroll
    for (int y = 0; y < 5; ++y)
#pragma unroll
        for (int x = 0; x < 5; ++x) {
            // pi: B[y, 2x+3y] takes rho(A[x, y])
            const int src = x + 5 * y;
            Bv[y + 5 * ((2 * x + 3 * y) % 5)] = rotw<W>(A[src] ^ D[x], rho_offset(src));
        }
#pragma unroll
    for (int y = 0; y < 5; ++y)
#pragma unroll
        for (int x = 0; x < 5; ++x)
            A[x + 5 * y] = chi3(Bv[x + 5 * y], Bv[(x + 1) % 5 + 5 * y], Bv[(x + 2) % 5 + 5 * y]);
    constexpr uint32_t mask = W == 32 ? 0xffffffffu : ((1u << W) - 1u);
    A[0] ^= uint32_t(c_rc255.v[ir]) & mask;
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_keccak_p_small(uint64_t *states, int first_ir, int nr, uint64_t n) {
    constexpr uint64_t mask = W == 32 ? 0xffffffffull : ((1ull << W) - 1ull);
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
        uint64_t *s = states + 25 * i;
        uint32_t A[25];
#pragma unroll
        for (int k = 0; k < 25; ++k) A[k] = uint32_t(s[k] & mask);
        int ir = ((first_ir % 255) + 255) % 255;  // rc has period 255 (Algorithm 5)
        for (int r = 0; r < nr; ++r) {
            small_round<W>(A, ir);
            ir = ir == 254 ? 0 : ir + 1;
        }
#pragma unroll
        for (int k = 0; k < 25; ++k) s[k] = A[k];
    }
}

// One round of Keccak-p[1600] (Eq. 10) with round-constant index ir of the
// period-255 table, in place.
__device__ __forceinline__ void p1600_round(uint32_t (&L)[25], uint32_t (&H)[25], int ir) {
    uint32_t NL[25], NH[25];
    plain_round_body(L, H, NL, NH);
    const uint64_t rc = c_rc255.v[ir];
    NL[0] ^= uint32_t(rc);
    NH[0] ^= uint32_t(rc >> 32);
#pragma unroll
    for (int k = 0; k < 25; ++k) {
        L[k] = NL[k];
        H[k] = NH[k];
    }
}

// Width 64: the plain 32-bit-half round of the hashing kernels.  Keccak-f[1600]
// itself (first_ir 0, 24 rounds) runs the hashing kernels' permutation;
// other round ranges run four rounds per loop pass, so that the compiler
// renames the state between rounds instead of copying it.
__global__ void __launch_bounds__(kThreads) k_keccak_p_1600(uint64_t *states, int first_ir, int nr, uint64_t n) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    const bool full = first_ir == 0 && nr == 24;
    const int ir0 = ((first_ir % 255) + 255) % 255;  // rc has period 255 (Algorithm 5)
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
        uint2 *s = reinterpret_cast<uint2 *>(states + 25 * i);
        uint32_t L[25], H[25];
#pragma unroll
        for (int k = 0; k < 25; ++k) {
            const uint2 v = s[k];
            L[k] = v.x;
            H[k] = v.y;
        }
        if (full) {
            keccak_f1600_plain<false>(L, H);
        } else {
            int ir = ir0, r = 0;
#pragma unroll 1
            for (; r + 4 <= nr; r += 4) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    p1600_round(L, H, ir);
                    ir = ir == 254 ? 0 : ir + 1;
                }
            }
            for (; r < nr; ++r) {
                p1600_round(L, H, ir);
                ir = ir == 254 ? 0 : ir + 1;
            }
        }
#pragma unroll
        for (int k = 0; k < 25; ++k) s[k] = make_uint2(L[k], H[k]);
    }
}

template <int W>
int launch_small(uint64_t *states, int first_ir, int nr, uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    const uint64_t g = persistent_grid(reinterpret_cast<const void *>(&k_keccak_p_small<W>), kThreads, 0, n, dev);
    k_keccak_p_small<W><<<unsigned(g), kThreads, 0, stream>>>(states, first_ir, nr, n);
    return cuda_status(cudaGetLastError());
}

}  // namespace

int launch_keccak_p(uint64_t *states, int b, int nr, uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    int l = -1;
    for (int k = 0; k <= 6; ++k)
        if (b == 25 * (1 << k)) l = k;
    if (l < 0) return KB_ERR_INVALID;
    const int first_ir = 12 + 2 * l - nr;
    switch (l) {
        case 0: return launch_small<1>(states, first_ir, nr, n, stream, dev);
        case 1: return launch_small<2>(states, first_ir, nr, n, stream, dev);
        case 2: return launch_small<4>(states, first_ir, nr, n, stream, dev);
        case 3: return launch_small<8>(states, first_ir, nr, n, stream, dev);
        case 4: return launch_small<16>(states, first_ir, nr, n, stream, dev);
        case 5: return launch_small<32>(states, first_ir, nr, n, stream, dev);
        default: {
            const uint64_t g =
                persistent_grid(reinterpret_cast<const void *>(&k_keccak_p_1600), kThreads, 0, n, dev);
            k_keccak_p_1600<<<unsigned(g), kThreads, 0, stream>>>(states, first_ir, nr, n);
            return cuda_status(cudaGetLastError());
        }
    }
}

}  // namespace kb
