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

// Widths up to 32: lane x + 5y in one 32-bit register that holds its w bits
// 32/w times over (bit z of the lane at bits z, z + w, z + 2w, ...).  As 32 is
// a multiple of w, rotating the register by n rotates every copy of the lane
// by n within its w bits, so a lane rotation is one funnel shift with no
// mask; XOR, AND and NOT keep the copies equal, and the round constant is
// replicated the same way.  Only the low w bits are stored back.
template <int W>
struct SmallLanes {
    static constexpr uint32_t mask = W == 32 ? 0xffffffffu : ((1u << W) - 1u);
    static constexpr uint32_t spread = 0xffffffffu / mask;  // 1 at bits 0, w, 2w, ...
    __device__ static __forceinline__ uint32_t load(uint32_t v) { return (v & mask) * spread; }
    __device__ static __forceinline__ uint32_t store(uint32_t v) { return v & mask; }
    __device__ static __forceinline__ uint32_t rot(uint32_t x, int n) {
        return n % W == 0 ? x : __funnelshift_l(x, x, uint32_t(n % W));
    }
};

template <int W>
__device__ __forceinline__ void small_round(uint32_t (&A)[25], int ir) {
    using L = SmallLanes<W>;
    uint32_t C[5], D[5], Bv[25];
#pragma unroll
    for (int x = 0; x < 5; ++x) C[x] = A[x] ^ A[x + 5] ^ A[x + 10] ^ A[x + 15] ^ A[x + 20];
#pragma unroll
    for (int x = 0; x < 5; ++x) D[x] = C[(x + 4) % 5] ^ L::rot(C[(x + 1) % 5], 1);
#pragma unroll
    for (int y = 0; y < 5; ++y)
#pragma unroll
        for (int x = 0; x < 5; ++x) {
            // pi: B[y, 2x+3y] takes rho(A[x, y])
            const int src = x + 5 * y;
            Bv[y + 5 * ((2 * x + 3 * y) % 5)] = L::rot(A[src] ^ D[x], rho_offset(src));
        }
#pragma unroll
    for (int y = 0; y < 5; ++y)
#pragma unroll
        for (int x = 0; x < 5; ++x)
            A[x + 5 * y] = chi3(Bv[x + 5 * y], Bv[(x + 1) % 5 + 5 * y], Bv[(x + 2) % 5 + 5 * y]);
    A[0] ^= L::load(uint32_t(c_rc255.v[ir]));
}

// States move between global memory and registers through shared memory:
// each warp takes tiles of 32 consecutive 200-byte states (6.4 KB), copied
// with coalesced 8-byte accesses (the warp touches 256 contiguous bytes per
// access), and each thread then reads its own state from shared memory.
// Every warp has two tile buffers of its own: the next tile's copies
// (cp.async, 8 bytes each) are issued before the current tile is permuted,
// so a warp's loads overlap its own arithmetic, and warps synchronise only
// among their own threads (tiles of 128 states per block, with block
// barriers, measured 5-10% slower).  Reading the states straight from
// global memory, each thread 25 accesses 200 bytes apart, left the
// reduced-round runs waiting on memory.
constexpr uint32_t kWarpTile = 32;                                   // states per warp tile
constexpr uint32_t kTileWords = kWarpTile * 25;                      // uint2 words of a tile (6.4 KB)
constexpr size_t kTileSmem = size_t(kThreads / 32) * 2 * kTileWords * sizeof(uint2);  // per block

// The warp tiles of this warp, one warp-stride apart over the grid, each
// permuted state by state by f(uint2 *state) in shared memory and written
// back in place.
template <class F>
__device__ __forceinline__ void run_tiles(uint64_t *states, uint64_t n, uint2 *sm, F f) {
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const uint64_t ntiles = (n + kWarpTile - 1) / kWarpTile;
    const uint64_t nwarps = uint64_t(gridDim.x) * (blockDim.x / 32);
    uint64_t tile = uint64_t(blockIdx.x) * (blockDim.x / 32) + wib;
    uint2 *mine = sm + wib * 2 * kTileWords;
    const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(mine));
    auto count = [&](uint64_t t) {
        return uint32_t(n - t * kWarpTile < kWarpTile ? n - t * kWarpTile : uint64_t(kWarpTile));
    };
    auto load = [&](uint32_t sdst, uint64_t t) {
        const uint2 *src = reinterpret_cast<const uint2 *>(states + 25 * t * kWarpTile);
        const uint32_t words = count(t) * 25;
        for (uint32_t j = lane; j < words; j += 32)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sdst + 8 * j), "l"(src + j) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (tile >= ntiles) return;
    load(sbase, tile);
    for (uint32_t b = 0; tile < ntiles; tile += nwarps, b ^= 1u) {
        const uint64_t next = tile + nwarps;
        // The other buffer was last read before the warp barrier that ended
        // the previous pass, so the next tile may be copied into it now.
        if (next < ntiles) load(sbase + (b ^ 1u) * kTileWords * 8u, next);
        else asm volatile("cp.async.commit_group;" ::: "memory");  // an empty group keeps the count below uniform
        asm volatile("cp.async.wait_group 1;" ::: "memory");         // this tile's copies have landed
        __syncwarp();
        uint2 *cur = mine + b * kTileWords;
        const uint32_t cnt = count(tile);
        if (lane < cnt) f(cur + 25 * lane);
        __syncwarp();
        uint2 *dst = reinterpret_cast<uint2 *>(states + 25 * tile * kWarpTile);
        for (uint32_t j = lane; j < cnt * 25; j += 32) dst[j] = cur[j];
        __syncwarp();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_keccak_p_small(uint64_t *states, int first_ir, int nr, uint64_t n) {
    using L = SmallLanes<W>;
    extern __shared__ uint2 sm[];
    const int ir0 = ((first_ir % 255) + 255) % 255;  // rc has period 255 (Algorithm 5)
    run_tiles(states, n, sm, [&](uint2 *s) {
        uint32_t A[25];
#pragma unroll
        for (int k = 0; k < 25; ++k) A[k] = L::load(s[k].x);
        int ir = ir0;
        for (int r = 0; r < nr; ++r) {
            small_round<W>(A, ir);
            ir = ir == 254 ? 0 : ir + 1;
        }
#pragma unroll
        for (int k = 0; k < 25; ++k) s[k] = make_uint2(L::store(A[k]), 0u);
    });
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

// Width 64: n_r rounds of the plain 32-bit-half round of the hashing kernels
// on registers L, H from round-constant index first_ir.  Keccak-f[1600]
// itself (first_ir 0, 24 rounds) runs the hashing kernels' permutation;
// other round ranges run four rounds per loop pass, so that the compiler
// renames the state between rounds instead of copying it.
__device__ __forceinline__ void p1600_rounds(uint32_t (&L)[25], uint32_t (&H)[25], int first_ir, int nr) {
    if (first_ir == 0 && nr == 24) {
        keccak_f1600_plain<false>(L, H);
        return;
    }
    int ir = ((first_ir % 255) + 255) % 255, r = 0;  // rc has period 255 (Algorithm 5)
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

// STAGED: states pass through shared memory as in k_keccak_p_small, which
// pays off when the rounds are few (the memory latency is then a large part
// of a state's time); without it each thread reads and writes its own state
// directly, which keeps blocks free of barriers when the rounds dominate.
template <bool STAGED>
__global__ void __launch_bounds__(kThreads) k_keccak_p_1600(uint64_t *states, int first_ir, int nr, uint64_t n) {
    if constexpr (STAGED) {
        extern __shared__ uint2 sm[];
        run_tiles(states, n, sm, [&](uint2 *s) {
            uint32_t L[25], H[25];
#pragma unroll
            for (int k = 0; k < 25; ++k) {
                const uint2 v = s[k];
                L[k] = v.x;
                H[k] = v.y;
            }
            p1600_rounds(L, H, first_ir, nr);
#pragma unroll
            for (int k = 0; k < 25; ++k) s[k] = make_uint2(L[k], H[k]);
        });
    } else {
        const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
        for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
            uint2 *s = reinterpret_cast<uint2 *>(states + 25 * i);
            uint32_t L[25], H[25];
#pragma unroll
            for (int k = 0; k < 25; ++k) {
                const uint2 v = s[k];
                L[k] = v.x;
                H[k] = v.y;
            }
            p1600_rounds(L, H, first_ir, nr);
#pragma unroll
            for (int k = 0; k < 25; ++k) s[k] = make_uint2(L[k], H[k]);
        }
    }
}

// Launches a tiled kernel with its two tile buffers (above the 48 KB a block
// gets without opting in).
template <class K>
int launch_tiled(K kernel, uint64_t *states, int first_ir, int nr, uint64_t n, cudaStream_t stream,
                 const DeviceInfo &dev) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTileSmem)) != cudaSuccess)
        return cuda_status(cudaGetLastError());
    const uint64_t g = persistent_grid(reinterpret_cast<const void *>(kernel), kThreads, kTileSmem, n, dev);
    kernel<<<unsigned(g), kThreads, kTileSmem, stream>>>(states, first_ir, nr, n);
    return cuda_status(cudaGetLastError());
}

template <int W>
int launch_small(uint64_t *states, int first_ir, int nr, uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    return launch_tiled(k_keccak_p_small<W>, states, first_ir, nr, n, stream, dev);
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
            // Staged through shared memory below 16 rounds (measured on 2^24
            // states: 12 rounds 2.53 ms read directly, 2.15 ms staged; 24
            // rounds 3.84 ms directly, 4.02 ms staged).
            if (nr < 16) return launch_tiled(k_keccak_p_1600<true>, states, first_ir, nr, n, stream, dev);
            const uint64_t g =
                persistent_grid(reinterpret_cast<const void *>(&k_keccak_p_1600<false>), kThreads, 0, n, dev);
            k_keccak_p_1600<false><<<unsigned(g), kThreads, 0, stream>>>(states, first_ir, nr, n);
            return cuda_status(cudaGetLastError());
        }
    }
}

}  // namespace kb
