// merkle.cu -- tree mode (Section 4: digests combined pairwise, level after
// level, up to one root; the paper leaves it to future work with
// reductions).
//
// Node format: leaf = SHA3-256(0x00 || leaf bytes), inner node =
// SHA3-256(0x01 || left || right); levels are reduced one at a time and an odd
// last node is carried up unchanged.  All levels are written back to back
// (leaf digests first, root last) so that callers can also take proofs.
//
// Kernels: one thread per leaf (the prefixed message is read through a
// one-byte funnel shift of the leaf's aligned words), then one launch per
// level (0x01 || left || right is exactly one 65-byte block at rate 136):
// one thread per parent node while a level has more than 4096 parents, one
// warp per parent (lane-parallel, about half the latency of a permutation in
// one thread) below that down to 64 nodes, and one single-block launch, also
// a warp per parent, for all the levels above.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "keccak_core.cuh"
#include "lane_parallel.cuh"
#include "runtime.cuh"
#include "sponge.cuh"

namespace kb {
namespace {

constexpr int kRate = Variant<1>::rate;   // SHA3-256
constexpr int kDomain = Variant<1>::domain;

// Lane word g of the virtual message 0x00 || leaf, built from leaf words g-1
// and g: the byte that falls off the top of word g-1 becomes byte 0 of word g.
// `carry` holds the high half of leaf word g-1 (prefix << 24 for g = 0).
__device__ __forceinline__ void prefixed_word(uint32_t &carry, uint32_t lo, uint32_t hi, uint32_t &vlo,
                                              uint32_t &vhi) {
    vlo = __funnelshift_l(carry, lo, 8);
    vhi = __funnelshift_l(lo, hi, 8);
    carry = hi;
}

// Leaves at 8-byte aligned addresses with leaf_bytes % 8 == 0.
// XORs block b of the padded message 0x00 || leaf (leaf_bytes bytes at p,
// mwords = leaf_bytes / 8 words, nfull full blocks, rem bytes in the last)
// into the state.  The prefix byte is shifted in through one-byte funnel
// shifts of the leaf's aligned 8-byte words; carry holds the byte carried
// between words (0 before block 0).
__device__ __forceinline__ void absorb_leaf_block_a8(uint32_t (&A)[25], uint32_t (&B)[25], const uint8_t *p,
                                                     uint64_t b, uint64_t nfull, uint32_t rem, uint64_t mwords,
                                                     uint32_t &carry) {
    const uint64_t g0 = b * (kRate / 8);
    if (b < nfull) {
#pragma unroll
        for (int k = 0; k < kRate / 8; ++k) {
            uint32_t lo, hi, vlo, vhi;
            ld_word_a8(p + 8 * (g0 + k), lo, hi);
            prefixed_word(carry, lo, hi, vlo, vhi);
            PlainRep::xor_word(A[k], B[k], vlo, vhi);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kRate / 8; ++k) {
            uint32_t lo = 0, hi = 0, vlo, vhi;
            if (g0 + k < mwords) ld_word_a8(p + 8 * (g0 + k), lo, hi);
            prefixed_word(carry, lo, hi, vlo, vhi);
            if (uint32_t(k) == rem / 8) {
                const uint32_t sh = (rem % 8) * 8;
                if (sh < 32) vlo ^= uint32_t(kDomain) << sh;
                else vhi ^= uint32_t(kDomain) << (sh - 32);
            }
            if (k == kRate / 8 - 1) vhi ^= 0x80000000u;
            PlainRep::xor_word(A[k], B[k], vlo, vhi);
        }
    }
}

// The state after absorbing 0x00 || leaf and its padding, permuted:
// SHA3-256 of the prefixed leaf sits in lanes 0..3.
__device__ __forceinline__ void leaf_state_a8(const uint8_t *p, uint64_t leaf_bytes, uint32_t (&A)[25],
                                              uint32_t (&B)[25]) {
    const uint64_t vlen = leaf_bytes + 1;  // prefixed message length
    const uint64_t nfull = vlen / kRate;
    const uint32_t rem = uint32_t(vlen - nfull * kRate);
#pragma unroll
    for (int k = 0; k < 25; ++k) A[k] = B[k] = 0;
    uint32_t carry = 0x00u << 24;  // leaf prefix byte
    for (uint64_t b = 0; b <= nfull; ++b) {
        absorb_leaf_block_a8(A, B, p, b, nfull, rem, leaf_bytes / 8, carry);
        PlainRep::permute<false>(A, B);
    }
}

__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_merkle_leaves_a8(const uint8_t *__restrict__ buf, uint64_t n_leaves, uint64_t leaf_bytes,
                       uint8_t *__restrict__ out) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_leaves; i += step) {
        uint32_t A[25], B[25];
        leaf_state_a8(buf + i * leaf_bytes, leaf_bytes, A, B);
        squeeze<kRate, PlainRep>(A, B, out + 32 * i, 32);
    }
}

// Any alignment / leaf size: byte-exact reads through ld_word_any.
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_merkle_leaves_any(const uint8_t *__restrict__ buf, uint64_t n_leaves, uint64_t leaf_bytes,
                        uint8_t *__restrict__ out) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t vlen = leaf_bytes + 1;
    const uint64_t nfull = vlen / kRate;
    const uint32_t rem = uint32_t(vlen - nfull * kRate);
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_leaves; i += step) {
        const uint8_t *p = buf + i * leaf_bytes;
        uint32_t A[25], B[25];
#pragma unroll
        for (int k = 0; k < 25; ++k) A[k] = B[k] = 0;
        for (uint64_t b = 0; b <= nfull; ++b) {
            const uint32_t valid = b < nfull ? uint32_t(kRate) : rem;  // virtual bytes in this block
#pragma unroll
            for (int k = 0; k < kRate / 8; ++k) {
                // Virtual bytes [v0, v0 + 8) are leaf bytes [v0 - 1, v0 + 7).
                const uint64_t v0 = b * kRate + 8 * k;
                uint32_t lo = 0, hi = 0;
                const uint32_t inblk = 8 * k;
                if (inblk < valid) {
                    const uint32_t nv = valid - inblk < 8 ? valid - inblk : 8;  // virtual bytes present
                    if (v0 == 0) {
                        if (nv > 1) ld_word_any(p, nv - 1, lo, hi);
                        hi = __funnelshift_l(lo, hi, 8);
                        lo = (lo << 8) | 0x00u;
                    } else {
                        ld_word_any(p + (v0 - 1), nv, lo, hi);
                    }
                }
                if (b == nfull) {
                    if (uint32_t(k) == rem / 8) {
                        const uint32_t sh = (rem % 8) * 8;
                        if (sh < 32) lo ^= uint32_t(kDomain) << sh;
                        else hi ^= uint32_t(kDomain) << (sh - 32);
                    }
                    if (k == kRate / 8 - 1) hi ^= 0x80000000u;
                }
                PlainRep::xor_word(A[k], B[k], lo, hi);
            }
            PlainRep::permute<false>(A, B);
        }
        squeeze<kRate, PlainRep>(A, B, out + 32 * i, 32);
    }
}

// Parent j of one level: SHA3-256(0x01 || in[2j] || in[2j+1]); for an odd
// count the last child is copied to out[count/2].  `in` is 32-byte aligned.
// No __restrict__: in the top-of-tree kernel a level written by the block is
// read back by it after a barrier, so the loads must stay coherent ones.
__device__ __forceinline__ void merkle_parent(const uint8_t *in, uint64_t count, uint8_t *out, uint64_t j) {
    const uint64_t pairs = count / 2;
    if (j == pairs) {
        const uint4 *s = reinterpret_cast<const uint4 *>(in + 32 * (count - 1));
        uint4 *d = reinterpret_cast<uint4 *>(out + 32 * j);
        d[0] = s[0];
        d[1] = s[1];
        return;
    }
    uint32_t A[25], B[25];
#pragma unroll
    for (int k = 0; k < 25; ++k) A[k] = B[k] = 0;
    const uint4 *q = reinterpret_cast<const uint4 *>(in + 64 * j);
    uint32_t carry = 0x01u << 24;  // node prefix byte
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const uint4 v = q[t];
        uint32_t vlo, vhi;
        prefixed_word(carry, v.x, v.y, vlo, vhi);
        PlainRep::set_word(A[2 * t], B[2 * t], vlo, vhi);
        prefixed_word(carry, v.z, v.w, vlo, vhi);
        PlainRep::set_word(A[2 * t + 1], B[2 * t + 1], vlo, vhi);
    }
    // Word 8: the last child byte, then the domain byte at message offset 65.
    uint32_t vlo = (carry >> 24) | (uint32_t(kDomain) << 8), vhi = 0;
    PlainRep::set_word(A[8], B[8], vlo, vhi);
    B[kRate / 8 - 1] ^= 0x80000000u;
    PlainRep::permute<true>(A, B);
    squeeze<kRate, PlainRep>(A, B, out + 32 * j, 32);
}

// One level, one thread per parent.
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_merkle_level(const uint8_t *in, uint64_t count, uint8_t *out) {
    const uint64_t parents = count / 2 + (count & 1);
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < parents; j += step)
        merkle_parent(in, count, out, j);
}

// Parent j of a level of `count` nodes by one warp: the 25 lanes of the
// state on threads 0..24 (lane_parallel.cuh).  Thread t < 17 builds its
// 8-byte word of the padded block 0x01 || left || right from two 8-byte words
// of the children (the children of parent j are the 64 bytes at in + 64j),
// shifted by the prefix byte; the domain byte follows at byte 65 and 0x80
// closes the rate at byte 135.  An odd last node is copied up unchanged.
// Every thread of the warp must call it with the same j.
__device__ __forceinline__ void merkle_parent_lanes(const LaneCtx &c, const uint8_t *in, uint64_t count, uint8_t *out,
                                                    uint64_t j) {
    const int t = c.t;
    if (2 * j + 1 == count) {  // odd last node: carried up
        if (t < 4) {
            const uint2 v = *reinterpret_cast<const uint2 *>(in + 64 * j + 8 * t);
            *reinterpret_cast<uint2 *>(out + 32 * j + 8 * t) = v;
        }
        return;
    }
    const uint2 *ch = reinterpret_cast<const uint2 *>(in + 64 * j);
    uint32_t lo = 0, hi = 0;
    if (t <= 8) {
        // Virtual bytes [8t, 8t+8) = child bytes [8t-1, 8t+7).
        const uint2 cur = t < 8 ? ch[t] : make_uint2(0u, 0u);
        const uint2 prev = t > 0 ? ch[t - 1] : make_uint2(0u, 0x01u << 24);  // prefix byte at virtual byte 0
        lo = __funnelshift_l(prev.y, cur.x, 8);
        hi = __funnelshift_l(cur.x, cur.y, 8);
        if (t == 8) lo = (prev.y >> 24) | (uint32_t(kDomain) << 8);  // byte 64 = last child byte, 65 = domain
    }
    if (t == kRate / 8 - 1) hi ^= 0x80000000u;
    lane_permute(c, lo, hi);
    if (t < 4) *reinterpret_cast<uint2 *>(out + 32 * j + 8 * t) = make_uint2(lo, hi);
}

// One level, one warp per parent (levels of at most kLaneParents parents,
// where a permutation's latency, not the ALU pipe's throughput, sets the
// time: the warp form takes about half a thread's latency).
constexpr uint64_t kLaneParents = 4096;

__global__ void __launch_bounds__(kThreads) k_merkle_level_lanes(const uint8_t *in, uint64_t count, uint8_t *out) {
    const LaneCtx c = lane_ctx();
    const uint64_t parents = count / 2 + (count & 1);
    const uint64_t warps = uint64_t(gridDim.x) * (blockDim.x / 32);
    for (uint64_t j = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; j < parents; j += warps)
        merkle_parent_lanes(c, in, count, out, j);
}

// The top of the tree, from a level of at most kTopCount nodes up to the
// root, in one block: a block barrier separates the levels (each level is
// written to global memory, which the barrier makes visible to the block).
// Levels above that take one launch each over all SMs.  One SM hashes a
// level of P parents in about P x 68 cycles once P fills it, so the block
// starts only where a level is a single permutation's latency anyway (at
// most 32 parents): from 4096 nodes it took ~165 us, where per-level launches
// down to 64 nodes and the block from there take ~70 us.
// The block runs one warp per parent (lane-parallel), so its 32 warps take
// the 32 parents of a 64-node level at once.
constexpr int kTopThreads = 1024;
constexpr uint64_t kTopCount = 64;

__global__ void __launch_bounds__(kTopThreads) k_merkle_top(uint8_t *level, uint64_t count) {
    const LaneCtx c = lane_ctx();
    const uint64_t warp = threadIdx.x / 32;
    while (count > 1) {
        uint8_t *next = level + 32 * count;
        const uint64_t parents = count / 2 + (count & 1);
        for (uint64_t j = warp; j < parents; j += kTopThreads / 32) merkle_parent_lanes(c, level, count, next, j);
        __syncthreads();
        level = next;
        count = parents;
    }
}

// ---- many small trees, one thread per tree ----------------------------------

// XORs block b of the padded message 0x00 || leaf (leaf_bytes bytes at p, any
// alignment; nfull full blocks, rem bytes in the last) into the state,
// reading the leaf byte-exactly.
__device__ __forceinline__ void absorb_leaf_block_any(uint32_t (&A)[25], uint32_t (&B)[25], const uint8_t *p,
                                                      uint64_t b, uint64_t nfull, uint32_t rem) {
    const uint32_t valid = b < nfull ? uint32_t(kRate) : rem;
#pragma unroll
    for (int k = 0; k < kRate / 8; ++k) {
        const uint64_t v0 = b * kRate + 8 * k;  // virtual bytes [v0, v0+8) = leaf bytes [v0-1, v0+7)
        uint32_t lo = 0, hi = 0;
        if (uint32_t(8 * k) < valid) {
            const uint32_t nv = valid - 8 * k < 8 ? valid - 8 * k : 8;
            if (v0 == 0) {
                if (nv > 1) ld_word_any(p, nv - 1, lo, hi);
                hi = __funnelshift_l(lo, hi, 8);
                lo = lo << 8;  // prefix byte 0x00
            } else {
                ld_word_any(p + (v0 - 1), nv, lo, hi);
            }
        }
        if (b == nfull) {
            if (uint32_t(k) == rem / 8) {
                const uint32_t sh = (rem % 8) * 8;
                if (sh < 32) lo ^= uint32_t(kDomain) << sh;
                else hi ^= uint32_t(kDomain) << (sh - 32);
            }
            if (k == kRate / 8 - 1) hi ^= 0x80000000u;
        }
        PlainRep::xor_word(A[k], B[k], lo, hi);
    }
}

// The state holding the padded block of 0x01 || left || right (digests as
// eight little-endian 32-bit words each), ready to permute.
__device__ __forceinline__ void load_node_block(uint32_t (&A)[25], uint32_t (&B)[25], const uint32_t (&l)[8],
                                                const uint32_t (&r)[8]) {
#pragma unroll
    for (int k = 0; k < 25; ++k) A[k] = B[k] = 0;
    uint32_t carry = 0x01u << 24;  // node prefix byte
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const uint32_t lo = t < 4 ? l[2 * t] : r[2 * (t - 4)];
        const uint32_t hi = t < 4 ? l[2 * t + 1] : r[2 * (t - 4) + 1];
        uint32_t vlo, vhi;
        prefixed_word(carry, lo, hi, vlo, vhi);
        PlainRep::set_word(A[t], B[t], vlo, vhi);
    }
    PlainRep::set_word(A[8], B[8], (carry >> 24) | (uint32_t(kDomain) << 8), 0u);
    B[kRate / 8 - 1] ^= 0x80000000u;
}

// Stack of subtree digests: sizes are distinct powers of two (the binary
// digits of the leaves seen so far), so 40 entries cover trees below 2^39.
constexpr int kStackDepth = 40;

// Tree t = leaves [t*L, (t+1)*L) of leaf_bytes each.  Leaves are hashed in
// order; equal-size subtrees on the stack merge at once, and the remaining
// ones merge right to left at the end, which builds exactly the level-by-
// level tree with odd nodes carried up.  Every leaf block and every node is
// one pass of a single loop around one permutation call site, so the kernel
// holds one copy of the permutation's code.
template <bool A8>
__global__ void __launch_bounds__(kThreads)
    k_merkle_many(const uint8_t *__restrict__ buf, uint64_t n_trees, uint64_t leaves_per_tree, uint64_t leaf_bytes,
                  uint8_t *__restrict__ roots) {
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t vlen = leaf_bytes + 1;
    const uint64_t nfull = vlen / kRate;
    const uint32_t rem = uint32_t(vlen - nfull * kRate);
    enum Mode { kLeaf, kMerge, kFold };
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n_trees; t += step) {
        uint32_t stack[kStackDepth][8];
        uint64_t size[kStackDepth];
        int top = 0;
        uint32_t cur[8];  // the digest being merged or folded
        uint32_t A[25], B[25];
        uint64_t leaf = 0, blk = 0, sz = 0;
        uint32_t carry = 0;
        int j = 0;  // fold position
        Mode mode = kLeaf;
        const uint8_t *first_leaf = buf + t * leaves_per_tree * leaf_bytes;
        for (;;) {
            if (mode == kLeaf) {
                const uint8_t *p = first_leaf + leaf * leaf_bytes;
                if (blk == 0) {
#pragma unroll
                    for (int k = 0; k < 25; ++k) A[k] = B[k] = 0;
                    carry = 0x00u << 24;  // leaf prefix byte
                }
                if constexpr (A8) absorb_leaf_block_a8(A, B, p, blk, nfull, rem, leaf_bytes / 8, carry);
                else absorb_leaf_block_any(A, B, p, blk, nfull, rem);
            } else {
                uint32_t l[8];
                const int li = mode == kMerge ? top - 1 : j;
#pragma unroll
                for (int k = 0; k < 8; ++k) l[k] = stack[li][k];
                load_node_block(A, B, l, cur);
            }
            PlainRep::permute<false>(A, B);
            if (mode == kLeaf && blk < nfull) {
                ++blk;
                continue;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                cur[2 * k] = A[k];
                cur[2 * k + 1] = B[k];
            }
            if (mode == kFold) {
                if (j == 0) break;  // cur is the root
                --j;
                continue;
            }
            if (mode == kLeaf) {
                sz = 1;
                blk = 0;
                ++leaf;
            } else {  // kMerge: cur = node(stack[top - 1], cur)
                sz *= 2;
                --top;
            }
            if (top > 0 && size[top - 1] == sz) {
                mode = kMerge;
                continue;
            }
            if (leaf < leaves_per_tree) {
#pragma unroll
                for (int k = 0; k < 8; ++k) stack[top][k] = cur[k];
                size[top++] = sz;
                mode = kLeaf;
                continue;
            }
            // All leaves are in: fold the stack's subtrees into cur, right to left.
            if (top == 0) break;  // cur is the root
            j = top - 1;
            mode = kFold;
        }
        uint4 *o = reinterpret_cast<uint4 *>(roots + 32 * t);
        o[0] = make_uint4(cur[0], cur[1], cur[2], cur[3]);
        o[1] = make_uint4(cur[4], cur[5], cur[6], cur[7]);
    }
}

}  // namespace

uint64_t merkle_nodes(uint64_t n_leaves) {
    if (n_leaves == 0) return 0;
    uint64_t total = 0, n = n_leaves;
    for (;;) {
        total += n;
        if (n == 1) break;
        n = (n + 1) / 2;
    }
    return total;
}

namespace {

int launch_leaves(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes, uint8_t *out, cudaStream_t stream) {
    if (n_leaves == 0) return KB_OK;
    const bool a8 = ((reinterpret_cast<uintptr_t>(buf) | leaf_bytes) & 7) == 0 && leaf_bytes > 0;
    // One thread per leaf and as many blocks as that takes: a leaf is a long
    // chain of permutations, and the block scheduler's dynamic placement
    // balances the last wave better than a fixed grid-stride split (measured
    // 5% faster on 4 GiB of 8 KiB leaves).
    const uint64_t grid = std::min<uint64_t>((n_leaves + kThreads - 1) / kThreads, uint64_t(INT32_MAX));
    if (a8) k_merkle_leaves_a8<<<unsigned(grid), kThreads, 0, stream>>>(buf, n_leaves, leaf_bytes, out);
    else k_merkle_leaves_any<<<unsigned(grid), kThreads, 0, stream>>>(buf, n_leaves, leaf_bytes, out);
    return cuda_status(cudaGetLastError());
}

// Every level above the n leaf digests at `nodes`, written after them.
int launch_upper_levels(uint8_t *nodes, uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    uint8_t *level = nodes;
    while (n > kTopCount) {
        uint8_t *next = level + 32 * n;
        const uint64_t parents = n / 2 + (n & 1);
        if (parents <= kLaneParents) {
            const uint64_t blocks = (parents + kThreads / 32 - 1) / (kThreads / 32);
            k_merkle_level_lanes<<<unsigned(blocks), kThreads, 0, stream>>>(level, n, next);
        } else {
            const uint64_t grid =
                persistent_grid(reinterpret_cast<const void *>(&k_merkle_level), kThreads, 0, parents, dev);
            k_merkle_level<<<unsigned(grid), kThreads, 0, stream>>>(level, n, next);
        }
        if (cudaGetLastError() != cudaSuccess) return KB_ERR_CUDA;
        level = next;
        n = parents;
    }
    if (n > 1) {
        k_merkle_top<<<1, kTopThreads, 0, stream>>>(level, n);
        if (cudaGetLastError() != cudaSuccess) return KB_ERR_CUDA;
    }
    return KB_OK;
}

}  // namespace

int launch_merkle_levels(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes, uint8_t *nodes,
                         cudaStream_t stream, const DeviceInfo &dev) {
    int rc = launch_leaves(buf, n_leaves, leaf_bytes, nodes, stream);
    if (rc != KB_OK) return rc;
    return launch_upper_levels(nodes, n_leaves, stream, dev);
}

int launch_merkle_many(const uint8_t *buf, uint64_t n_trees, uint64_t leaves_per_tree, uint64_t leaf_bytes,
                       uint8_t *roots, cudaStream_t stream, const DeviceInfo & /*dev*/) {
    // Leaves on 8-byte boundaries (buffer and leaf size) take the aligned
    // 8-byte loads; others the byte-exact reads.
    const bool a8 = ((reinterpret_cast<uintptr_t>(buf) | leaf_bytes) & 7) == 0;
    // One thread per tree and as many blocks as that takes: the block
    // scheduler balances the last wave, where a grid-stride split would give
    // some threads one tree more than others.
    const uint64_t grid = std::min<uint64_t>((n_trees + kThreads - 1) / kThreads, uint64_t(INT32_MAX));
    if (a8)
        k_merkle_many<true><<<unsigned(grid), kThreads, 0, stream>>>(buf, n_trees, leaves_per_tree, leaf_bytes,
                                                                      roots);
    else
        k_merkle_many<false><<<unsigned(grid), kThreads, 0, stream>>>(buf, n_trees, leaves_per_tree, leaf_bytes,
                                                                       roots);
    return cuda_status(cudaGetLastError());
}

uint64_t merkle_message_leaves(uint64_t len, uint64_t chunk_bytes) {
    return len == 0 ? 1 : (len + chunk_bytes - 1) / chunk_bytes;
}

int launch_merkle_message(const uint8_t *msg, uint64_t len, uint64_t chunk_bytes, uint8_t *nodes,
                          cudaStream_t stream, const DeviceInfo &dev) {
    const uint64_t n = merkle_message_leaves(len, chunk_bytes);
    const uint64_t full = len / chunk_bytes;
    int rc = launch_leaves(msg, full, chunk_bytes, nodes, stream);
    if (rc != KB_OK) return rc;
    if (full < n) {  // the short (or empty) last chunk
        const uint64_t last = len - full * chunk_bytes;
        k_merkle_leaves_any<<<1, kThreads, 0, stream>>>(msg + full * chunk_bytes, 1, last, nodes + 32 * full);
        if (cudaGetLastError() != cudaSuccess) return KB_ERR_CUDA;
    }
    return launch_upper_levels(nodes, n, stream, dev);
}

}  // namespace kb
