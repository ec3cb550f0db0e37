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
// one-byte funnel shift of the leaf's aligned words), then the levels above
// (0x01 || left || right is exactly one 65-byte block at rate 136), one thread
// per parent node: one launch per level while a level has more than 16384
// parents, and above that climbing launches that reduce up to six levels
// each, the upper ones inside each warp through shuffles.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "keccak_core.cuh"
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

// Digest (eight little-endian 32-bit words) of SHA3-256(0x01 || l || r).
__device__ __forceinline__ void node_digest(const uint32_t (&l)[8], const uint32_t (&r)[8], uint32_t (&d)[8]) {
    uint32_t A[25], B[25];
    load_node_block(A, B, l, r);
    PlainRep::permute<true>(A, B);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        d[2 * k] = A[k];
        d[2 * k + 1] = B[k];
    }
}

// Levels where a permutation's latency, not the ALU pipe's throughput, sets
// the time (at most kClimbParents parents: under one warp per SM
// sub-partition), up to kClimbLevels + 1 of them in one launch.  Warp w takes
// parents [32w, 32w + 32) of the first level, one thread each; at climb step
// l, lane i (a multiple of 2^l) combines its node with that of lane
// i + 2^(l-1), fetched by a shuffle, into node (32w + i) / 2^l of the next
// level, or carries it up unchanged when it is that level's odd last node.
// The warps' ranges nest (the children of nodes [16w, 16w + 16) of a level
// are nodes [32w, 32w + 32) of the level below), so every node of every level
// is computed as the level-by-level reduction computes it, and each is
// written out.  One loop around one permutation call site covers all steps.
constexpr uint64_t kClimbParents = 16384;
constexpr int kClimbLevels = 5;

__global__ void __launch_bounds__(kThreads) k_merkle_climb(const uint8_t *in, uint64_t count, uint8_t *out, int climb) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    uint64_t cnt = count;  // nodes of the level being reduced
    const uint8_t *src = in;
    uint8_t *dst = out;
    uint32_t d[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int l = 0; l <= climb; ++l) {
        const uint64_t parents = cnt / 2 + (cnt & 1);
        uint32_t lft[8], rgt[8];
        uint64_t q;  // parent index
        bool act;
        if (l == 0) {
            q = warp * 32 + lane;
            act = q < parents;
#pragma unroll
            for (int t = 0; t < 8; ++t) lft[t] = rgt[t] = 0;
            if (act) {
                const uint4 *c = reinterpret_cast<const uint4 *>(src + 64 * q);
                const uint4 a = c[0], b = c[1];
                lft[0] = a.x, lft[1] = a.y, lft[2] = a.z, lft[3] = a.w;
                lft[4] = b.x, lft[5] = b.y, lft[6] = b.z, lft[7] = b.w;
                if (2 * q + 1 < cnt) {
                    const uint4 e = c[2], f = c[3];
                    rgt[0] = e.x, rgt[1] = e.y, rgt[2] = e.z, rgt[3] = e.w;
                    rgt[4] = f.x, rgt[5] = f.y, rgt[6] = f.z, rgt[7] = f.w;
                }
            }
        } else {
            const uint32_t step = 1u << (l - 1);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                lft[t] = d[t];
                rgt[t] = __shfl_down_sync(0xFFFFFFFFu, d[t], step);
            }
            const uint64_t c = warp * (32u >> (l - 1)) + (lane >> (l - 1));  // this lane's node: the left child
            act = (lane & (2 * step - 1)) == 0 && c < cnt;
            q = c >> 1;
        }
        if (act) {
            if (2 * q + 1 < cnt) node_digest(lft, rgt, d);
            else {
#pragma unroll
                for (int t = 0; t < 8; ++t) d[t] = lft[t];  // odd last node: carried up
            }
            uint4 *o = reinterpret_cast<uint4 *>(dst + 32 * q);
            o[0] = make_uint4(d[0], d[1], d[2], d[3]);
            o[1] = make_uint4(d[4], d[5], d[6], d[7]);
        }
        src = dst;
        dst += 32 * parents;
        cnt = parents;
    }
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

// Every level above the n leaf digests at `nodes`, written after them: one
// launch per level while a level has more than kClimbParents parents (there
// the ALU pipe's throughput sets the time), then climbing launches of up to
// kClimbLevels + 1 levels each.
int launch_upper_levels(uint8_t *nodes, uint64_t n, cudaStream_t stream, const DeviceInfo &dev) {
    uint8_t *level = nodes;
    while (n > 1) {
        const uint64_t parents = n / 2 + (n & 1);
        if (parents > kClimbParents) {
            const uint64_t grid =
                persistent_grid(reinterpret_cast<const void *>(&k_merkle_level), kThreads, 0, parents, dev);
            k_merkle_level<<<unsigned(grid), kThreads, 0, stream>>>(level, n, level + 32 * n);
            if (cudaGetLastError() != cudaSuccess) return KB_ERR_CUDA;
            level += 32 * n;
            n = parents;
            continue;
        }
        int climb = 0;
        for (uint64_t m = parents; climb < kClimbLevels && m > 1; m = m / 2 + (m & 1)) ++climb;
        const uint64_t threads = (parents + 31) / 32 * 32;
        const uint64_t blocks = (threads + kThreads - 1) / kThreads;
        k_merkle_climb<<<unsigned(blocks), kThreads, 0, stream>>>(level, n, level + 32 * n, climb);
        if (cudaGetLastError() != cudaSuccess) return KB_ERR_CUDA;
        for (int l = 0; l <= climb; ++l) {
            level += 32 * n;
            n = n / 2 + (n & 1);
        }
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
