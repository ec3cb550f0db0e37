/*
 * keccak_ref.c -- plain, slow CPU oracle for the batch SHA-3 library.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * What it computes: the Keccak-p permutations, the sponge construction and the
 * six SHA-3 functions exactly as the paper restates them (Section 3: Table 1,
 * Eq. 1-18), read against FIPS 202, which the paper cites as the standard.
 * The state is kept as a string of bits, one bit per byte, and every step
 * mapping is written per bit from its defining equation, so that a reader can
 * hold each line against the paper.  Where the paper's equations are garbled
 * the code follows FIPS 202 and says so at the spot:
 *   - rho (Eq. 5): FIPS 202 Algorithm 2 (rotate left, lane (0,0) untouched,
 *     the (x,y) walk updates the lane coordinates, not the destination);
 *   - pad10*1 (Eq. 11): j = (-m-2) mod x, FIPS 202 Algorithm 9;
 *   - iota (Eq. 8, the paper's "zeta"): j runs over 0..l inclusive;
 *   - rc: the LFSR of FIPS 202 Algorithm 5 (the paper names it only);
 *   - bit order: FIPS 202 Appendix B (bits LSB-first inside each byte).
 * No byte-level shortcut (domain bytes, lane words) appears here: messages are
 * turned into bit strings, suffix and padding bits are appended as bits, and
 * the output bits are packed back into bytes.
 *
 * Parity pins for this file live in tests/test_oracle_*.py (hashlib digests,
 * LFSR and rho regeneration, Keccak-f[25] brute-force bijectivity, step-wise
 * bijectivity of Keccak-f[50], sponge prefix and incremental-absorb identities,
 * a second recursive Merkle definition).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "keccak_ref.h"

/* ---------------------------------------------------------------------------
 * Section 3.1, Table 1: b = 25w, l = log2(w).
 * ------------------------------------------------------------------------- */
static int width_to_l(int w) {
    int l = 0;
    while ((1 << l) < w) ++l;
    return ((1 << l) == w && l <= 6) ? l : -1;
}

/* Eq. 1: A[x,y,z] = S[w(5y+x)+z], 0 <= x,y < 5, 0 <= z < w (the paper prints
 * the bounds as "<= 5"/"<= w"; the array has 5 x 5 x w entries). */
#define A_AT(S, w, x, y, z) ((S)[(size_t)(w) * (5 * (y) + (x)) + (z)])

static int mod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }

/* Definition 1, Eq. 2-4: theta. */
void oracle_theta(int w, uint8_t *S) {
    uint8_t C[5][64], D[5][64], Out[1600];
    for (int x = 0; x < 5; ++x)
        for (int z = 0; z < w; ++z)
            C[x][z] = A_AT(S, w, x, 0, z) ^ A_AT(S, w, x, 1, z) ^ A_AT(S, w, x, 2, z) ^
                      A_AT(S, w, x, 3, z) ^ A_AT(S, w, x, 4, z);
    for (int x = 0; x < 5; ++x)
        for (int z = 0; z < w; ++z)
            D[x][z] = C[mod(x - 1, 5)][z] ^ C[mod(x + 1, 5)][mod(z - 1, w)];
    for (int x = 0; x < 5; ++x)
        for (int y = 0; y < 5; ++y)
            for (int z = 0; z < w; ++z)
                A_AT(Out, w, x, y, z) = A_AT(S, w, x, y, z) ^ D[x][z];
    memcpy(S, Out, (size_t)25 * w);
}

/* Definition 2, Eq. 5, read as FIPS 202 Algorithm 2: lane (0,0) is copied;
 * starting from (x,y) = (1,0), for t = 0..23 the lane (x,y) is rotated so that
 * A'[x,y,z] = A[x,y,(z-(t+1)(t+2)/2) mod w], then (x,y) <- (y,(2x+3y) mod 5).
 * (The paper's printed form writes the walk update into the destination
 * index; that would move lanes, which is pi's job.) */
void oracle_rho(int w, uint8_t *S) {
    uint8_t Out[1600];
    for (int z = 0; z < w; ++z) A_AT(Out, w, 0, 0, z) = A_AT(S, w, 0, 0, z);
    int x = 1, y = 0;
    for (int t = 0; t < 24; ++t) {
        int off = (t + 1) * (t + 2) / 2;
        for (int z = 0; z < w; ++z)
            A_AT(Out, w, x, y, z) = A_AT(S, w, x, y, mod(z - off, w));
        int nx = y, ny = mod(2 * x + 3 * y, 5);
        x = nx; y = ny;
    }
    memcpy(S, Out, (size_t)25 * w);
}

/* Definition 3, Eq. 6: pi. */
void oracle_pi(int w, uint8_t *S) {
    uint8_t Out[1600];
    for (int x = 0; x < 5; ++x)
        for (int y = 0; y < 5; ++y)
            for (int z = 0; z < w; ++z)
                A_AT(Out, w, x, y, z) = A_AT(S, w, mod(x + 3 * y, 5), x, z);
    memcpy(S, Out, (size_t)25 * w);
}

/* Definition 4, Eq. 7: chi. The product of bits is the Boolean AND. */
void oracle_chi(int w, uint8_t *S) {
    uint8_t Out[1600];
    for (int x = 0; x < 5; ++x)
        for (int y = 0; y < 5; ++y)
            for (int z = 0; z < w; ++z)
                A_AT(Out, w, x, y, z) =
                    A_AT(S, w, x, y, z) ^
                    (A_AT(S, w, mod(x + 2, 5), y, z) & (1 ^ A_AT(S, w, mod(x + 1, 5), y, z)));
    memcpy(S, Out, (size_t)25 * w);
}

/* The LFSR function rc(t) the paper names under Definition 5 without defining
 * it: FIPS 202 Algorithm 5.  R is an 8-bit register written R[0..7]; each
 * step prepends a 0 (making 9 bits), feeds R[8] back into bits 0, 4, 5, 6,
 * and truncates to 8 bits.  The output is R[0]. */
int oracle_rc_bit(long t) {
    long tm = t % 255;
    if (tm < 0) tm += 255;
    if (tm == 0) return 1;
    int R[9] = {1, 0, 0, 0, 0, 0, 0, 0, 0};
    for (long i = 1; i <= tm; ++i) {
        for (int k = 8; k >= 1; --k) R[k] = R[k - 1];  /* R = 0 || R */
        R[0] = 0;
        R[0] ^= R[8];
        R[4] ^= R[8];
        R[5] ^= R[8];
        R[6] ^= R[8];
        R[8] = 0;                                       /* Trunc_8 */
    }
    return R[0];
}

/* Definition 5, Eq. 8: RC[2^j - 1] = rc(j + 7 i_r) for 0 <= j <= l (the l+1
 * bits the same paragraph describes; the printed "j < l" drops one), all
 * other bits of RC zero.  Returned as an integer whose bit z is RC[z]. */
uint64_t oracle_round_constant(int l, int ir) {
    uint64_t rc = 0;
    for (int j = 0; j <= l; ++j)
        if (oracle_rc_bit((long)j + 7L * ir)) rc |= (uint64_t)1 << ((1 << j) - 1);
    return rc;
}

/* Definition 5, Eq. 9: iota (the paper's "zeta"). */
void oracle_iota(int w, int ir, uint8_t *S) {
    int l = width_to_l(w);
    uint64_t rc = oracle_round_constant(l, ir);
    for (int z = 0; z < w; ++z) A_AT(S, w, 0, 0, z) ^= (uint8_t)((rc >> z) & 1);
}

/* Eq. 10: Rnd(A, i_r) = iota(chi(pi(rho(theta(A)))), i_r). */
void oracle_rnd(int w, int ir, uint8_t *S) {
    oracle_theta(w, S);
    oracle_rho(w, S);
    oracle_pi(w, S);
    oracle_chi(w, S);
    oracle_iota(w, ir, S);
}

/* Keccak-p[b, n_r]: n_r iterations of Rnd with i_r running over the last n_r
 * of the 12+2l round indices (FIPS 202 Algorithm 7; the paper states only
 * "n_r iterations").  S holds b bits, one per byte, in the Eq. 1 order. */
int oracle_keccak_p(int b, int nr, uint8_t *S) {
    if (b % 25 != 0 || nr < 0) return ORACLE_ERR_INVALID;
    int w = b / 25, l = width_to_l(w);
    if (l < 0) return ORACLE_ERR_INVALID;
    for (int ir = 12 + 2 * l - nr; ir <= 12 + 2 * l - 1; ++ir) oracle_rnd(w, ir, S);
    return ORACLE_OK;
}

/* Returns the rho offset the Algorithm 2 walk gives lane (x,y), mod w. */
int oracle_rho_offset(int w, int x, int y) {
    if (x == 0 && y == 0) return 0;
    int cx = 1, cy = 0;
    for (int t = 0; t < 24; ++t) {
        if (cx == x && cy == y) return mod((t + 1) * (t + 2) / 2, w);
        int nx = cy, ny = mod(2 * cx + 3 * cy, 5);
        cx = nx; cy = ny;
    }
    return -1;
}

/* Eq. 11 read as FIPS 202 Algorithm 9: pad10*1(x, m) = 1 || 0^j || 1 with
 * j = (-m-2) mod x, so that m + |pad| is a positive multiple of x.  Writes
 * the padding bits into P and returns their count. */
static size_t pad10star1(size_t x, size_t m, uint8_t *P) {
    size_t j = (x - ((m + 2) % x)) % x;
    P[0] = 1;
    memset(P + 1, 0, j);
    P[j + 1] = 1;
    return j + 2;
}

/* Section 3.2 sponge, Sponge[Keccak-p[1600,24], pad10*1, r](N, d), in the
 * steps of FIPS 202 Algorithm 8 (the paper gives only the prose): pad N,
 * absorb each r-bit block P_i as S = f(S xor (P_i || 0^c)), then squeeze
 * Z = Z || Trunc_r(S), applying f between output blocks, until d bits. */
static int sponge_1600(size_t r, const uint8_t *N, size_t n_bits, size_t d_bits, uint8_t *Z) {
    const int b = 1600;
    size_t plen = n_bits + r + 2;
    uint8_t *P = (uint8_t *)malloc(plen);
    if (!P) return ORACLE_ERR_NOMEM;
    memcpy(P, N, n_bits);
    plen = n_bits + pad10star1(r, n_bits, P + n_bits);
    uint8_t S[1600];
    memset(S, 0, sizeof S);
    for (size_t i = 0; i < plen / r; ++i) {
        for (size_t k = 0; k < r; ++k) S[k] ^= P[i * r + k];   /* P_i || 0^c */
        oracle_keccak_p(b, 24, S);
    }
    free(P);
    size_t have = 0;
    for (;;) {
        size_t take = (d_bits - have < r) ? d_bits - have : r;
        memcpy(Z + have, S, take);
        have += take;
        if (have >= d_bits) break;
        oracle_keccak_p(b, 24, S);
    }
    return ORACLE_OK;
}

/* Eq. 12: Keccak[c](N, d) = Sponge[Keccak-p[1600,24], pad10*1, 1600-c](N, d). */
int oracle_keccak_c(int c, const uint8_t *N, size_t n_bits, size_t d_bits, uint8_t *Z) {
    if (c <= 0 || c >= 1600) return ORACLE_ERR_INVALID;
    return sponge_1600((size_t)(1600 - c), N, n_bits, d_bits, Z);
}

/* Eq. 13-18 and the variant numbering the library uses:
 * 0..3 SHA3-224/256/384/512 = Keccak[2d](M || 01, d);
 * 4, 5 SHAKE128/256 = Keccak[256 / 512](M || 1111, d).
 * c = 2d holds only for the four hashes (the paper states it generally). */
static int variant_params(int variant, int *c, int *d_bytes, int *suffix_len) {
    static const int caps[6] = {448, 512, 768, 1024, 256, 512};
    static const int dlen[6] = {28, 32, 48, 64, -1, -1};
    if (variant < 0 || variant > 5) return ORACLE_ERR_INVALID;
    *c = caps[variant];
    *d_bytes = dlen[variant];
    *suffix_len = variant < 4 ? 2 : 4;
    return ORACLE_OK;
}

/* FIPS 202 Appendix B.1: byte i, bit j (LSB first) is string bit 8i+j. */
static void bytes_to_bits(const uint8_t *M, size_t len, uint8_t *S) {
    for (size_t i = 0; i < len; ++i)
        for (int j = 0; j < 8; ++j) S[8 * i + j] = (M[i] >> j) & 1;
}

static void bits_to_bytes(const uint8_t *S, size_t nbytes, uint8_t *M) {
    for (size_t i = 0; i < nbytes; ++i) {
        uint8_t v = 0;
        for (int j = 0; j < 8; ++j) v |= (uint8_t)(S[8 * i + j] << j);
        M[i] = v;
    }
}

/* The suffix bit strings of Eq. 13-18, in string order: "01" and "1111". */
static void append_suffix(int variant, uint8_t *N) {
    if (variant < 4) { N[0] = 0; N[1] = 1; }
    else { N[0] = 1; N[1] = 1; N[2] = 1; N[3] = 1; }
}

int oracle_hash(int variant, const uint8_t *msg, size_t len, uint8_t *out, size_t out_len) {
    int c, d, sl;
    if (variant_params(variant, &c, &d, &sl) != ORACLE_OK) return ORACLE_ERR_INVALID;
    if (d >= 0 && out_len != (size_t)d) return ORACLE_ERR_INVALID;
    if (len > 0 && !msg) return ORACLE_ERR_INVALID;
    if (out_len == 0) return ORACLE_OK;
    if (!out) return ORACLE_ERR_INVALID;
    size_t n_bits = 8 * len + (size_t)sl;
    uint8_t *N = (uint8_t *)malloc(n_bits);
    uint8_t *Z = (uint8_t *)malloc(8 * out_len);
    if (!N || !Z) { free(N); free(Z); return ORACLE_ERR_NOMEM; }
    bytes_to_bits(msg, len, N);
    append_suffix(variant, N + 8 * len);
    int rc = oracle_keccak_c(c, N, n_bits, 8 * out_len, Z);
    if (rc == ORACLE_OK) bits_to_bytes(Z, out_len, out);
    free(N);
    free(Z);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Incremental form of the same sponge: absorb the message in pieces of any
 * size, then finish.  Blocks are absorbed as soon as r bits have arrived, so
 * it must agree with oracle_hash for every split of the message.
 * ------------------------------------------------------------------------- */
size_t oracle_inc_size(void) { return sizeof(oracle_inc); }

int oracle_inc_init(oracle_inc *st, int variant) {
    int c, d, sl;
    if (!st || variant_params(variant, &c, &d, &sl) != ORACLE_OK) return ORACLE_ERR_INVALID;
    memset(st, 0, sizeof *st);
    st->variant = variant;
    st->r_bits = 1600 - c;
    return ORACLE_OK;
}

static void inc_push_bit(oracle_inc *st, uint8_t bit) {
    st->buf[st->nbuf++] = bit;
    if (st->nbuf == (size_t)st->r_bits) {
        for (int k = 0; k < st->r_bits; ++k) st->S[k] ^= st->buf[k];
        oracle_keccak_p(1600, 24, st->S);
        st->nbuf = 0;
    }
}

int oracle_inc_absorb(oracle_inc *st, const uint8_t *msg, size_t len) {
    if (!st || (len > 0 && !msg)) return ORACLE_ERR_INVALID;
    for (size_t i = 0; i < len; ++i)
        for (int j = 0; j < 8; ++j) inc_push_bit(st, (msg[i] >> j) & 1);
    return ORACLE_OK;
}

int oracle_inc_final(oracle_inc *st, uint8_t *out, size_t out_len) {
    int c, d, sl;
    if (!st || variant_params(st->variant, &c, &d, &sl) != ORACLE_OK) return ORACLE_ERR_INVALID;
    if (d >= 0 && out_len != (size_t)d) return ORACLE_ERR_INVALID;
    uint8_t suf[4];
    append_suffix(st->variant, suf);
    for (int k = 0; k < sl; ++k) inc_push_bit(st, suf[k]);
    uint8_t pad[1600 + 2];
    size_t np = pad10star1((size_t)st->r_bits, st->nbuf, pad);
    for (size_t k = 0; k < np; ++k) inc_push_bit(st, pad[k]);
    uint8_t *Z = (uint8_t *)malloc(8 * out_len + 1);
    if (!Z) return ORACLE_ERR_NOMEM;
    size_t have = 0, d_bits = 8 * out_len;
    while (have < d_bits) {
        size_t take = (d_bits - have < (size_t)st->r_bits) ? d_bits - have : (size_t)st->r_bits;
        memcpy(Z + have, st->S, take);
        have += take;
        if (have >= d_bits) break;
        oracle_keccak_p(1600, 24, st->S);
    }
    bits_to_bytes(Z, out_len, out);
    free(Z);
    return ORACLE_OK;
}

/* ---------------------------------------------------------------------------
 * Tree mode (Section 4: digests combined pairwise up to one root).  The
 * paper fixes no node format; the library's rules are: leaf digest
 * SHA3-256(0x00 || leaf), node digest SHA3-256(0x01 || left || right), one
 * level at a time, an odd last node carried up unchanged.
 * oracle_merkle_levels writes every level (leaves first) back to back.
 * ------------------------------------------------------------------------- */
uint64_t oracle_merkle_node_count(uint64_t n_leaves) {
    uint64_t total = 0, n = n_leaves;
    if (n == 0) return 0;
    for (;;) {
        total += n;
        if (n == 1) break;
        n = (n + 1) / 2;
    }
    return total;
}

int oracle_merkle_levels(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes, uint8_t *nodes) {
    if (n_leaves == 0 || leaf_bytes == 0 || !buf || !nodes) return ORACLE_ERR_INVALID;
    uint8_t *tmp = (uint8_t *)malloc(1 + (leaf_bytes > 64 ? leaf_bytes : 64));
    if (!tmp) return ORACLE_ERR_NOMEM;
    int rc = ORACLE_OK;
    tmp[0] = 0x00;
    for (uint64_t i = 0; i < n_leaves && rc == ORACLE_OK; ++i) {
        memcpy(tmp + 1, buf + i * leaf_bytes, leaf_bytes);
        rc = oracle_hash(1, tmp, 1 + leaf_bytes, nodes + 32 * i, 32);
    }
    uint8_t *level = nodes;
    uint64_t n = n_leaves;
    while (n > 1 && rc == ORACLE_OK) {
        uint8_t *next = level + 32 * n;
        uint64_t pairs = n / 2;
        tmp[0] = 0x01;
        for (uint64_t j = 0; j < pairs && rc == ORACLE_OK; ++j) {
            memcpy(tmp + 1, level + 64 * j, 64);
            rc = oracle_hash(1, tmp, 65, next + 32 * j, 32);
        }
        if (n & 1) memcpy(next + 32 * pairs, level + 32 * (n - 1), 32);
        level = next;
        n = pairs + (n & 1);
    }
    free(tmp);
    return rc;
}

int oracle_merkle_sha3_256(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes, uint8_t root[32]) {
    if (n_leaves == 0 || leaf_bytes == 0 || !buf || !root) return ORACLE_ERR_INVALID;
    uint64_t total = oracle_merkle_node_count(n_leaves);
    uint8_t *nodes = (uint8_t *)malloc(32 * total);
    if (!nodes) return ORACLE_ERR_NOMEM;
    int rc = oracle_merkle_levels(buf, n_leaves, leaf_bytes, nodes);
    if (rc == ORACLE_OK) memcpy(root, nodes + 32 * (total - 1), 32);
    free(nodes);
    return rc;
}

/* The same tree over one message cut into chunks of chunk_bytes bytes (the
 * last chunk shorter, an empty message giving one empty leaf): the tree mode
 * applied to a single large input, which Section 1 names as the way to spread
 * one long message over parallel hardware.  Leaf and node rules as above. */
int oracle_merkle_message(const uint8_t *msg, uint64_t len, uint64_t chunk_bytes, uint8_t root[32]) {
    if (chunk_bytes == 0 || (len > 0 && !msg) || !root) return ORACLE_ERR_INVALID;
    uint64_t n = len == 0 ? 1 : (len + chunk_bytes - 1) / chunk_bytes;
    uint8_t *level = (uint8_t *)malloc(32 * n);
    uint8_t *tmp = (uint8_t *)malloc(1 + (chunk_bytes > 64 ? chunk_bytes : 64));
    if (!level || !tmp) { free(level); free(tmp); return ORACLE_ERR_NOMEM; }
    int rc = ORACLE_OK;
    tmp[0] = 0x00;
    for (uint64_t i = 0; i < n && rc == ORACLE_OK; ++i) {
        uint64_t start = i * chunk_bytes;
        uint64_t take = len - start < chunk_bytes ? len - start : chunk_bytes;
        if (len == 0) take = 0;
        if (take) memcpy(tmp + 1, msg + start, take);
        rc = oracle_hash(1, tmp, 1 + take, level + 32 * i, 32);
    }
    tmp[0] = 0x01;
    while (n > 1 && rc == ORACLE_OK) {
        uint64_t pairs = n / 2;
        for (uint64_t j = 0; j < pairs && rc == ORACLE_OK; ++j) {
            memcpy(tmp + 1, level + 64 * j, 64);
            rc = oracle_hash(1, tmp, 65, level + 32 * j, 32);
        }
        if (n & 1) memmove(level + 32 * pairs, level + 32 * (n - 1), 32);
        n = pairs + (n & 1);
    }
    if (rc == ORACLE_OK) memcpy(root, level, 32);
    free(level);
    free(tmp);
    return rc;
}
