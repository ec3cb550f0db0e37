/*
 * keccak_ref.h -- interface of the CPU oracle (test infrastructure only).
 *
 * Bit strings are arrays of uint8_t holding one bit (0 or 1) per element, in
 * string order; a Keccak-p state of width b is such a string of b bits laid
 * out as A[x,y,z] = S[w(5y+x)+z] (the paper's Eq. 1).  Byte strings follow
 * FIPS 202 Appendix B: byte i holds string bits 8i..8i+7, least significant
 * bit first.
 *
 * Variant numbers: 0 SHA3-224, 1 SHA3-256, 2 SHA3-384, 3 SHA3-512,
 * 4 SHAKE128, 5 SHAKE256.
 */
#ifndef KECCAK_REF_H
#define KECCAK_REF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_OK = 0, ORACLE_ERR_INVALID = -1, ORACLE_ERR_NOMEM = -2 };

/* Step mappings on a state of width b = 25w (w in 1..64), in place. */
void oracle_theta(int w, uint8_t *S);
void oracle_rho(int w, uint8_t *S);
void oracle_pi(int w, uint8_t *S);
void oracle_chi(int w, uint8_t *S);
void oracle_iota(int w, int ir, uint8_t *S);
void oracle_rnd(int w, int ir, uint8_t *S);
int oracle_keccak_p(int b, int nr, uint8_t *S);

/* rc(t) bit, the round-constant lane for (l, i_r) with bit z = RC[z], and the
 * rho offset of lane (x,y) mod w. */
int oracle_rc_bit(long t);
uint64_t oracle_round_constant(int l, int ir);
int oracle_rho_offset(int w, int x, int y);

/* Keccak[c](N, d) on bit strings; Z receives d_bits bits. */
int oracle_keccak_c(int c, const uint8_t *N, size_t n_bits, size_t d_bits, uint8_t *Z);

/* SHA3-224/256/384/512 (out_len must equal the digest size) and
 * SHAKE128/256 (any out_len) of a byte string. */
int oracle_hash(int variant, const uint8_t *msg, size_t len, uint8_t *out, size_t out_len);

/* Incremental absorb: init, any number of absorb calls, one final. */
typedef struct {
    int variant;
    int r_bits;
    uint8_t S[1600];
    uint8_t buf[1600];
    size_t nbuf;
} oracle_inc;
size_t oracle_inc_size(void);
int oracle_inc_init(oracle_inc *st, int variant);
int oracle_inc_absorb(oracle_inc *st, const uint8_t *msg, size_t len);
int oracle_inc_final(oracle_inc *st, uint8_t *out, size_t out_len);

/* Merkle tree over n_leaves leaves of leaf_bytes bytes each. */
uint64_t oracle_merkle_node_count(uint64_t n_leaves);
int oracle_merkle_levels(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes, uint8_t *nodes);
int oracle_merkle_sha3_256(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes, uint8_t root[32]);
/* The tree of one message cut into chunk_bytes chunks (last one shorter). */
int oracle_merkle_message(const uint8_t *msg, uint64_t len, uint64_t chunk_bytes, uint8_t root[32]);

/* Batch harness (batch.c): hashes n messages on nthreads host threads.
 * Message i is msgs[offsets[i] .. offsets[i]+lens[i]), its variant
 * variants[i], its output out_lens[i] bytes written at the exclusive prefix
 * sum of out_lens.  Returns ORACLE_OK or the first error. */
int oracle_hash_batch(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                      const uint8_t *variants, const uint32_t *out_lens, uint8_t *digests,
                      uint64_t n, int nthreads);

/* Brute force for tests: applies Keccak-p[25, nr] to all 2^25 states on
 * nthreads threads and returns how many distinct outputs appeared. */
int64_t oracle_count_images_b25(int nr, int nthreads);

#ifdef __cplusplus
}
#endif

#endif
