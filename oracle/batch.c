/*
 * batch.c -- host-thread harness around the oracle (test infrastructure only).
 *
 * It adds no arithmetic of its own: each message goes through oracle_hash as
 * is, and the threads only split the message list between them.  Used by the
 * test suite for large parity checks and by the benchmark's CPU-baseline leg.
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

#include "keccak_ref.h"

typedef struct {
    const uint8_t *msgs;
    const uint64_t *offsets, *lens, *out_off;
    const uint8_t *variants;
    const uint32_t *out_lens;
    uint8_t *digests;
    uint64_t n;
    atomic_ullong next;
    atomic_int status;
} batch_job;

static void *batch_worker(void *arg) {
    batch_job *job = (batch_job *)arg;
    for (;;) {
        uint64_t i = atomic_fetch_add(&job->next, 1);
        if (i >= job->n) break;
        int rc = oracle_hash(job->variants[i], job->msgs + job->offsets[i], job->lens[i],
                             job->digests + job->out_off[i], job->out_lens[i]);
        if (rc != ORACLE_OK) {
            int expected = ORACLE_OK;
            atomic_compare_exchange_strong(&job->status, &expected, rc);
        }
    }
    return NULL;
}

int oracle_hash_batch(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                      const uint8_t *variants, const uint32_t *out_lens, uint8_t *digests,
                      uint64_t n, int nthreads) {
    if (n == 0) return ORACLE_OK;
    if (!offsets || !lens || !variants || !out_lens) return ORACLE_ERR_INVALID;
    uint64_t *out_off = (uint64_t *)malloc(sizeof(uint64_t) * n);
    if (!out_off) return ORACLE_ERR_NOMEM;
    uint64_t acc = 0;
    for (uint64_t i = 0; i < n; ++i) { out_off[i] = acc; acc += out_lens[i]; }
    batch_job job;
    job.msgs = msgs; job.offsets = offsets; job.lens = lens; job.out_off = out_off;
    job.variants = variants; job.out_lens = out_lens; job.digests = digests; job.n = n;
    atomic_init(&job.next, 0);
    atomic_init(&job.status, ORACLE_OK);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, batch_worker, &job) == 0) ++started;
    if (started == 0) batch_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(out_off);
    return atomic_load(&job.status);
}

/* Brute-force image count of Keccak-p[25, nr]: every 25-bit state, as the
 * integer whose bit k is string bit k, is permuted and its image marked in a
 * 2^25-bit map; the count of marked bits is returned. */
typedef struct {
    int nr;
    atomic_uint *bitmap;
    atomic_ullong next;
} b25_job;

static void *b25_worker(void *arg) {
    b25_job *job = (b25_job *)arg;
    const uint64_t total = (uint64_t)1 << 25, chunk = 1 << 14;
    for (;;) {
        uint64_t start = atomic_fetch_add(&job->next, chunk);
        if (start >= total) break;
        for (uint64_t v = start; v < start + chunk; ++v) {
            uint8_t S[25];
            for (int k = 0; k < 25; ++k) S[k] = (v >> k) & 1;
            oracle_keccak_p(25, job->nr, S);
            uint32_t img = 0;
            for (int k = 0; k < 25; ++k) img |= (uint32_t)S[k] << k;
            atomic_fetch_or(&job->bitmap[img >> 5], 1u << (img & 31));
        }
    }
    return NULL;
}

int64_t oracle_count_images_b25(int nr, int nthreads) {
    const uint64_t words = ((uint64_t)1 << 25) / 32;
    atomic_uint *bitmap = (atomic_uint *)calloc(words, sizeof(atomic_uint));
    if (!bitmap) return -1;
    b25_job job;
    job.nr = nr;
    job.bitmap = bitmap;
    atomic_init(&job.next, 0);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, b25_worker, &job) == 0) ++started;
    if (started == 0) b25_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    int64_t count = 0;
    for (uint64_t i = 0; i < words; ++i) count += __builtin_popcount(atomic_load(&bitmap[i]));
    free(bitmap);
    return count;
}
