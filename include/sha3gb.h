/*
 * sha3gb.h -- C ABI of the batch SHA-3 library for NVIDIA GB300 (sm_103a).
 *
 * The library hashes many independent messages at once: the batch mode of
 * Section 4 of "GPU Accelerated Keccak (SHA3) Algorithm" (Wang & Chu), with
 * one Keccak[c] sponge per message (Section 3.2, Eq. 12) for the six
 * functions of Eq. 13-18, bit-exact to FIPS 202.  Tree mode (Section 4, named
 * there as future work) is offered as a binary Merkle root.
 *
 * Conventions for every entry point below:
 *  - Unless marked "host", pointer arguments are CUDA device pointers
 *    (memory on the current device, e.g. allocated by PyTorch).  The caller
 *    owns them; the library never frees them.
 *  - `stream` is a cudaStream_t handle passed as void*; NULL means the legacy
 *    default stream.  Calls are stream-ordered and return once the work is
 *    enqueued, unless stated otherwise.
 *  - Return value: KB_OK (0) or a negative kb_status.  Argument errors are
 *    detected on the host and returned at once, before anything is enqueued.
 *  - Byte order: messages and digests are byte strings as in FIPS 202
 *    Appendix B (bits LSB-first inside each byte).  Only whole-byte messages
 *    are accepted.
 *  - Scratch: the library may allocate internal device scratch on first use
 *    and cache it per device; keccak_release() frees it.
 */
#ifndef SHA3GB_H
#define SHA3GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Variant numbers (Eq. 13-18).  Rate r = 1600 - c bits:
 *   0 SHA3-224  c=448   r=144 B  digest 28 B
 *   1 SHA3-256  c=512   r=136 B  digest 32 B
 *   2 SHA3-384  c=768   r=104 B  digest 48 B
 *   3 SHA3-512  c=1024  r=72 B   digest 64 B
 *   4 SHAKE128  c=256   r=168 B  any output length
 *   5 SHAKE256  c=512   r=136 B  any output length */
typedef enum {
    KB_SHA3_224 = 0,
    KB_SHA3_256 = 1,
    KB_SHA3_384 = 2,
    KB_SHA3_512 = 3,
    KB_SHAKE128 = 4,
    KB_SHAKE256 = 5
} kb_variant;

typedef enum {
    KB_OK = 0,
    KB_ERR_INVALID = -1,  /* bad argument (null pointer, unknown variant, bad size) */
    KB_ERR_NOMEM = -2,    /* internal scratch could not be allocated */
    KB_ERR_CUDA = -3,     /* a CUDA runtime call failed (launch, copy, ...) */
    KB_ERR_TIMEOUT = -4,  /* a bounded device-side wait gave up */
    KB_ERR_TOO_LARGE = -5 /* a size beyond a fixed maximum (keccak_batch_noalloc) */
} kb_status;

/* Bits of the device status word read by keccak_last_error(). */
#define KB_DEV_BAD_VARIANT 0x1u   /* a message named a variant outside 0..5 */
#define KB_DEV_BAD_OUTLEN 0x2u    /* a SHA3-x message asked for out_len != digest size */
#define KB_DEV_TIMEOUT 0x4u       /* a bounded device wait expired */

/*
 * keccak_batch_uniform -- the fixed-stride batch mode (Section 4: the input
 * split into equal parts that are hashed independently; Section 4.3 hashes
 * many same-length messages): message i is the `len` bytes at
 * msgs + i*stride, i = 0..n-1, all hashed with one variant.  Output i is
 * `out_len` bytes at digests + i*out_len.
 *   msgs     device, >= (n-1)*stride + len bytes (may be NULL when len == 0)
 *   stride   distance in bytes between message starts (any value)
 *   len      message length in bytes (same for all messages)
 *   variant  0..5 (kb_variant)
 *   out_len  digest size for variants 0..3 (28/32/48/64, anything else is
 *            KB_ERR_INVALID); any value >= 0 for SHAKE
 *   digests  device, n*out_len bytes
 * n == 0 is a no-op returning KB_OK.  Reads touch only the 8-byte-aligned
 * words that hold message bytes.
 */
int keccak_batch_uniform(const uint8_t *msgs, uint64_t stride, uint64_t len, int variant,
                         uint32_t out_len, uint8_t *digests, uint64_t n, void *stream);

/*
 * keccak_batch -- the ragged batch mode: n independent messages of any
 * lengths and any mix of the six variants in one call (Section 4 batch mode,
 * generalised from the paper's equal-length messages of Section 4.3).
 *   msgs      device byte buffer holding all messages
 *   offsets   device uint64[n]: message i starts at msgs + offsets[i]
 *   lens      device uint64[n]: length of message i in bytes
 *   variant   device uint8[n]: kb_variant of message i
 *   out_lens  device uint32[n]: output bytes of message i (must equal the
 *             digest size for variants 0..3)
 *   digests   device: output i is written at byte exclusive_scan(out_lens)[i]
 *             (outputs packed back to back in message order)
 *   n         number of messages, at most 2^32 - 1; 0 is a no-op
 * Per-message errors (a variant outside 0..5, a SHA3-x out_len that is not
 * the digest size) cannot be seen on the host without a sync: those messages
 * are skipped (their output bytes are left untouched) and a bit is set in the
 * device status word (see keccak_last_error).  Uses cached internal scratch
 * of 12 bytes per message plus a 46 KiB work-queue descriptor.  The schedule
 * (KB_TUNE_RAGGED_SCHEDULE) changes only the order of the work, never a byte
 * of the output.
 */
int keccak_batch(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                 const uint8_t *variant, const uint32_t *out_lens, uint8_t *digests,
                 uint64_t n, void *stream);

/*
 * keccak_batch_autotune -- the autotuner of the ragged schedule: hashes the
 * given batch (same arguments and outputs as keccak_batch) once per candidate
 * configuration of the persistent queue (register budget x blocks per SM x
 * staging of message blocks, then threads per message: one thread for every
 * message, or one warp for each of the K costliest), checks that every
 * candidate writes the same bytes as the first, and records the fastest for
 * this device and this batch size class (n rounded down to a power of two);
 * later keccak_batch calls of that class use it.  Synchronous.  The chosen
 * register budget, blocks per SM and its time in ms are written to the HOST
 * pointers when they are not NULL (keccak_batch_autotune_ex reports every
 * dimension).  Allocates a temporary device copy of the outputs.
 * Environment, read by the library:
 *   SHA3GB_TUNE_CACHE  a file path: configurations the autotuner finds are
 *     written there and read back by later processes on the same kind of GPU.
 *     JSON Lines, one object per GPU name, SM count and size class
 *     floor(log2 n): {"gpu": "...", "sms": S, "size_class": C,
 *     "min_blocks": M, "blocks_per_sm": B}.  Unreadable files and lines that
 *     do not parse are ignored.
 *   SHA3GB_TUNE  "off": keccak_batch ignores tuned configurations; "full":
 *     keccak_batch tunes a size class the first time it sees it (that call
 *     is then synchronous and allocates as keccak_batch_autotune does, and
 *     not inside stream capture); "cached" or unset: configurations found by
 *     keccak_batch_autotune or read from the file are used.
 */
int keccak_batch_autotune(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                          const uint8_t *variant, const uint32_t *out_lens, uint8_t *digests, uint64_t n,
                          void *stream, int64_t *chosen_min_blocks, int64_t *chosen_blocks_per_sm, float *ms);

/*
 * One configuration of keccak_batch's queue schedule (Section 4.1's choice of
 * granularity, made per batch by the autotuner):
 *   min_blocks     register budget: blocks of 128 threads per SM the kernel
 *                  is compiled for (2, 3, 4, 5, 6 or 8)
 *   blocks_per_sm  blocks per SM of the persistent launch (0: as many as fit)
 *   staging        KB_QUEUE_STAGING_DIRECT, _DIRECT_LOOPED, _ASYNC or _REGS
 *                  (below)
 *   warp_messages  threads per message: the warp_messages costliest messages
 *                  run one warp (32 threads) each, the rest one thread each;
 *                  0 = one thread for every message
 *   ms             keccak_batch_autotune_ex: time of the chosen configuration
 *                  on the tuned batch; 0 elsewhere
 */
typedef struct kb_queue_config {
    int64_t min_blocks;
    int64_t blocks_per_sm;
    int64_t staging;
    int64_t warp_messages;
    float ms;
} kb_queue_config;

/* keccak_batch_autotune with every chosen dimension written to *chosen (HOST,
 * may be NULL). */
int keccak_batch_autotune_ex(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                             const uint8_t *variant, const uint32_t *out_lens, uint8_t *digests, uint64_t n,
                             void *stream, kb_queue_config *chosen);

/* The whole configuration keccak_batch would use for n messages on the
 * current device (as keccak_tuned_config), written to *cfg (HOST). */
int keccak_tuned_config_ex(uint64_t n, kb_queue_config *cfg);

/*
 * keccak_tuned_config -- the configuration keccak_batch's queue schedule
 * would use for a batch of n messages on the current device, after the
 * tuning knobs, the tuned configurations and the cache file: the register
 * budget (blocks per SM the kernel is compiled for) and the blocks per SM of
 * the launch (0: as many as fit), written to the HOST pointers when not NULL.
 * Returns KB_OK, or KB_ERR_CUDA when no device can be used.
 */
int keccak_tuned_config(uint64_t n, int64_t *min_blocks, int64_t *blocks_per_sm);

/*
 * keccak_batch_noalloc -- keccak_batch for callers that cannot allocate
 * device memory.  The paper has no counterpart: it is a deployment variant of
 * the ragged batch entry point above.  keccak_batch allocates its scratch (the
 * work queue's control block, the digest offsets and the work order) with
 * cudaMalloc on first use and whenever a larger batch arrives; a serving
 * process that reserves all device memory up front, a plugin or real-time
 * host where cudaMalloc (which can synchronise the whole device) is not
 * allowed, or code that must know its footprint in advance cannot accept
 * that.  This entry point runs keccak_batch's cost-bucketed queue (the same
 * kernels, in the built-in configuration with one thread per message,
 * launched directly rather than from a cached graph) with the scratch in a
 * fixed device array compiled into the library, of KB_NOALLOC_SCRATCH_BYTES
 * (about 814 KiB: a 256-byte status word, the 46,336-byte control block and
 * 12 bytes per message plus the scan's tile sums for KB_NOALLOC_MAX_MESSAGES
 * messages), which every GPU that loads the library holds until the process
 * exits.  It never calls cudaMalloc or cudaFree.
 *   Arguments and output layout are those of keccak_batch.
 *   n > KB_NOALLOC_MAX_MESSAGES returns KB_ERR_TOO_LARGE and does nothing.
 *   The first call in each CUDA context looks up the array's address
 *   (cudaGetSymbolAddress) with that context current; make that first call
 *   before capturing any stream into a CUDA graph.  After cudaDeviceReset,
 *   call keccak_release() before the next call so the address is looked up
 *   again.
 *   All calls share the one array and each call overwrites it: calls whose
 *   work overlaps on the GPU (several streams or host threads) race, so the
 *   caller must order them.
 *   Messages with an invalid variant or SHA3 output size are skipped (their
 *   outputs left untouched) but, unlike keccak_batch, not reported through
 *   keccak_last_error.
 */
#define KB_NOALLOC_MAX_MESSAGES 65536u
#define KB_NOALLOC_SCRATCH_BYTES 833152u
int keccak_batch_noalloc(const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                         const uint8_t *variant, const uint32_t *out_lens, uint8_t *digests,
                         uint64_t n, void *stream);

/*
 * keccak_batch_uniform_host -- keccak_batch_uniform on HOST buffers, the whole
 * job including the transfers.  Two paths, chosen by KB_TUNE_HOST_PATH:
 * staged (the messages are copied to the device, hashed and the digests
 * copied back in chunks pipelined over internal streams, with cached device
 * staging buffers, so copies overlap the hashing) or in place (on page-locked
 * buffers the kernel reads and writes the host memory directly).  With
 * KB_HOST_PATH_AUTO (the default) and page-locked buffers, the first call of
 * a size class (n rounded down to a power of two, at least 2^14 messages) on
 * a device times both paths on parts of its own batch and keeps the faster
 * for that class (keccak_host_path_for reports the decision); pageable
 * buffers always take the staged path.  Synchronous: returns when h_digests
 * holds every output.
 *   h_msgs     host, (n-1)*stride + len bytes
 *   h_digests  host, n*out_len bytes
 * Other arguments as keccak_batch_uniform.  `stream` orders the job after
 * earlier work on that stream.
 */
int keccak_batch_uniform_host(const uint8_t *h_msgs, uint64_t stride, uint64_t len, int variant,
                              uint32_t out_len, uint8_t *h_digests, uint64_t n, void *stream);

/* The path keccak_batch_uniform_host takes for n messages on the current
 * device: KB_HOST_PATH_STAGED or KB_HOST_PATH_ZERO_COPY (set by the knob or
 * decided by a trial), or KB_HOST_PATH_AUTO while undecided; KB_ERR_CUDA
 * when no device can be used. */
int keccak_host_path_for(uint64_t n);

/*
 * keccak_host_alloc -- page-locked host memory for keccak_batch_uniform_host
 * and the serving loop's message pools (cudaHostAlloc, mapped for device
 * access), populated under a preferred-node policy for the host NUMA node
 * nearest the current device (the device's cudaDevAttrHostNumaId; no
 * placement where the system reports none or refuses the policy), so that
 * neither path crosses the link between the host's CPUs.  *ptr receives the HOST address
 * (NULL on failure).  KB_ERR_INVALID for bytes == 0 or ptr == NULL,
 * KB_ERR_NOMEM when the memory cannot be mapped or page-locked.
 * keccak_host_free releases it (KB_ERR_INVALID for a pointer this library did
 * not return).  keccak_host_numa_node returns the NUMA node holding the page
 * at ptr, or -1 when the system does not say.
 */
int keccak_host_alloc(size_t bytes, void **ptr);
int keccak_host_free(void *ptr);
int keccak_host_numa_node(const void *ptr);

/*
 * Streaming (incremental) hashing of n messages at once, for messages that
 * arrive in pieces or are larger than one call should hold: the sponge of
 * Section 3.2 paused between calls.  Each message has a state of
 * KB_STATE_BYTES bytes in device memory (the caller allocates n of them, back
 * to back, 8-byte aligned): its 25 lanes, into which the bytes of the block
 * not yet complete are already XORed, and the count of those bytes.  Pieces
 * may have any length; the digest equals the one-shot hash of the
 * concatenated pieces.
 *   keccak_stream_init: states for variants[i] (device uint8[n]).
 *   keccak_stream_absorb: appends piece i (msgs + offsets[i], lens[i] bytes;
 *     lens[i] = 0 is allowed) to message i.
 *   keccak_stream_final: pads and squeezes out_lens[i] bytes (digest size for
 *     SHA3-x) into digests at the exclusive scan of out_lens, as
 *     keccak_batch does; a finalised state refuses further pieces.
 * Errors per message (unknown variant, wrong SHA3 output size, absorbing into
 * or finalising a finalised state) set KB_DEV_* bits and skip that message.
 * Stream-ordered; calls on the same states must be ordered by the caller.
 */
#define KB_STATE_BYTES 384
int keccak_stream_init(uint8_t *states, const uint8_t *variant, uint64_t n, void *stream);
int keccak_stream_absorb(uint8_t *states, const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                         uint64_t n, void *stream);
int keccak_stream_final(uint8_t *states, const uint32_t *out_lens, uint8_t *digests, uint64_t n, void *stream);
/* The first and the last step fused with a piece each, so that a message fed
 * in k pieces takes k calls: keccak_stream_init_absorb initialises the states
 * (as keccak_stream_init) and absorbs piece i into state i (as
 * keccak_stream_absorb) in one launch; keccak_stream_absorb_final absorbs
 * piece i and then finalises (as keccak_stream_final) in one launch.  Same
 * results as the separate calls. */
int keccak_stream_init_absorb(uint8_t *states, const uint8_t *variant, const uint8_t *msgs, const uint64_t *offsets,
                              const uint64_t *lens, uint64_t n, void *stream);
int keccak_stream_absorb_final(uint8_t *states, const uint8_t *msgs, const uint64_t *offsets, const uint64_t *lens,
                               const uint32_t *out_lens, uint8_t *digests, uint64_t n, void *stream);

/*
 * merkle_sha3_256 -- tree mode (Section 4: digests combined pairwise, level
 * after level, up to a single root).  The buffer holds n_leaves leaves of
 * leaf_bytes bytes each; leaf digest = SHA3-256(0x00 || leaf), node digest =
 * SHA3-256(0x01 || left || right), level by level, an odd last node carried
 * up unchanged.
 *   buf        device, n_leaves*leaf_bytes bytes
 *   root       HOST, 32 bytes, written before the call returns
 * Synchronous on `stream`.  n_leaves == 0 or leaf_bytes == 0 is
 * KB_ERR_INVALID; n_leaves == 1 gives the single leaf digest.  Uses cached
 * scratch of 32 bytes per leaf.
 */
int merkle_sha3_256(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes, uint8_t *root,
                    void *stream);

/*
 * merkle_sha3_256_many -- many small trees at once, one thread per tree: the
 * granularity Section 4.1 gives for tree mode, a thread per tree.  Tree t
 * is leaves t*leaves_per_tree .. (t+1)*leaves_per_tree - 1 of buf (leaf_bytes
 * bytes each), with the leaf/node rules of merkle_sha3_256; its root goes to
 * roots + 32*t.
 *   buf    device, n_trees*leaves_per_tree*leaf_bytes bytes, any alignment
 *   roots  device, 32*n_trees bytes, 16-byte aligned
 * Stream-ordered.  n_trees == 0 is a no-op; leaves_per_tree == 0 or >= 2^39,
 * or leaf_bytes == 0, is KB_ERR_INVALID.  Each thread works through its tree
 * sequentially, so this suits many trees of modest size; one large tree is
 * faster with merkle_sha3_256.
 */
int merkle_sha3_256_many(const uint8_t *buf, uint64_t n_trees, uint64_t leaves_per_tree, uint64_t leaf_bytes,
                         uint8_t *roots, void *stream);

/*
 * merkle_sha3_256_message -- the same tree over ONE message cut into chunks
 * of chunk_bytes bytes (the last chunk shorter; an empty message is one empty
 * leaf): tree hashing of a single large input, the way the paper's Section 1
 * names for spreading one long message over parallel hardware.  The root is
 * a different value from SHA3-256(msg): a digest of its own kind.
 *   msg    device, len bytes (may be NULL when len == 0), any alignment
 *   root   HOST, 32 bytes, written before the call returns
 * Synchronous on `stream`.  chunk_bytes == 0 is KB_ERR_INVALID.
 */
int merkle_sha3_256_message(const uint8_t *msg, uint64_t len, uint64_t chunk_bytes, uint8_t *root, void *stream);

/* Number of nodes in the tree of n_leaves leaves, all levels counted (0 for 0). */
uint64_t merkle_node_count(uint64_t n_leaves);

/*
 * merkle_sha3_256_levels -- the same tree, every level kept: nodes (device,
 * 32*merkle_node_count(n_leaves) bytes) receives the leaf digests, then each
 * level above, the root last.  Stream-ordered (asynchronous).
 */
int merkle_sha3_256_levels(const uint8_t *buf, uint64_t n_leaves, uint64_t leaf_bytes,
                           uint8_t *nodes, void *stream);

/*
 * Serving loop (continuous batching).  A server owns one device arena of
 * hbm_budget_bytes -- the admission budget: a request enters a batch only when
 * its message fits in the arena's free space, and its bytes stay resident
 * there while it is hashed.  Requests travel in two lanes by cost (number of
 * Keccak-f permutations): short requests get an eighth of the arena and
 * max_inflight streams of their own, so they never wait behind the long
 * sequential chains of large messages, which use the rest.  Whenever a lane
 * has a free stream and waiting requests, the server forms a batch of them
 * (oldest first, at most max_batch_requests and max_batch_bytes),
 * copies their messages into the arena, hashes them longest first and writes
 * each output directly to its host buffer; requests that arrive meanwhile go
 * into the next batches, which run concurrently on other streams.  Each
 * request completes as soon as its own output is written (through a
 * completion ring in host memory when the device supports native host
 * atomics, otherwise with its batch).  The paper has no serving loop; this is
 * the batch mode of Section 4 fed continuously.
 *
 * Message and output buffers are HOST memory that the device can access
 * (page-locked: cudaHostAlloc / cudaHostRegister, or torch pin_memory); they
 * must stay valid until the request completes.
 */
typedef struct kb_server kb_server;

typedef struct {
    uint64_t hbm_budget_bytes;     /* device arena size (>= 4096) */
    uint32_t max_inflight;         /* batches in flight at once per lane, 1..64 */
    uint32_t max_batch_requests;   /* requests per batch, 1..65536 */
    uint64_t max_batch_bytes;      /* message bytes per batch (capped at the budget) */
    uint64_t long_threshold_perms; /* requests costing more permutations go to the
                                      long lane (0 = 64) */
    uint32_t long_lane_kernel;     /* KB_SERVER_LONG_LANE_PARALLEL (0, default: one
                                      warp per long request) or
                                      KB_SERVER_LONG_THREAD_PER_REQUEST (1) */
    uint32_t reserved;
} kb_server_config;
#define KB_SERVER_LONG_LANE_PARALLEL 0
#define KB_SERVER_LONG_THREAD_PER_REQUEST 1

typedef struct {
    uint64_t requests;                /* completed by the replay */
    uint64_t message_bytes;           /* their message bytes */
    uint64_t batches;                 /* batches launched by the server so far */
    uint64_t max_batch_requests_seen; /* largest batch so far */
    uint64_t peak_arena_bytes;        /* peak arena bytes in use (the admitted load) */
    uint64_t rejected;                /* requests refused as larger than the budget */
    uint32_t completion_ring;         /* 1: per-request completion, 0: per batch */
    uint32_t reserved;
    double wall_s;                    /* first arrival to last completion */
    double throughput_rps, throughput_gbs;
    double lat_mean_us, lat_p50_us, lat_p90_us, lat_p99_us, lat_p999_us, lat_max_us;
    /* Where a request's latency went (p50 and p99 over the replay's requests):
     * submit lag = when the replay handed it to the server minus its
     * scheduled arrival (host side); queue wait = batch launch minus submit
     * (waiting for a stream slot or arena space); service = completion minus
     * batch launch (copy into the arena, hashing, completion). */
    double submit_lag_p50_us, submit_lag_p99_us;
    double queue_wait_p50_us, queue_wait_p99_us;
    double service_p50_us, service_p99_us;
} kb_server_stats;

/* Creates a server on the current device; NULL on error (*status says why:
 * KB_ERR_INVALID for a bad config, KB_ERR_NOMEM, KB_ERR_CUDA). */
kb_server *kb_server_create(const kb_server_config *cfg, int *status);
/* Waits for outstanding requests (up to 60 s), stops the server, frees it. */
void kb_server_destroy(kb_server *server);
/* Queues one request and returns at once; *ticket (HOST, may be NULL)
 * identifies it.  variant/out_len as in keccak_batch (out_len <= 1 MiB).
 * KB_ERR_TOO_LARGE when the message can never fit the budget. */
int kb_server_submit(kb_server *server, const uint8_t *msg, uint64_t len, int variant, uint32_t out_len,
                     uint8_t *out, uint64_t *ticket);
/* Waits until request `ticket` has completed: KB_OK, KB_ERR_TIMEOUT, or the
 * server's error status. */
int kb_server_wait(kb_server *server, uint64_t ticket, int timeout_ms);
/* Waits until every submitted request has completed (timeout_ms < 0: no limit). */
int kb_server_drain(kb_server *server, int timeout_ms);
/*
 * kb_server_replay -- drives the server with a recorded arrival schedule:
 * request i (message pool + offsets[i], lens[i] bytes, variants[i],
 * out_lens[i]) is submitted at arrival_ns[i] nanoseconds after the start
 * (non-decreasing); outputs are packed in request order into `outputs`
 * (HOST, device-visible, sum(out_lens) bytes).  Latency of a request = its
 * completion time minus its scheduled arrival.  Fills latency_ns[i] (HOST,
 * may be NULL) and *stats (HOST, may be NULL).  Synchronous; the caller must
 * not submit to the same server meanwhile.
 */
int kb_server_replay(kb_server *server, const uint8_t *pool, const uint64_t *offsets, const uint64_t *lens,
                     const uint8_t *variants, const uint32_t *out_lens, const int64_t *arrival_ns, uint64_t n,
                     uint8_t *outputs, int64_t *latency_ns, kb_server_stats *stats);

/*
 * keccak_p_batch -- the permutation alone, Keccak-p[b, n_r] (Section 3.1:
 * Table 1 widths b = 25, 50, 100, 200, 400, 800, 1600; Eq. 10 rounds), applied
 * in place to n states.  State i is 25 lanes at states + 25*i (device uint64,
 * 8-byte aligned): lane x + 5y is word x + 5y, its bit z (Eq. 1: string bit
 * w(5y+x)+z) is bit z of the word; for b < 1600 only the low w = b/25 bits are
 * read and the rest are written as zero.  The n_r rounds are the last n_r of
 * the 12 + 2l round indices (FIPS 202 Algorithm 7), so n_r = 12 + 2l gives
 * Keccak-f[b]; n_r may exceed that (earlier, negative indices).  For
 * reduced-round and small-width experiments; the hash entry points use
 * Keccak-f[1600] directly.  Stream-ordered.  Bad b, n_r < 0 or n_r > 10^6:
 * KB_ERR_INVALID; n == 0 or n_r == 0: no-op.
 */
int keccak_p_batch(uint64_t *states, int b, int nr, uint64_t n, void *stream);

/* Synchronises `stream`, returns the device status word (KB_DEV_* bits, 0 if
 * clean) accumulated by kernels on this device since the last call, and
 * clears it.  Returns KB_ERR_CUDA if the synchronisation fails. */
int keccak_last_error(void *stream);

/* Frees the cached scratch, staging buffers, streams and graphs of the
 * calling thread's current device.  Safe to call at any time when no work
 * of this library is in flight. */
void keccak_release(void);

/* Process-wide tuning knobs.  keccak_tune_set returns KB_OK or KB_ERR_INVALID
 * (unknown key or value); keccak_tune_get returns the value or -1 for an
 * unknown key.  Changing a knob affects calls issued afterwards.
 *   KB_TUNE_REPRESENTATION: register layout of the Keccak state in the
 *     fixed-stride SHA3-256 kernels -- KB_REP_PLAIN (default: 32-bit low/high
 *     halves of each lane) or KB_REP_INTERLEAVED (even/odd bit halves, the
 *     layout whose rotations need fewer funnel shifts but whose every message
 *     word must be bit-interleaved; kept as a measured control).  Other
 *     variants always use the plain layout. */
#define KB_TUNE_REPRESENTATION 0
#define KB_REP_PLAIN 0
#define KB_REP_INTERLEAVED 1
/*   KB_TUNE_RAGGED_SCHEDULE: how keccak_batch orders its work --
 *     KB_SCHEDULE_QUEUE (default: messages sorted into cost buckets, longest
 *     first, consumed by one persistent launch, one thread per message),
 *     KB_SCHEDULE_LANE_PARALLEL (the same order, one warp per message: the 25
 *     state lanes on 25 threads; about 2x lower latency per message at about
 *     4x the instructions, for few long messages), KB_SCHEDULE_PER_VARIANT (a
 *     control: one launch per variant over that variant's messages, rate fixed
 *     at compile time, not ordered by length) or KB_SCHEDULE_INPUT_ORDER (one
 *     thread per message in input order, the plain one-launch control).
 *   KB_TUNE_GRAPHS: 1 (default) replays the queue schedule's launches from a
 *     CUDA graph cached per call signature (pointers, n, stream); 0 launches
 *     directly.  Work issued on the legacy default stream or on a stream that
 *     is being captured is always launched directly.
 *   KB_TUNE_AUTOTUNE: 1 (default) uses configurations found by
 *     keccak_batch_autotune, in this process or read from the
 *     SHA3GB_TUNE_CACHE file, for batches of the same size class; 0 ignores
 *     them (as SHA3GB_TUNE=off does for the whole process).
 *   KB_TUNE_QUEUE_MIN_BLOCKS: register budget of the queue kernel, as the
 *     minimum resident 128-thread blocks per SM it is compiled for (2, 3, 4,
 *     5, 6 or 8; 0 = tuned or default 2).
 *   KB_TUNE_QUEUE_BLOCKS_PER_SM: blocks per SM of the persistent launch
 *     (1..32; 0 = tuned or as many as fit). */
#define KB_TUNE_RAGGED_SCHEDULE 1
#define KB_SCHEDULE_INPUT_ORDER 0
#define KB_SCHEDULE_QUEUE 1
#define KB_SCHEDULE_LANE_PARALLEL 2
#define KB_SCHEDULE_PER_VARIANT 3
#define KB_TUNE_GRAPHS 2
#define KB_TUNE_AUTOTUNE 3
#define KB_TUNE_QUEUE_MIN_BLOCKS 4
#define KB_TUNE_QUEUE_BLOCKS_PER_SM 5
/*   KB_TUNE_HOST_PATH: how keccak_batch_uniform_host moves data --
 *     KB_HOST_PATH_AUTO (default: decided per size class by a timed trial on
 *     page-locked buffers, staged for pageable ones), KB_HOST_PATH_STAGED
 *     (copy in chunks through device buffers), KB_HOST_PATH_ZERO_COPY (the
 *     kernel reads and writes the page-locked host buffers in place;
 *     KB_ERR_INVALID for pageable ones). */
#define KB_TUNE_HOST_PATH 6
#define KB_HOST_PATH_AUTO 0
#define KB_HOST_PATH_STAGED 1
#define KB_HOST_PATH_ZERO_COPY 2
/*   KB_TUNE_STAGING: how the fixed-stride kernel reads 64-byte messages packed
 *     back to back (stride 64, 16-byte aligned, device memory) --
 *     KB_STAGING_TMA (default: bulk asynchronous copies of 8 KiB tiles into
 *     shared memory, two deep, then each thread reads its message from there;
 *     measured ~0.8% faster) or KB_STAGING_DIRECT (each thread loads its
 *     message with four 16-byte loads; the measured control).  Other shapes,
 *     and host-mapped buffers, always load directly. */
#define KB_TUNE_STAGING 7
#define KB_STAGING_DIRECT 0
#define KB_STAGING_TMA 1
/*   KB_TUNE_QUEUE_STAGING: how keccak_batch's queue kernel reads message
 *     blocks and which form of the permutation it runs -- 0 (default: tuned,
 *     else KB_QUEUE_STAGING_REGS), KB_QUEUE_STAGING_DIRECT (each thread loads a block's
 *     words when it absorbs them; permutation with its last rounds unrolled),
 *     KB_QUEUE_STAGING_DIRECT_LOOPED (the same with all 24 rounds in a loop,
 *     half the code), KB_QUEUE_STAGING_ASYNC (looped; each thread's next block
 *     is copied into shared memory with cp.async while the current
 *     permutation runs) or KB_QUEUE_STAGING_REGS (looped; the next block is
 *     loaded into registers before the permutation and absorbed after it).
 *     The looped forms exist for register budgets 2..4 (KB_QUEUE_STAGING_REGS:
 *     2 and 3); with another budget the kernel loads directly.
 *   KB_TUNE_QUEUE_WARP_MESSAGES: threads per message -- -1 (default: tuned,
 *     else 0) or K >= 0: the K costliest messages of a batch run one warp each
 *     (the lane-parallel sponge) in a kernel started first on a side stream,
 *     concurrently with the queue kernel, which takes the rest one thread
 *     each. */
#define KB_TUNE_QUEUE_STAGING 8
#define KB_QUEUE_STAGING_DIRECT 1
#define KB_QUEUE_STAGING_DIRECT_LOOPED 2
#define KB_QUEUE_STAGING_ASYNC 3
#define KB_QUEUE_STAGING_REGS 4
#define KB_TUNE_QUEUE_WARP_MESSAGES 9
int keccak_tune_set(int key, int64_t value);
int64_t keccak_tune_get(int key);

/* The 24 round constants (Definition 5, Eq. 8-9) and 25 rho offsets (lane
 * index x+5y) compiled into the kernels, written to HOST arrays, so that
 * tests can compare them with an independent generation. */
int sha3gb_round_constants(uint64_t *rc24);
int sha3gb_rho_offsets(uint32_t *rho25);

/* Integer-issue microbenchmark for the ALU roofline (diagnostic, not part of
 * the hashing path): each thread runs `iters` rounds of 8 instructions of one
 * kind (op 0 LOP3 with the chi truth table, 1 SHF funnel shift by a register
 * amount, 2 PRMT with a register selector, 3 three-input 32-bit add), each
 * instruction taking three values of the previous round, so that no two
 * rounds fold into one instruction, on a one-wave grid, and writes the
 * measured thread-instructions issued per SM clock to *lanes_per_clk_per_sm
 * (HOST).  Synchronous on `stream`; allocates and frees a small device
 * buffer. */
int sha3gb_int_issue_probe(int op, uint32_t iters, double *lanes_per_clk_per_sm, void *stream);

/* Host-link diagnostic for the end-to-end figures (not part of the hashing
 * path): moves `bytes` (a multiple of 16, at least 32) between the HOST
 * buffer `host` and the DEVICE buffer `device` `reps` times after one untimed
 * pass and writes the rate in GB/s (10^9 bytes per second) to *gb_s (HOST).
 * mode 0: copy engine, host to device; 1: copy engine, device to host; 2: the
 * two directions at once, half of `bytes` each way on two streams; 3: SM
 * loads of page-locked host memory stored to the device buffer (KB_ERR_INVALID
 * for pageable memory).  Synchronous on `stream`; the buffers' contents are
 * overwritten. */
int sha3gb_host_link_probe(const void *host, void *device, size_t bytes, int mode, int reps, double *gb_s,
                           void *stream);

/* Exercises the bounded device wait of the 64-byte staging kernel (its
 * mbarrier wait for bulk copies) without a fault (diagnostic, not part of the
 * hashing path): one thread waits for phase 0 of a fresh shared-memory
 * mbarrier that, with arrive = 0, nothing completes.  The wait gives up after
 * limit_ns nanoseconds (1 .. 2e9) of the GPU's global timer, sets
 * KB_DEV_TIMEOUT in the device status word and the kernel returns; the
 * context stays usable.  With arrive = 1 the thread arrives first and the
 * wait returns at once.  Stream-ordered; read the result with
 * keccak_last_error.  KB_ERR_INVALID for arguments out of range. */
int sha3gb_wait_timeout_probe(uint64_t limit_ns, int arrive, void *stream);

/* Library version string (static storage). */
const char *sha3gb_version(void);

#ifdef __cplusplus
}
#endif

#endif
