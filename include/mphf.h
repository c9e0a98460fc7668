/*
 * mphf.h -- C ABI of the GB300-native PtrHash library (libmphf.so).
 *
 * PtrHash (Groot Koerkamp, SEA 2025) is a minimal perfect hash function: it
 * maps a set of n distinct keys bijectively onto [0, n).  The structure is
 * an array of 8-bit pilots, one per bucket, with P parts of B buckets and S
 * slots each, plus one remap table for slots >= n (Sec. 3.1, Fig. overview).
 *
 * Conventions for every entry point below:
 *  - Return 0 (MPHF_OK) or a negative MPHF_ERR_* code.  Nothing aborts and
 *    no C++ exception crosses this boundary.  mphf_last_error() gives a
 *    human-readable detail of the most recent failure on the calling thread.
 *  - "device pointer" means memory of the current CUDA device, owned by the
 *    caller, which must stay valid until the work on `stream` completes.
 *    "host pointer" means ordinary host memory owned by the caller; host
 *    memory that is page-locked (cudaHostAlloc / pinned) copies fastest.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Query calls are asynchronous on that stream unless stated.
 *  - A structure (mphf_t) owns its device memory and is released with
 *    mphf_free().  It may be queried concurrently from several streams.
 *  - Integer arithmetic is exact; results are bit-identical to the formula
 *    of Sec. 3.1 (Eq. partbucket, Eq. slot) and Sec. 3.4 (Eq. clef).
 */
#ifndef GB300_MPHF_H
#define GB300_MPHF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- codes */
#define MPHF_OK                 0
#define MPHF_ERR_ARG           -1  /* invalid argument (NULL, size, alignment) */
#define MPHF_ERR_OOM           -2  /* device or host allocation failed        */
#define MPHF_ERR_DUP_KEYS      -3  /* the key set holds duplicates            */
#define MPHF_ERR_BUILD_FAILED  -4  /* pilot search failed after every reseed  */
#define MPHF_ERR_FORMAT        -5  /* serialized bytes are not a valid structure */
#define MPHF_ERR_CUDA          -6  /* a CUDA runtime call failed              */
#define MPHF_ERR_TIMEOUT       -7  /* a bounded device wait gave up           */
#define MPHF_ERR_OVERFULL      -8  /* a part holds more keys than slots       */
#define MPHF_ERR_CAPACITY      -9  /* a fixed capacity of the library exceeded */

#define MPHF_KEY_U64    0  /* 64-bit integer keys, h(k) = C k (Sec. 3.1)       */
#define MPHF_KEY_BYTES  1  /* byte strings: packed bytes + n+1 u64 offsets     */

#define MPHF_GAMMA_LINEAR 1  /* gamma_1(x) = x                 (Sec. 3.3)     */
#define MPHF_GAMMA_CUBIC  3  /* gamma_3, the Default          (Sec. 3.3)     */

#define MPHF_REMAP_CLEF 0  /* CacheLineEF remap table         (Sec. 3.4)      */
#define MPHF_REMAP_VEC  1  /* plain u32 remap table           (Sec. 3.4)      */

/* ------------------------------------------------------------ parameters */
/* Construction parameters (Sec. 3.1 "Parameter values", Sec. 4.1.2
 * "Recommended parameters").  Default: lambda 3.5, alpha 0.99, gamma_3,
 * CacheLineEF; Fast: lambda 3.0, gamma_1, Vec; Compact: lambda 4.0. */
typedef struct {
    double   lambda;          /* expected bucket size                         */
    double   alpha;           /* load factor in (0, 1]                        */
    int32_t  gamma;           /* MPHF_GAMMA_*                                 */
    int32_t  remap;           /* MPHF_REMAP_*                                 */
    uint64_t seed;            /* global seed of hp(p) = C (p xor seed), and of
                                 the string hash                              */
    uint64_t C;               /* odd 64-bit mixing constant                   */
    uint64_t slots_override;  /* 0: the parameter rule picks S; else forced S */
    int32_t  max_reseeds;     /* extra attempts with seed+1, seed+2, ...      */
    uint32_t evict_mult;      /* a part fails after evict_mult * S evictions  */
    uint64_t shard_keys;      /* build in shards of whole parts holding about
                                 this many keys each (in-memory sharding,
                                 Appendix B); 0: automatic, from the free
                                 device memory.  The structure is the same
                                 for every value.                             */
    int32_t  hash128;         /* byte keys: 1 = the 128-bit string hash (the
                                 high half picks part and bucket, the low half
                                 the slot, Sec. 3.1); 0 = only when n > 2^32.
                                 u64 keys ignore it (h = C k is injective).   */
    int32_t  reserved;        /* 0                                            */
} mphf_params;

/* Fills *p with the Default parameters.  Returns MPHF_ERR_ARG for NULL. */
int mphf_default_params(mphf_params *p);

typedef struct mphf mphf_t;

/* Description of a structure. */
typedef struct {
    uint64_t n, P, S, B;      /* keys, parts, slots per part, buckets per part */
    uint64_t C, seed;
    int32_t  gamma, remap, reduce, key_kind;  /* reduce: 0 = hi(C x) mod 2^k,
                                                 1 = x mod S (Sec. 3.1)      */
    uint64_t remap_len;       /* P*S - n entries of the remap table F          */
    uint64_t pilot_bytes;     /* P*B                                           */
    uint64_t remap_bytes;     /* CacheLineEF: 64 per 44 entries; Vec: 4 each
                                 (8 once n > 2^32)                             */
    double   bits_per_key;    /* 8 (pilot_bytes + remap_bytes) / n              */
    uint64_t evictions;       /* hash-evict evictions of the build (0 if loaded)*/
    double   build_ms;        /* device time of mphf_build (0 if loaded)        */
    double   build_hash_sort_ms;  /* of which hashing, sorting, bucket bounds   */
    double   build_search_ms;     /* pilot search (Sec. 3.2)                    */
    double   build_remap_ms;      /* remap and CacheLineEF encoding (Sec. 3.4)  */
} mphf_info_t;

/* --------------------------------------------------------------- build */
/* Builds the structure of n distinct keys on the GPU (Sec. 3.2: hash, sort,
 * per-part greedy pilot search with hash-evict, then the remap of Sec. 3.4).
 *   key_kind  MPHF_KEY_U64: keys_dev = n uint64_t (device pointer,
 *             8-byte aligned); offsets_dev must be NULL.
 *             MPHF_KEY_BYTES: keys_dev = packed bytes (device pointer);
 *             offsets_dev = n+1 non-decreasing uint64_t (device), key i being
 *             bytes [offsets[i], offsets[i+1]).
 *   n         1 <= n <= 2^40 (CacheLineEF stores values below 2^40).
 *             Beyond 2^32 keys the values need the _wide queries, and the
 *             build runs in shards of whole parts (see shard_keys).
 * Runs on `stream` and returns once the structure is complete (it
 * synchronizes that stream).  Temporary device memory comes from the
 * stream-ordered allocator on `stream` and goes back to it, without
 * synchronizing the device, so builds called from several host threads on
 * different streams run concurrently (many small structures fill the GPU
 * together).  Errors: MPHF_ERR_ARG, MPHF_ERR_DUP_KEYS (equal u64 keys, or equal
 * strings), MPHF_ERR_OVERFULL, MPHF_ERR_BUILD_FAILED, MPHF_ERR_OOM,
 * MPHF_ERR_CUDA.  On error *out is set to NULL.
 * u64 keys are hashed as h = C k (Sec. 3.1), which suits random-looking keys;
 * strongly structured key sets (multiples of a power of two, arithmetic
 * progressions) can end in MPHF_ERR_BUILD_FAILED in small layouts, and should
 * be passed through a bijective 64-bit mixer first. */
int mphf_build(const mphf_params *params, int key_kind, const void *keys_dev,
               const uint64_t *offsets_dev, uint64_t n, void *stream,
               mphf_t **out);

/* ------------------------------------------------------------- queries */
/* Evaluates the MPHF on m u64 keys (Sec. 3.1, Eq. partbucket and Eq. slot;
 * Sec. 3.4 remap for slots >= n):
 *   out[i] = slot(k_i) if slot(k_i) < n, else F[slot(k_i) - n].
 * keys_dev: m uint64_t (device, 8-byte aligned; 16-byte alignment takes the
 * vectorized path); out_dev: m uint32_t (device, 4-byte aligned).  Keys that
 * are not members give a deterministic value in [0, n).  m = 0 is a no-op.
 * Needs n <= 2^32 (values fit 32 bits).  Asynchronous on `stream`.  Errors:
 * MPHF_ERR_ARG, MPHF_ERR_CUDA (launch). */
int mphf_query_u64(const mphf_t *m, const uint64_t *keys_dev, uint64_t count,
                   uint32_t *out_dev, void *stream);
/* How mphf_query_u64 runs: a batch of at least 2^24 keys against a pilot
 * array above 72 MiB, with 16-byte aligned keys and out aligned to two
 * elements, takes the windowed path of mphf_query_u64_windowed in W =
 * ceil(pilot bytes / 100 MB) windows (at least 2), as long as W is at most 6
 * (pilot arrays up to 600 MB: n from about 2.6e8 to 2.1e9 with the Default
 * parameters); everything else runs the single-pass kernel.  Both
 * give the same values.  mphf_query_u64_phf, mphf_query_u64_wide and
 * mphf_lookup_u64 choose the same way.  The windowed path's first use on a
 * structure allocates its scratch (cudaMalloc, 6 bytes per key of a chunk of
 * at most 2^28 keys, 1.6 GB at most), which the structure keeps until
 * mphf_free; make that first large query outside stream capture.  If the
 * scratch cannot be allocated, the single-pass kernel runs instead. */

/* The windowed evaluation of the same function (no paper counterpart; the
 * paper's query reads each key's pilot where it lies, Sec. 3.1).  The pilot
 * array is cut into W = ceil(P B / window_bytes) byte ranges, each small
 * enough to stay in L2, and the keys are streamed once per range: the first
 * pass computes every key's bucket (Eq. partbucket) and keeps it in a 32-bit
 * stream for the passes that read it, each pass reads the pilots of the keys
 * whose bucket lies in its range, and the last pass computes the slot and
 * remap value (Eq. slot, Sec. 3.4); for gamma_1 structures the last pass
 * computes the bucket again from the key instead of reading the stream.  Random DRAM reads of the pilot array become L2 hits, at the
 * cost of reading the keys twice and 6 bytes of scratch traffic per key and
 * middle pass.  Results equal mphf_query_u64's, key by key.
 *   window_bytes  pilot bytes per range; 0: the automatic W above (which
 *                 may be 1).  W = 1 (window_bytes >= P B) runs the
 *                 single-pass kernel.
 *   chunk_keys    keys per chunk (even, at most 2^31; 0: 2^28).  Every chunk
 *                 reads the pilot array once more; the scratch is 6 bytes per
 *                 key of a chunk rounded up to 16 keys, owned by the
 *                 structure (allocated on first use, grown when a larger
 *                 chunk is asked for, freed by mphf_free).  Uses of the scratch from different streams are
 *                 ordered on the GPU.
 * keys_dev 16-byte and out_dev 8-byte aligned when W >= 2.  Asynchronous on
 * `stream`, except that allocating or growing the scratch synchronizes the
 * device.  Errors: MPHF_ERR_ARG (alignment, odd or oversized chunk, P B >=
 * 2^32, byte-key structure, n > 2^32), MPHF_ERR_OOM (scratch), MPHF_ERR_CUDA. */
int mphf_query_u64_windowed(const mphf_t *m, const uint64_t *keys_dev, uint64_t count,
                            uint32_t *out_dev, uint64_t window_bytes, uint64_t chunk_keys,
                            void *stream);

/* The same for byte-string keys: key i = bytes_dev[offsets_dev[i] ..
 * offsets_dev[i+1]).  offsets_dev: count+1 non-decreasing uint64_t (device).
 * Requires a structure built for MPHF_KEY_BYTES (else MPHF_ERR_ARG). */
int mphf_query_bytes(const mphf_t *m, const uint8_t *bytes_dev,
                     const uint64_t *offsets_dev, uint64_t count,
                     uint32_t *out_dev, void *stream);

/* The same queries with uint64_t results, for any structure (needed once
 * n > 2^32; for smaller n the values equal the 32-bit ones).  out_dev: m
 * uint64_t (device, 8-byte aligned).  Other arguments and errors as above. */
int mphf_query_u64_wide(const mphf_t *m, const uint64_t *keys_dev, uint64_t count,
                        uint64_t *out_dev, void *stream);
int mphf_query_bytes_wide(const mphf_t *m, const uint8_t *bytes_dev,
                          const uint64_t *offsets_dev, uint64_t count,
                          uint64_t *out_dev, void *stream);

/* Perfect (non-minimal) hash: slot(k_i) in [0, P*S) without the remap
 * (Sec. 3.1 Eq. slot; Table remap "Query PHF").  Same arguments as
 * mphf_query_u64. */
int mphf_query_u64_phf(const mphf_t *m, const uint64_t *keys_dev, uint64_t count,
                       uint32_t *out_dev, void *stream);

/* End-to-end query from host memory.  When both buffers are page-locked
 * and mapped (cudaHostAlloc, cudaHostRegister), the kernel reads the keys
 * and writes the results across the host link directly.  Otherwise the keys
 * are copied to the device in chunks, evaluated, and the results copied
 * back, overlapping the copies with the kernels on `stream` and two
 * internal copy streams (staging buffers owned by the structure, allocated
 * on first use).
 * keys_host: count uint64_t (host); out_host: count uint32_t (host).
 * Returns when every result is in out_host (synchronous).  Errors:
 * MPHF_ERR_ARG, MPHF_ERR_OOM, MPHF_ERR_CUDA. */
int mphf_query_u64_host(mphf_t *m, const uint64_t *keys_host, uint64_t count,
                        uint32_t *out_host, void *stream);

/* ------------------------------------------------ serialize / describe */
/* Serialized format (little-endian): a 128-byte header, the P*B pilot bytes
 * padded to 64, then the remap payload.  This is the interchange format
 * with other implementations.  With host_buf NULL or cap too small, only
 * *needed is set and MPHF_ERR_ARG is returned if host_buf is not NULL.
 * Synchronous. */
int mphf_serialize(const mphf_t *m, void *host_buf, size_t cap, size_t *needed);

/* Loads a serialized structure onto the current device (synchronous).
 * Errors: MPHF_ERR_FORMAT (bad magic, version, sizes or fields),
 * MPHF_ERR_OOM, MPHF_ERR_CUDA. */
int mphf_deserialize(const void *host_buf, size_t len, mphf_t **out);

int mphf_info(const mphf_t *m, mphf_info_t *out);

/* Releases the structure and its device memory.  NULL is a no-op.  The
 * caller must ensure no query on it is still running. */
void mphf_free(mphf_t *m);

const char *mphf_strerror(int code);

/* Detail of the last failure on the calling thread (never NULL). */
const char *mphf_last_error(void);

/* Layout chosen by the parameter rule for n keys (Sec. 3.1 "Parameter
 * values"), without building: fills P, S, B and reduce of *out. */
int mphf_layout(const mphf_params *params, uint64_t n, mphf_info_t *out);

/* ------------------------------------------------------ roofline probe */
/* The random-gather microbenchmark that bounds the query kernel: for each
 * of `count` u64 keys, one byte is read from table_dev[fastrange(mix(k),
 * table_bytes)] and written out as u32, with the same key stream and the
 * same launch shape as mphf_query_u64.  No paper counterpart: this is the
 * measured denominator for the query kernel's roofline fraction.
 * keys_dev: count u64 (device); table_dev: table_bytes bytes (device);
 * out_dev: count u32 (device).  Asynchronous on `stream`. */
int mphf_gather_probe(const uint64_t *keys_dev, uint64_t count,
                      const uint8_t *table_dev, uint64_t table_bytes,
                      uint32_t *out_dev, void *stream);

/* The probe matched to the query's own access pattern: out_dev[i] =
 * table_dev[idx_dev[i]] (0 where idx_dev[i] >= table_bytes), with the launch
 * shape of mphf_query_u64, 8 index bytes in and 4 result bytes out per key.
 * Given the bucket indexes of a query stream (mphf_bucket_u64) and the
 * structure's own pilot array (mphf_device_view), it makes exactly the
 * query's pilot gathers, at the same addresses and with the same skew,
 * without the hashing, slot and remap arithmetic around them: the measured
 * random-gather bound of that query.  No paper counterpart.
 * idx_dev: count u64 (device, 16-byte aligned); table_dev: table_bytes bytes
 * (device); out_dev: count u32 (device, 8-byte aligned).  Asynchronous on
 * `stream`.  Errors: MPHF_ERR_ARG. */
int mphf_gather_probe_at(const uint64_t *idx_dev, uint64_t count,
                         const uint8_t *table_dev, uint64_t table_bytes,
                         uint32_t *out_dev, void *stream);

/* Bucket of each u64 key as an index into the pilot array: out_dev[i] =
 * part(k_i) B + bucket(k_i) (Sec. 3.1, Eq. partbucket), the position of the
 * pilot the query of k_i reads.  keys_dev: count u64 (device, 8-byte
 * aligned); out_dev: count u64 (device, 8-byte aligned).  Requires a
 * structure built for MPHF_KEY_U64.  Asynchronous on `stream`.  Errors:
 * MPHF_ERR_ARG, MPHF_ERR_CUDA. */
int mphf_bucket_u64(const mphf_t *m, const uint64_t *keys_dev, uint64_t count,
                    uint64_t *out_dev, void *stream);

/* --------------------------------------------------- multi-MPHF batches */
/* One request of a batch: `count` keys of structure m.  For u64 structures
 * keys_dev holds count uint64_t and offsets_dev is NULL; for byte-key
 * structures keys_dev holds packed bytes and offsets_dev count+1 uint64_t.
 * out_dev receives count uint32_t.  All device pointers, caller-owned. */
typedef struct {
    const mphf_t   *m;
    const void     *keys_dev;
    const uint64_t *offsets_dev;
    uint64_t        count;          /* < 2^32 */
    uint32_t       *out_dev;
} mphf_request;

/* Launch shape of the persistent batch kernel. */
typedef struct {
    int32_t keys_per_thread;  /* 2, 4, 8 or 16 gathers in flight per thread  */
    int32_t threads;          /* 128, 256 or 512 threads per CTA             */
    int32_t blocks_per_sm;    /* 1..16 persistent CTAs per SM                */
    int32_t use_graph;        /* replay a captured CUDA graph (1) or launch  */
} mphf_batch_config;

typedef struct mphf_batch mphf_batch_t;

/* A batch executor for up to max_requests (<= 4096) requests per run: one
 * persistent kernel launch per run evaluates every request, whatever its
 * structure and size (the paper's query_all over many structures, App. A;
 * no paper counterpart for the multi-structure dispatch).  Owns two staging
 * sets (page-locked host + device descriptor buffers) and their graphs.
 * Default shape: 8 keys per thread, 512 threads, 2 CTAs per SM, graphs on. */
int mphf_batch_create(uint32_t max_requests, mphf_batch_t **out);

/* Evaluates every request; results are identical to mphf_query_u64 /
 * mphf_query_bytes on each request.  Asynchronous on `stream`: returns once
 * the work is queued (waits only for the run two calls back, whose staging
 * set it reuses).  The structures and buffers must stay valid until the
 * stream reaches this point.  Errors: MPHF_ERR_ARG, MPHF_ERR_CAPACITY,
 * MPHF_ERR_CUDA. */
int mphf_batch_run(mphf_batch_t *b, const mphf_request *reqs, uint32_t nreq, void *stream);

int mphf_batch_set_config(mphf_batch_t *b, const mphf_batch_config *c);
int mphf_batch_get_config(const mphf_batch_t *b, mphf_batch_config *c);

/* Times every launch shape on this batch (best of 3 runs after a warm-up),
 * keeps the fastest, and writes it to *best (may be NULL).  With a non-NULL
 * cache_path the choice is looked up in / appended to that JSON-lines file,
 * keyed by key kind, decade of the total key count, SM count and the
 * library's build time (a rebuilt library tunes again).
 * Synchronous. */
int mphf_batch_autotune(mphf_batch_t *b, const mphf_request *reqs, uint32_t nreq, void *stream,
                        const char *cache_path, mphf_batch_config *best);

/* Waits for outstanding runs and releases the executor.  NULL is a no-op. */
void mphf_batch_free(mphf_batch_t *b);

/* ----------------------------------------------------------- serving */
/* A serving loop with continuous batching (no paper counterpart; the
 * paper's streaming query_all of App. A is the single-caller analogue).
 * Structures are registered as serialized bytes and kept on the device
 * while their pilot + remap bytes fit hbm_budget_bytes; idle ones (nothing
 * queued or in flight) are evicted least-recently-used when a structure with
 * queued requests needs room, and re-admitted later from the host copy.
 * A dispatcher thread coalesces queued requests of resident structures,
 * in arrival order, into batches of at most max_batch_requests requests and
 * max_batch_keys keys, and runs each batch on one of `slots` streams
 * (persistent batch kernel), so up to `slots` batches overlap on the GPU and
 * requests that arrive meanwhile join the next free slot. */
typedef struct {
    uint64_t hbm_budget_bytes;    /* device bytes for resident structures   */
    uint32_t max_batch_requests;  /* 1..4096 requests per launch             */
    uint64_t max_batch_keys;      /* keys per launch (a single larger request
                                     still runs alone)                        */
    int32_t  slots;               /* 1..16 concurrent batches (streams)      */
} mphf_server_config;

typedef struct {
    uint32_t        structure;    /* id from mphf_server_add                 */
    const void     *keys_dev;     /* u64 keys, or packed bytes (device)      */
    const uint64_t *offsets_dev;  /* byte keys: count+1 offsets; else NULL   */
    uint64_t        count;
    uint32_t       *out_dev;      /* count uint32_t (device)                 */
} mphf_server_req;

typedef struct {
    double   p50_us, p99_us, max_us, mean_us;   /* arrival -> completion   */
    double   queries_per_s;       /* completed keys / (last completion -
                                     first arrival)                          */
    uint64_t requests, queries, batches;
    double   mean_requests_per_batch;
    uint64_t admissions, evictions, resident_bytes;
} mphf_server_stats_t;

typedef struct mphf_server mphf_server_t;

/* Defaults: 16 GiB budget, 1024 requests and 2^24 keys per batch, 4 slots. */
int mphf_server_default_config(mphf_server_config *c);
int mphf_server_create(const mphf_server_config *cfg, mphf_server_t **out);
/* Registers a structure (copied; validated by loading it once).  It is
 * admitted onto the device when requests for it are queued.  Errors:
 * MPHF_ERR_FORMAT, MPHF_ERR_CAPACITY (larger than the whole budget). */
int mphf_server_add(mphf_server_t *s, const void *serialized, size_t len, uint32_t *id);
/* Unregisters: waits for its queued and in-flight requests, frees it. */
int mphf_server_remove(mphf_server_t *s, uint32_t id);
/* Queues one request; the caller's buffers must stay valid until it is done.
 * Latency is measured from this call. */
int mphf_server_submit(mphf_server_t *s, const mphf_server_req *r, uint64_t *ticket);
/* Open-loop load: request i arrives arrival_us[i] microseconds after the
 * call; the calling thread submits each at its time and its latency is
 * measured from that scheduled arrival.  Returns after the last submit. */
int mphf_server_replay(mphf_server_t *s, const mphf_server_req *reqs, const double *arrival_us, uint32_t n,
                       uint64_t *tickets);
/* Waits for one request (MPHF_ERR_TIMEOUT after timeout_us); *status gets
 * the request's own result code. */
int mphf_server_wait(mphf_server_t *s, uint64_t ticket, uint64_t timeout_us, int *status);
/* Waits until nothing is queued or in flight. */
int mphf_server_drain(mphf_server_t *s, uint64_t timeout_us);
/* Latency percentiles and throughput of completed requests (reset: clear). */
int mphf_server_stats(mphf_server_t *s, int reset, mphf_server_stats_t *out);
/* Stops the dispatcher after the queued work, and frees everything. */
void mphf_server_free(mphf_server_t *s);

/* ------------------------------------------------ build without allocating */
/* Builds the structure of n <= 65536 distinct u64 keys like mphf_build, but
 * allocates no device memory: all of its device working memory lives in one
 * fixed 8 MiB array that is part of the library's builder module.  It serves
 * callers that may not allocate device memory: code running under a
 * framework that owns all device memory through its own pool and budget,
 * threads where the device-wide synchronization of cudaMalloc/cudaFree would
 * stall other streams, or processes whose device memory is fully committed.
 * The paper has no counterpart; this is a deployment variant of the build.
 *   keys_dev   n uint64_t (device, 8-byte aligned), 1 <= n <= 65536.
 *   out_host   host buffer receiving the structure in the serialized format
 *              of mphf_serialize (load it with mphf_deserialize); cap bytes.
 *   needed     set to the serialized size (may be NULL).
 * The result is byte-identical to mphf_serialize(mphf_build(...)) for the
 * same keys and parameters.
 * Errors: MPHF_ERR_CAPACITY if n, the number of parts, or the layout's
 * working memory exceeds the fixed array (the message names the limit);
 * MPHF_ERR_ARG if out_host is NULL or smaller than *needed (retry with a
 * larger buffer); otherwise as mphf_build.
 * When the 8 MiB are taken: the CUDA runtime gives the array device memory
 * when it loads the builder's module on a device.  With lazy module loading
 * (the CUDA default) that is the first call into the builder on that device,
 * this function or mphf_build; with CUDA_MODULE_LOADING=EAGER it is the
 * creation of the device's context.  A caller that must not allocate later
 * (a device it will fill up) makes one call early, while memory is free, or
 * sets CUDA_MODULE_LOADING=EAGER.  The device then holds the array until its
 * context is destroyed.
 * The call is synchronous: it waits for its own work on `stream` and copies
 * the result to out_host, so it must not be issued on a stream that is being
 * captured into a CUDA graph.  The array's device address is looked up
 * (cudaGetSymbolAddress) on the first call in each context of a device and
 * cached; after cudaDeviceReset the next call looks it up again.
 * Every call on a device shares the one array and overwrites what the
 * previous call left there, so calls that overlap on the GPU (from several
 * host threads or streams) race: serialize them. */
int mphf_build_u64_noalloc(const mphf_params *params, const uint64_t *keys_dev, uint64_t n,
                           void *out_host, size_t cap, size_t *needed, void *stream);

/* -------------------------------------------------- device-side view */
/* Everything a kernel needs to evaluate a structure (see mphf_device.cuh):
 * device pointers into the structure's memory plus its layout. */
typedef struct {
    const uint8_t *pilots;     /* P*B pilot bytes (device)                       */
    const void    *remap;      /* CacheLineEF lines or u32 entries (device)      */
    uint64_t n, P, S, B, C, seed;
    uint64_t barrett;          /* floor(2^64 / S) when reduce = x mod S          */
    uint64_t s_mask;           /* S - 1 when S is a power of two                 */
    int32_t  gamma;            /* MPHF_GAMMA_*                                   */
    int32_t  reduce;           /* 0: S = 2^k, reduce(x) = hi(C x) & (S - 1);
                                  1: reduce(x) = x mod S (Sec. 3.1)              */
    int32_t  remap_kind;       /* MPHF_REMAP_*                                   */
    int32_t  key_kind;         /* MPHF_KEY_*                                     */
    int32_t  hash128;          /* byte keys: 1 = 128-bit string hash (its high
                                  half picks part and bucket, Sec. 3.1)          */
    int32_t  reserved;
} mphf_view_t;

/* Fills *out with the structure's device view, for fusing the evaluation
 * into a caller's own kernels through include/mphf_device.cuh (no paper
 * counterpart; the paper's conclusion asks for streaming queries inside
 * applications).  The view stays valid until mphf_free(m).  Errors:
 * MPHF_ERR_ARG. */
int mphf_device_view(const mphf_t *m, mphf_view_t *out);

/* Sets the maximum L2 fetch granularity of the calling thread's current
 * CUDA context to `bytes` (0..128; a performance hint the platform may clamp)
 * and stores the value in force before the call in *previous (if non-NULL).
 * No paper counterpart.  For random byte gathers over tables far larger than
 * L2 (the pilot array), 128 reduces the query time on GB300.  The limit is
 * context-wide: it applies to every kernel of the process on that device
 * until it is set again, and it ends with the context.  The library never
 * changes it by itself.  Errors: MPHF_ERR_ARG (bytes outside 0..128),
 * MPHF_ERR_CUDA. */
int mphf_set_l2_fetch_granularity(int bytes, int *previous);

/* Fused lookup through the MPHF: out[i] = table[h(keys[i])] for i < count,
 * where h is the structure's value for a u64 key (Sec. 3.1 Eq. slot,
 * Sec. 3.4) and table holds n elements of elem_bytes (4 or 8) bytes.  This is
 * the MPHF's use as the index of a static key set (Sec. 1, Motivation) with
 * the lookup streamed inside the consuming kernel (Sec. 5): one kernel, the
 * value never stored (large batches against a pilot array above L2 run the
 * windowed passes of mphf_query_u64_windowed, whose last pass reads the
 * table entry instead of writing the value).  Non-member keys read some
 * element of the table.
 * keys_dev: count u64 (device, 8-byte aligned); table_dev: n elements
 * (device, aligned to elem_bytes; owned by the caller); out_dev: count
 * elements (device, aligned to elem_bytes).  Any n, including n > 2^32.
 * Asynchronous on `stream`.  Errors: MPHF_ERR_ARG (NULL or misaligned
 * pointers, elem_bytes not 4 or 8, a byte-key structure). */
int mphf_lookup_u64(const mphf_t *m, const uint64_t *keys_dev, uint64_t count,
                    const void *table_dev, uint32_t elem_bytes, void *out_dev,
                    void *stream);

/* Number of kernel launches this library issued since it was loaded
 * (all entry points, all threads). */
uint64_t mphf_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif
