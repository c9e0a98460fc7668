/*
 * PtrHash CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of the PtrHash minimal
 * perfect hash function (Groot Koerkamp, "PtrHash: Minimal Perfect Hashing
 * at RAM Throughput", SEA 2025): parameter rule, key hashing, part / bucket /
 * slot formulas, the greedy + hash-evict pilot search, remapping, and the
 * CacheLineEF encoding.  Only the test-suite, the smoke check and the CPU
 * baseline legs of the benchmark may load this library; the product path
 * never does.  It shares no code, header, table or constant generator with
 * the CUDA library: both sides read and write the same serialized byte
 * format, each with its own code.
 *
 * Parity status of each function is stated next to its declaration.
 * "parity unpinned" marks a function with no pin other than itself.
 */
#ifndef PTRHASH_ORACLE_H
#define PTRHASH_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes (0 = success). */
#define ORC_OK              0
#define ORC_ERR_ARG        -1
#define ORC_ERR_OOM        -2
#define ORC_ERR_DUP_KEYS   -3
#define ORC_ERR_BUILD      -4
#define ORC_ERR_FORMAT     -5
#define ORC_ERR_CLEF_SPAN  -6
#define ORC_ERR_OVERFULL   -7

#define ORC_GAMMA_LINEAR 1 /* gamma_1(x) = x            (Sec. 3.3)        */
#define ORC_GAMMA_CUBIC  3 /* gamma_3, the default      (Sec. 3.3)        */

#define ORC_REMAP_CLEF 0   /* CacheLineEF               (Sec. 3.4, Eq. clef) */
#define ORC_REMAP_VEC  1   /* plain array F: u32, u64 once n > 2^32 (Sec. 3.4) */

#define ORC_REDUCE_POW2 0  /* reduce(x,S) = hi(C x) mod S, S = 2^k (Sec. 3.1) */
#define ORC_REDUCE_MOD  1  /* reduce(x,S) = x mod S, S not 2^k  (Sec. 3.1)  */

#define ORC_KEY_U64   0
#define ORC_KEY_BYTES 1

#define ORC_CLEF_PER_LINE 44

/* CacheLineEF keeps values below 2^40 (a 32-bit offset in units of 256),
 * which bounds n; values pass 32 bits once n > 2^32. */
#define ORC_MAX_KEYS (1ull << 40)

/* Layout chosen by the parameter rule (Sec. 3.1 "Parameter values"). */
typedef struct {
    uint64_t n;      /* number of keys                                  */
    uint64_t P;      /* parts                                           */
    uint64_t S;      /* slots per part                                  */
    uint64_t B;      /* buckets per part                                */
    int32_t  reduce; /* ORC_REDUCE_POW2 / ORC_REDUCE_MOD                 */
    int32_t  pad;
} orc_layout;

/* Build parameters. */
typedef struct {
    double   lambda;          /* expected bucket size (3.5 Default)        */
    double   alpha;           /* load factor (0.99)                        */
    int32_t  gamma;           /* ORC_GAMMA_*                               */
    int32_t  remap;           /* ORC_REMAP_*                               */
    uint64_t seed;            /* global seed of hp() (and of string hash)  */
    uint64_t C;               /* mixing constant (odd)                     */
    uint64_t slots_override;  /* 0 = parameter rule; else forced S          */
    int32_t  max_reseeds;     /* reseed attempts after a failed part        */
    uint32_t evict_mult;      /* eviction cap = evict_mult * S per part     */
    int32_t  threads;         /* worker threads for independent parts       */
    int32_t  hash128;         /* byte keys: 1 = 128-bit hash; 0 = only when
                                 n > 2^32 (Sec. 3.1, "Hash functions")       */
} orc_params;

/* Constructed structure, host memory. */
typedef struct {
    orc_layout L;
    int32_t  gamma, remap, key_kind, hash128;
    uint64_t C, seed;
    double   lambda, alpha;
    uint8_t *pilots;        /* P*B bytes                                   */
    uint64_t remap_len;     /* P*S - n entries of F                        */
    uint8_t *clef;          /* ceil(remap_len/44) lines of 64 bytes        */
    uint64_t *vec;          /* remap_len entries (ORC_REMAP_VEC)           */
    uint64_t clef_lines;
} orc_mphf;

/* ---- arithmetic primitives (pinned by closed forms in the tests) ---- */
uint64_t orc_hi(uint64_t a, uint64_t b);
uint64_t orc_lo(uint64_t a, uint64_t b);
uint64_t orc_gamma(int gamma, uint64_t x);
uint64_t orc_hash_u64(uint64_t C, uint64_t k);
/* The string hash is this project's own definition (the paper's GxHash is
 * not specified in it).  Its finishing mixer is SplitMix64's, pinned to that
 * generator's published outputs through the empty string; the per-word fold
 * and sum are parity unpinned against external values and pinned only by
 * structural properties in the tests. */
uint64_t orc_hash_bytes(const uint8_t *s, uint64_t len, uint64_t seed);
/* The 128-bit variant: *lo is orc_hash_bytes, *hi the same construction
 * with its own seed tweak and fold constant.  hi picks the part and bucket,
 * lo the slot.  Pinned like the 64-bit hash: the finishing mixer against
 * SplitMix64's outputs, the fold (parity unpinned) by properties. */
void     orc_hash_bytes128(const uint8_t *s, uint64_t len, uint64_t seed, uint64_t *hi, uint64_t *lo);
uint64_t orc_hp(uint64_t C, uint64_t seed, uint64_t pilot);
uint64_t orc_reduce(int reduce, uint64_t C, uint64_t x, uint64_t S);
void     orc_part_bucket(const orc_layout *L, int gamma, uint64_t h,
                         uint64_t *part, uint64_t *bucket_in_part);

/* ---- parameter rule ---- */
int orc_layout_for(uint64_t n, double lambda, double alpha,
                   uint64_t slots_override, orc_layout *out);
void orc_default_params(orc_params *p);

/* ---- CacheLineEF ---- */
int      orc_clef_encode(const uint64_t *vals, uint64_t len, uint8_t *lines);
uint64_t orc_clef_get(const uint8_t *lines, uint64_t j);

/* ---- construction ---- */
int orc_build_u64(const uint64_t *keys, uint64_t n, const orc_params *p,
                  orc_mphf **out);
int orc_build_bytes(const uint8_t *bytes, const uint64_t *offsets, uint64_t n,
                    const orc_params *p, orc_mphf **out);
void orc_free(orc_mphf *m);

/* ---- query (one key at a time) ---- */
uint64_t orc_slot_of_hash(const orc_mphf *m, uint64_t h);
/* With separate hashes for the part and bucket (hb) and the slot (hs). */
uint64_t orc_slot_of_hash2(const orc_mphf *m, uint64_t hb, uint64_t hs);
uint64_t orc_query_hash(const orc_mphf *m, uint64_t h);
void orc_query_u64_many(const orc_mphf *m, const uint64_t *keys, uint64_t cnt,
                        uint64_t *out, int threads);
void orc_query_bytes_many(const orc_mphf *m, const uint8_t *bytes,
                          const uint64_t *offsets, uint64_t cnt, uint64_t *out,
                          int threads);
/* PHF (non-minimal) query: the slot before remapping. */
void orc_slot_u64_many(const orc_mphf *m, const uint64_t *keys, uint64_t cnt,
                       uint64_t *out);

/* ---- serialized format ---- */
uint64_t orc_serialized_size(const orc_mphf *m);
int orc_serialize(const orc_mphf *m, uint8_t *buf, uint64_t cap);
int orc_deserialize(const uint8_t *buf, uint64_t len, orc_mphf **out);

/* ---- accessors for tests ---- */
void orc_get_layout(const orc_mphf *m, orc_layout *L);
const uint8_t *orc_pilots(const orc_mphf *m);
uint64_t orc_remap_len(const orc_mphf *m);
void orc_remap_values(const orc_mphf *m, uint64_t *out); /* decoded F */
uint64_t orc_seed(const orc_mphf *m);
int orc_remap_kind(const orc_mphf *m);
int orc_gamma_kind(const orc_mphf *m);
uint64_t orc_total_evictions(void); /* of the most recent build          */

#ifdef __cplusplus
}
#endif
#endif
