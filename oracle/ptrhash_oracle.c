/*
 * PtrHash CPU oracle -- TEST INFRASTRUCTURE ONLY (see ptrhash_oracle.h).
 *
 * Plain C, exact 128-bit integer arithmetic through unsigned __int128, no
 * blocking, fusion or reordering beyond what the paper states.  Sections and
 * equations cited below are those of the PtrHash paper (SEA 2025):
 *   Sec. 3.1  Overview: Eq. partbucket, Eq. slot, hp(), reduce, parameters
 *   Sec. 3.2  Construction: greedy placement + hash-evict
 *   Sec. 3.3  Bucket assignment functions: gamma_1, gamma_3
 *   Sec. 3.4  Remapping using CacheLineEF: Eq. clef and its lookup
 * Where the paper is silent the reading taken is stated inline.
 */
#define _GNU_SOURCE
#include "ptrhash_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define NONE32 0xFFFFFFFFu

/* ------------------------------------------------------------------ */
/* Arithmetic primitives                                                */
/* ------------------------------------------------------------------ */

/* hi(a*b): the high 64 bits of the 128-bit product (Sec. 3.1, Eq. partbucket). */
uint64_t orc_hi(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * (u128)b) >> 64); }

/* lo(a*b): the low 64 bits of the 128-bit product (Sec. 3.1). */
uint64_t orc_lo(uint64_t a, uint64_t b) { return (uint64_t)((u128)a * (u128)b); }

/* Bucket assignment function on 64-bit fixed point, input and output being
 * fractions of 2^64 (Sec. 3.3, "Approximations").
 *   gamma_1(x) = x
 *   gamma_3(x) = (255/256) * (x^2 + x^3)/2 + x/256, with x^2 = hi(x*x) and
 *   x^3 = hi(x^2 * x); every division rounds down (reading: the paper only
 *   says the powers are computed through hi()). */
uint64_t orc_gamma(int gamma, uint64_t x) {
    if (gamma == ORC_GAMMA_LINEAR) return x;
    uint64_t x2 = orc_hi(x, x);
    uint64_t x3 = orc_hi(x2, x);
    uint64_t half_sum = (x2 >> 1) + (x3 >> 1);      /* (x^2 + x^3) / 2 */
    return half_sum - (half_sum >> 8) + (x >> 8);   /* 255/256 * . + x/256 */
}

/* Integer keys: h(k) = C * k mod 2^64 (Sec. 3.1, "Hash functions"). */
uint64_t orc_hash_u64(uint64_t C, uint64_t k) { return C * k; }

/* Pilot hash hp(p) = C * (p xor seed) mod 2^64 (Sec. 3.1, Eq. hp). */
uint64_t orc_hp(uint64_t C, uint64_t seed, uint64_t pilot) { return C * (pilot ^ seed); }

/* reduce(x, S) (Sec. 3.1, "The reduce function"):
 *   S a power of two:  hi(C * x) mod S
 *   otherwise:         x mod S (the exact value that "fast mod" computes). */
uint64_t orc_reduce(int reduce, uint64_t C, uint64_t x, uint64_t S) {
    if (reduce == ORC_REDUCE_POW2) return orc_hi(C, x) % S;
    return x % S;
}

/* Eq. partbucket (Sec. 3.1):
 *   part(k)   = hi(P * h)
 *   x         = lo(P * h) / 2^64
 *   bucket(k) = hi(B * (2^64 * gamma(x)))        (bucket within its part) */
void orc_part_bucket(const orc_layout *L, int gamma, uint64_t h,
                     uint64_t *part, uint64_t *bucket_in_part) {
    *part = orc_hi(L->P, h);
    uint64_t x = orc_lo(L->P, h);
    *bucket_in_part = orc_hi(L->B, orc_gamma(gamma, x));
}

/* String keys.  The paper uses GxHash, which it does not define; this is the
 * project's own 64-bit string hash (the finishing mixer, and the fold and
 * sum at word inputs 0, 1 and 2^63, are pinned to SplitMix64's outputs):
 *   fold(x) = high 64 bits xor low 64 bits of the 128-bit product x * K3
 *   w_j     = little-endian u64 of bytes [8j, 8j+8), zero-padded past len
 *   acc     = sum_j fold(w_j xor (seed + j * K1))             (mod 2^64)
 *   h       = mix(acc xor (len * K2) xor seed)
 *   mix(z)  = splitmix64 finalizer (Steele, Lea, Flood 2014):
 *             z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
 *             z *= 0x94D049BB133111EB; z ^= z>>31
 * with K1 = 0x9E3779B97F4A7C15, K2 = 0xC2B2AE3D27D4EB4F and the fold
 * constant K3 = 0xA173621FA8385BE3.  The sum makes the words independent of
 * each other, so any split of the words over parallel workers gives the
 * same value; one multiply per word keeps the per-word work small. */
static uint64_t str_mix(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

static uint64_t str_fold(uint64_t x, uint64_t K3) {
    const unsigned __int128 p = (unsigned __int128)x * K3;
    return (uint64_t)(p >> 64) ^ (uint64_t)p;
}

static uint64_t hash_words(const uint8_t *s, uint64_t len, uint64_t seed, uint64_t K3) {
    const uint64_t K1 = 0x9E3779B97F4A7C15ull, K2 = 0xC2B2AE3D27D4EB4Full;
    uint64_t acc = 0;
    uint64_t nwords = (len + 7) / 8;
    for (uint64_t j = 0; j < nwords; j++) {
        uint64_t w = 0;
        for (uint64_t b = 0; b < 8; b++) {
            uint64_t pos = 8 * j + b;
            uint64_t byte = pos < len ? s[pos] : 0;
            w |= byte << (8 * b);
        }
        acc += str_fold(w ^ (seed + j * K1), K3);
    }
    return str_mix(acc ^ (len * K2) ^ seed);
}

uint64_t orc_hash_bytes(const uint8_t *s, uint64_t len, uint64_t seed) {
    return hash_words(s, len, seed, 0xA173621FA8385BE3ull);
}

/* 128-bit variant (Sec. 3.1: beyond 2^32 keys, a 128-bit string hash whose
 * high half picks the part and bucket and whose low half the slot):
 * lo = the 64-bit hash; hi = the same construction with seed xor K4 and the
 * fold constant K5, K4 = 0x47523634D9D6709B, K5 = 0x2EF8175451B07575. */
void orc_hash_bytes128(const uint8_t *s, uint64_t len, uint64_t seed, uint64_t *hi, uint64_t *lo) {
    *lo = orc_hash_bytes(s, len, seed);
    *hi = hash_words(s, len, seed ^ 0x47523634D9D6709Bull, 0x2EF8175451B07575ull);
}

/* ------------------------------------------------------------------ */
/* Parameter rule (Sec. 3.1, "Parameter values")                        */
/* ------------------------------------------------------------------ */

static int is_pow2(uint64_t v) { return v && !(v & (v - 1)); }

/* Keys per part alpha*S >= 80000 * ln(n / 80000), at least 80000.
 * S is the smallest power of two with alpha*S >= that, P = ceil(n/(alpha S)),
 * B = ceil(alpha*S / lambda).  Reading for the "few parts" case: when the
 * power-of-two S would leave more than 5% of all slots beyond n/alpha, the
 * layout switches to reduce = x mod S with P = ceil(n / kpp) and
 * S = max(ceil(n / (alpha P)), ceil(n / P) + 16), bumped by one if it is
 * even.  Sec. 3.1 asks for an S that is not a power of two so that x mod S
 * depends on every bit of x; an even S still passes the low bits of x
 * through (x mod 2 = (x mod S) mod 2), and keys whose hashes end in t zero
 * bits (h = C k keeps the trailing zeros of k) would reach only
 * S / gcd(S, 2^t) slots.  An odd S is never a power of two (S > 16 here).
 * slots_override != 0 forces S (reduce then follows S being a power of 2). */
int orc_layout_for(uint64_t n, double lambda, double alpha,
                   uint64_t slots_override, orc_layout *out) {
    if (n == 0 || n > ORC_MAX_KEYS || !(lambda > 0.0) || !(alpha > 0.0) || alpha > 1.0)
        return ORC_ERR_ARG;
    memset(out, 0, sizeof(*out));
    out->n = n;
    double nd = (double)n;
    double kpp = 80000.0 * log(nd / 80000.0);
    if (kpp < 80000.0) kpp = 80000.0;
    uint64_t S, P;
    int reduce;
    if (slots_override) {
        S = slots_override;
        P = (uint64_t)ceil(nd / (alpha * (double)S));
        reduce = is_pow2(S) ? ORC_REDUCE_POW2 : ORC_REDUCE_MOD;
    } else {
        S = 1;
        while ((double)S < kpp / alpha) S <<= 1;
        P = (uint64_t)ceil(nd / (alpha * (double)S));
        reduce = ORC_REDUCE_POW2;
        if ((double)(P * S) > 1.05 * nd / alpha) {
            P = (uint64_t)ceil(nd / kpp);
            if (P < 1) P = 1;
            S = (uint64_t)ceil(nd / (alpha * (double)P));
            /* Reading for tiny n: 1% slack is then below a slot or two, and
             * with fewer buckets than the 16-entry tabu ring no eviction is
             * possible; keep at least 16 spare slots per part. */
            uint64_t min_s = (n + P - 1) / P + 16;
            if (S < min_s) S = min_s;
            if (S % 2 == 0) S += 1;
            reduce = ORC_REDUCE_MOD;
        }
    }
    if (P < 1) P = 1;
    uint64_t B = (uint64_t)ceil(alpha * (double)S / lambda);
    if (B < 1) B = 1;
    if (P * S < n || P * S - n >= ORC_MAX_KEYS || S > 0xFFFFFFFFull) return ORC_ERR_ARG;
    out->P = P;
    out->S = S;
    out->B = B;
    out->reduce = reduce;
    return ORC_OK;
}

void orc_default_params(orc_params *p) {
    memset(p, 0, sizeof(*p));
    p->lambda = 3.5;             /* Default (Sec. 4.1.2, recommended parameters) */
    p->alpha = 0.99;
    p->gamma = ORC_GAMMA_CUBIC;
    p->remap = ORC_REMAP_CLEF;
    p->seed = 0;
    p->C = 0x9E3779B97F4A7C15ull; /* reading: the paper prints no value; any odd constant */
    p->slots_override = 0;
    p->max_reseeds = 8;
    p->evict_mult = 10;          /* "a total of 10S evictions" (Sec. 4.1.2) */
    p->threads = 1;
}

/* ------------------------------------------------------------------ */
/* CacheLineEF (Sec. 3.4, Eq. clef)                                     */
/* ------------------------------------------------------------------ */
/* Line layout (reading; the figure is not available): bytes 0..15 hold the
 * 128-bit relative-high bitmap as two little-endian u64 words (bit j lives
 * in word j/64 at bit j%64), bytes 16..19 the 32-bit offset floor(v_0/256),
 * bytes 20..63 the 44 low bytes.  A short final chunk repeats its last
 * value. */

static void put_u64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void put_u32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static uint64_t get_u64(const uint8_t *p) { uint64_t v = 0; for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i); return v; }
static uint32_t get_u32(const uint8_t *p) { uint32_t v = 0; for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i); return v; }

int orc_clef_encode(const uint64_t *vals, uint64_t len, uint8_t *lines) {
    uint64_t nlines = (len + ORC_CLEF_PER_LINE - 1) / ORC_CLEF_PER_LINE;
    for (uint64_t c = 0; c < nlines; c++) {
        uint64_t v[ORC_CLEF_PER_LINE];
        for (uint64_t i = 0; i < ORC_CLEF_PER_LINE; i++) {
            uint64_t idx = c * ORC_CLEF_PER_LINE + i;
            v[i] = idx < len ? vals[idx] : vals[len - 1];
            if (v[i] >= (1ull << 40)) return ORC_ERR_ARG;        /* 40-bit limit */
            if (i > 0 && v[i] < v[i - 1]) return ORC_ERR_ARG;    /* non-decreasing */
        }
        uint64_t offset = v[0] >> 8;
        uint64_t word[2] = {0, 0};
        uint8_t *line = lines + 64 * c;
        for (uint64_t i = 0; i < ORC_CLEF_PER_LINE; i++) {
            uint64_t bit = i + ((v[i] >> 8) - offset);   /* bit i + high(v_i) - high(v_0) */
            if (bit >= 128) return ORC_ERR_CLEF_SPAN;
            word[bit / 64] |= 1ull << (bit % 64);
            line[20 + i] = (uint8_t)(v[i] & 0xFF);       /* low 8 bits */
        }
        put_u64(line, word[0]);
        put_u64(line + 8, word[1]);
        put_u32(line + 16, (uint32_t)offset);
    }
    return ORC_OK;
}

/* Lookup: v_i = 2^8 * (offset + select(i) - i) + low[i], select(i) being the
 * position of the i-th (0-based) set bit of the 128-bit field (Sec. 3.4,
 * "Lookup").  Select is a plain scan over the 128 bits. */
uint64_t orc_clef_get(const uint8_t *lines, uint64_t j) {
    const uint8_t *line = lines + 64 * (j / ORC_CLEF_PER_LINE);
    uint64_t i = j % ORC_CLEF_PER_LINE;
    uint64_t word[2] = {get_u64(line), get_u64(line + 8)};
    uint64_t offset = get_u32(line + 16);
    uint64_t seen = 0, sel = 0;
    for (uint64_t bit = 0; bit < 128; bit++) {
        if ((word[bit / 64] >> (bit % 64)) & 1) {
            if (seen == i) { sel = bit; break; }
            seen++;
        }
    }
    return 256 * (offset + sel - i) + line[20 + i];
}

/* ------------------------------------------------------------------ */
/* Query (Sec. 3.1, Eq. slot; Sec. 3.4 remap)                           */
/* ------------------------------------------------------------------ */

/* slot(k) = part * S + reduce(h xor hp(p_bucket), S)   (Eq. slot) */
uint64_t orc_slot_of_hash(const orc_mphf *m, uint64_t h) { return orc_slot_of_hash2(m, h, h); }

/* 128-bit string hashes: hb (the high half) picks the part and bucket in
 * Eq. partbucket, hs (the low half) enters Eq. slot. */
uint64_t orc_slot_of_hash2(const orc_mphf *m, uint64_t hb, uint64_t hs) {
    uint64_t part, b;
    orc_part_bucket(&m->L, m->gamma, hb, &part, &b);
    uint64_t pilot = m->pilots[part * m->L.B + b];
    uint64_t x = hs ^ orc_hp(m->C, m->seed, pilot);
    return part * m->L.S + orc_reduce(m->L.reduce, m->C, x, m->L.S);
}

static uint64_t remap_get(const orc_mphf *m, uint64_t j) {
    if (m->remap == ORC_REMAP_VEC) return m->vec[j];
    return orc_clef_get(m->clef, j);
}

/* A slot >= n is replaced by F[slot - n] (Sec. 3.4, "Remapping"). */
uint64_t orc_query_hash(const orc_mphf *m, uint64_t h) {
    uint64_t s = orc_slot_of_hash(m, h);
    if (s < m->L.n) return s;
    return remap_get(m, s - m->L.n);
}

static uint64_t query_hash2(const orc_mphf *m, uint64_t hb, uint64_t hs) {
    uint64_t s = orc_slot_of_hash2(m, hb, hs);
    if (s < m->L.n) return s;
    return remap_get(m, s - m->L.n);
}

typedef struct {
    const orc_mphf *m;
    const uint64_t *keys;
    const uint8_t *bytes;
    const uint64_t *offsets;
    uint64_t *out;
    uint64_t lo, hi;
} query_job;

static void *query_u64_worker(void *arg) {
    query_job *J = (query_job *)arg;
    for (uint64_t i = J->lo; i < J->hi; i++)
        J->out[i] = orc_query_hash(J->m, orc_hash_u64(J->m->C, J->keys[i]));
    return NULL;
}

static void *query_bytes_worker(void *arg) {
    query_job *J = (query_job *)arg;
    for (uint64_t i = J->lo; i < J->hi; i++) {
        uint64_t a = J->offsets[i], b = J->offsets[i + 1];
        if (J->m->hash128) {
            uint64_t hi, lo;
            orc_hash_bytes128(J->bytes + a, b - a, J->m->seed, &hi, &lo);
            J->out[i] = query_hash2(J->m, hi, lo);
        } else {
            J->out[i] = orc_query_hash(J->m, orc_hash_bytes(J->bytes + a, b - a, J->m->seed));
        }
    }
    return NULL;
}

static void run_split(void *(*fn)(void *), query_job base, uint64_t cnt, int threads) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((uint64_t)threads > cnt) threads = cnt ? (int)cnt : 1;
    pthread_t tid[256];
    query_job jobs[256];
    for (int t = 0; t < threads; t++) {
        jobs[t] = base;
        jobs[t].lo = cnt * (uint64_t)t / (uint64_t)threads;
        jobs[t].hi = cnt * (uint64_t)(t + 1) / (uint64_t)threads;
    }
    if (threads == 1) { fn(&jobs[0]); return; }
    for (int t = 0; t < threads; t++) pthread_create(&tid[t], NULL, fn, &jobs[t]);
    for (int t = 0; t < threads; t++) pthread_join(tid[t], NULL);
}

void orc_query_u64_many(const orc_mphf *m, const uint64_t *keys, uint64_t cnt,
                        uint64_t *out, int threads) {
    query_job J = {m, keys, NULL, NULL, out, 0, 0};
    run_split(query_u64_worker, J, cnt, threads);
}

void orc_query_bytes_many(const orc_mphf *m, const uint8_t *bytes,
                          const uint64_t *offsets, uint64_t cnt, uint64_t *out,
                          int threads) {
    query_job J = {m, NULL, bytes, offsets, out, 0, 0};
    run_split(query_bytes_worker, J, cnt, threads);
}

void orc_slot_u64_many(const orc_mphf *m, const uint64_t *keys, uint64_t cnt, uint64_t *out) {
    for (uint64_t i = 0; i < cnt; i++) out[i] = orc_slot_of_hash(m, orc_hash_u64(m->C, keys[i]));
}

/* ------------------------------------------------------------------ */
/* Construction (Sec. 3.2)                                              */
/* ------------------------------------------------------------------ */

static uint64_t g_total_evictions;
uint64_t orc_total_evictions(void) { return g_total_evictions; }

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

typedef struct { uint64_t hi, lo; } pair128;

static int cmp_pair128(const void *a, const void *b) {
    const pair128 *x = (const pair128 *)a, *y = (const pair128 *)b;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    return x->lo < y->lo ? -1 : x->lo > y->lo;
}

/* Per-part state of the pilot search. */
typedef struct {
    uint64_t *h;          /* the part's slot hashes, sorted                */
    uint64_t *hb;         /* its bucket hashes: h itself, or the high halves
                             of 128-bit hashes (sorted by (hb, h))         */
    uint64_t cnt;
    uint32_t *start;      /* B+1 bucket offsets into h                     */
    uint32_t *owner;      /* S entries: bucket that holds the slot, or NONE */
    uint32_t *heap;       /* max-heap of bucket ids                        */
    uint64_t heap_len;
    uint32_t recent[16];  /* ring of the 16 most recently placed buckets   */
    int recent_pos;
} part_state;

static uint64_t bsize(const part_state *ps, uint32_t b) { return ps->start[b + 1] - ps->start[b]; }

/* Heap order: larger bucket first, ties by lower bucket id (reading). */
static int heap_before(const part_state *ps, uint32_t a, uint32_t b) {
    uint64_t sa = bsize(ps, a), sb = bsize(ps, b);
    if (sa != sb) return sa > sb;
    return a < b;
}

static void heap_push(part_state *ps, uint32_t b) {
    uint64_t i = ps->heap_len++;
    ps->heap[i] = b;
    while (i > 0) {
        uint64_t parent = (i - 1) / 2;
        if (!heap_before(ps, ps->heap[i], ps->heap[parent])) break;
        uint32_t t = ps->heap[i]; ps->heap[i] = ps->heap[parent]; ps->heap[parent] = t;
        i = parent;
    }
}

static uint32_t heap_pop(part_state *ps) {
    uint32_t top = ps->heap[0];
    ps->heap[0] = ps->heap[--ps->heap_len];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, best = i;
        if (l < ps->heap_len && heap_before(ps, ps->heap[l], ps->heap[best])) best = l;
        if (r < ps->heap_len && heap_before(ps, ps->heap[r], ps->heap[best])) best = r;
        if (best == i) break;
        uint32_t t = ps->heap[i]; ps->heap[i] = ps->heap[best]; ps->heap[best] = t;
        i = best;
    }
    return top;
}

static int in_recent(const part_state *ps, uint32_t b) {
    for (int i = 0; i < 16; i++) if (ps->recent[i] == b) return 1;
    return 0;
}

typedef struct {
    const orc_mphf *m;     /* layout, gamma, C, seed                        */
    uint32_t evict_mult;
} build_ctx;

/* Slot (within the part) of every key of bucket b under pilot p. */
static void bucket_slots(const build_ctx *bc, const part_state *ps, uint32_t b,
                         uint64_t pilot, uint64_t *slots) {
    const orc_mphf *m = bc->m;
    uint64_t hp = orc_hp(m->C, m->seed, pilot);
    for (uint64_t j = ps->start[b]; j < ps->start[b + 1]; j++)
        slots[j - ps->start[b]] = orc_reduce(m->L.reduce, m->C, ps->h[j] ^ hp, m->L.S);
}

static int self_collides(const uint64_t *slots, uint64_t s) {
    for (uint64_t a = 0; a < s; a++)
        for (uint64_t c = a + 1; c < s; c++)
            if (slots[a] == slots[c]) return 1;
    return 0;
}

/* Greedy placement with hash-evict for one part (Sec. 3.2).  Writes the
 * part's B pilots and marks taken[slot] for its S slots.  Returns ORC_OK,
 * ORC_ERR_DUP_KEYS (two equal hashes) or ORC_ERR_BUILD (no pilot at all, or
 * more than evict_mult * S evictions). */
static int build_part(const build_ctx *bc, part_state *ps, uint64_t part,
                      uint8_t *pilots, uint8_t *taken, uint64_t *evictions_out) {
    const orc_mphf *m = bc->m;
    const uint64_t S = m->L.S, B = m->L.B;
    *evictions_out = 0;

    /* Sort the part's hashes; equal neighbours are duplicate keys. */
    if (ps->hb == ps->h) {
        qsort(ps->h, ps->cnt, sizeof(uint64_t), cmp_u64);
        for (uint64_t i = 1; i < ps->cnt; i++)
            if (ps->h[i] == ps->h[i - 1]) return ORC_ERR_DUP_KEYS;
    } else {   /* 128-bit hashes: sort the pairs (hb, h) */
        pair128 *pr = (pair128 *)malloc((ps->cnt + 1) * sizeof(pair128));
        if (!pr) return ORC_ERR_OOM;
        for (uint64_t i = 0; i < ps->cnt; i++) { pr[i].hi = ps->hb[i]; pr[i].lo = ps->h[i]; }
        qsort(pr, ps->cnt, sizeof(pair128), cmp_pair128);
        for (uint64_t i = 0; i < ps->cnt; i++) { ps->hb[i] = pr[i].hi; ps->h[i] = pr[i].lo; }
        free(pr);
        for (uint64_t i = 1; i < ps->cnt; i++)
            if (ps->hb[i] == ps->hb[i - 1] && ps->h[i] == ps->h[i - 1]) return ORC_ERR_DUP_KEYS;
    }

    /* Bucket boundaries by counting (sorted hashes fall in bucket order). */
    for (uint64_t b = 0; b <= B; b++) ps->start[b] = 0;
    for (uint64_t i = 0; i < ps->cnt; i++) {
        uint64_t pp, b;
        orc_part_bucket(&m->L, m->gamma, ps->hb[i], &pp, &b);
        ps->start[b + 1]++;
    }
    for (uint64_t b = 0; b < B; b++) ps->start[b + 1] += ps->start[b];

    for (uint64_t s = 0; s < S; s++) ps->owner[s] = NONE32;
    for (int i = 0; i < 16; i++) ps->recent[i] = NONE32;
    ps->recent_pos = 0;
    ps->heap_len = 0;
    for (uint64_t b = 0; b < B; b++) {
        pilots[b] = 0;
        if (bsize(ps, (uint32_t)b) > 0) heap_push(ps, (uint32_t)b);
    }

    uint64_t max_bucket = 0;
    for (uint64_t b = 0; b < B; b++) if (bsize(ps, (uint32_t)b) > max_bucket) max_bucket = bsize(ps, (uint32_t)b);
    uint64_t *slots = (uint64_t *)malloc((max_bucket + 1) * sizeof(uint64_t));
    if (!slots) return ORC_ERR_OOM;

    uint64_t evictions = 0;
    int rc = ORC_OK;
    while (ps->heap_len > 0) {
        uint32_t b = heap_pop(ps);
        uint64_t s = bsize(ps, b);
        int chosen = -1;
        /* Greedy: the smallest pilot whose keys all land in distinct free slots. */
        for (int p = 0; p < 256 && chosen < 0; p++) {
            bucket_slots(bc, ps, b, (uint64_t)p, slots);
            if (self_collides(slots, s)) continue;
            int ok = 1;
            for (uint64_t j = 0; j < s; j++) if (ps->owner[slots[j]] != NONE32) { ok = 0; break; }
            if (ok) chosen = p;
        }
        if (chosen < 0) {
            /* Hash-evict: the pilot of least weighted collisions, a collision
             * with a key of a bucket of size s' weighing s'^2; pilots that
             * hit one of the 16 most recently placed buckets are skipped. */
            uint64_t best_cost = UINT64_MAX;
            for (int p = 0; p < 256; p++) {
                bucket_slots(bc, ps, b, (uint64_t)p, slots);
                if (self_collides(slots, s)) continue;
                uint64_t cost = 0;
                int blocked = 0;
                for (uint64_t j = 0; j < s; j++) {
                    uint32_t o = ps->owner[slots[j]];
                    if (o == NONE32) continue;
                    if (in_recent(ps, o)) { blocked = 1; break; }
                    cost += bsize(ps, o) * bsize(ps, o);
                }
                if (blocked) continue;
                if (cost < best_cost) { best_cost = cost; chosen = p; }
            }
            if (chosen < 0) {
                /* Reading: the tabu only exists to break eviction cycles; when
                 * it blocks every pilot that does not self-collide, it is
                 * ignored for this bucket.  Only a bucket whose every pilot
                 * self-collides fails the part. */
                for (int p = 0; p < 256; p++) {
                    bucket_slots(bc, ps, b, (uint64_t)p, slots);
                    if (self_collides(slots, s)) continue;
                    uint64_t cost = 0;
                    for (uint64_t j = 0; j < s; j++) {
                        uint32_t o = ps->owner[slots[j]];
                        if (o != NONE32) cost += bsize(ps, o) * bsize(ps, o);
                    }
                    if (cost < best_cost) { best_cost = cost; chosen = p; }
                }
            }
            if (chosen < 0) { rc = ORC_ERR_BUILD; break; }
            bucket_slots(bc, ps, b, (uint64_t)chosen, slots);
            for (uint64_t j = 0; j < s; j++) {
                uint32_t o = ps->owner[slots[j]];
                if (o == NONE32) continue;
                /* Evict o: empty every slot it maps to and queue it again. */
                uint64_t os = bsize(ps, o);
                uint64_t *oslots = (uint64_t *)malloc(os * sizeof(uint64_t));
                if (!oslots) { rc = ORC_ERR_OOM; break; }
                bucket_slots(bc, ps, o, pilots[o], oslots);
                for (uint64_t t = 0; t < os; t++) ps->owner[oslots[t]] = NONE32;
                free(oslots);
                heap_push(ps, o);
                evictions++;
            }
            if (rc != ORC_OK) break;
            if (evictions > (uint64_t)bc->evict_mult * S) { rc = ORC_ERR_BUILD; break; }
        }
        pilots[b] = (uint8_t)chosen;
        bucket_slots(bc, ps, b, (uint64_t)chosen, slots);
        for (uint64_t j = 0; j < s; j++) ps->owner[slots[j]] = b;
        ps->recent[ps->recent_pos] = b;
        ps->recent_pos = (ps->recent_pos + 1) % 16;
    }
    free(slots);
    *evictions_out = evictions;
    if (rc != ORC_OK) return rc;
    for (uint64_t sl = 0; sl < S; sl++) taken[part * S + sl] = ps->owner[sl] != NONE32;
    return ORC_OK;
}

typedef struct {
    const build_ctx *bc;
    const uint64_t *by_part;    /* hashes grouped by part                   */
    const uint64_t *by_part_hi; /* their high halves (128-bit), else NULL   */
    const uint64_t *part_start; /* P+1 offsets                              */
    uint8_t *taken;
    uint64_t next_part;         /* shared work counter                      */
    pthread_mutex_t lock;
    int rc;
    uint64_t evictions;
} build_pool;

static void *build_worker(void *arg) {
    build_pool *bp = (build_pool *)arg;
    const orc_mphf *m = bp->bc->m;
    part_state ps;
    memset(&ps, 0, sizeof(ps));
    uint64_t max_cnt = 0;
    for (uint64_t p = 0; p < m->L.P; p++) {
        uint64_t c = bp->part_start[p + 1] - bp->part_start[p];
        if (c > max_cnt) max_cnt = c;
    }
    ps.h = (uint64_t *)malloc((max_cnt + 1) * sizeof(uint64_t));
    ps.hb = bp->by_part_hi ? (uint64_t *)malloc((max_cnt + 1) * sizeof(uint64_t)) : ps.h;
    ps.start = (uint32_t *)malloc((m->L.B + 1) * sizeof(uint32_t));
    ps.owner = (uint32_t *)malloc(m->L.S * sizeof(uint32_t));
    ps.heap = (uint32_t *)malloc(m->L.B * sizeof(uint32_t));
    int rc = (ps.h && ps.hb && ps.start && ps.owner && ps.heap) ? ORC_OK : ORC_ERR_OOM;
    uint64_t ev_total = 0;
    while (rc == ORC_OK) {
        pthread_mutex_lock(&bp->lock);
        uint64_t p = bp->next_part++;
        int stop = bp->rc != ORC_OK;
        pthread_mutex_unlock(&bp->lock);
        if (stop || p >= m->L.P) break;
        ps.cnt = bp->part_start[p + 1] - bp->part_start[p];
        memcpy(ps.h, bp->by_part + bp->part_start[p], ps.cnt * sizeof(uint64_t));
        if (bp->by_part_hi) memcpy(ps.hb, bp->by_part_hi + bp->part_start[p], ps.cnt * sizeof(uint64_t));
        uint64_t ev = 0;
        rc = build_part(bp->bc, &ps, p, m->pilots + p * m->L.B, bp->taken, &ev);
        ev_total += ev;
    }
    if (ps.hb != ps.h) free(ps.hb);
    free(ps.h); free(ps.start); free(ps.owner); free(ps.heap);
    pthread_mutex_lock(&bp->lock);
    if (rc != ORC_OK && bp->rc == ORC_OK) bp->rc = rc;
    bp->evictions += ev_total;
    pthread_mutex_unlock(&bp->lock);
    return NULL;
}

/* Remap (Sec. 3.4): with q_0 < ... < q_{R-1} the taken slots >= n and
 * L_0 < ... < L_{R-1} the free slots < n, F[q_i - n] = L_i.  Undefined
 * entries take their predecessor's value; entries before the first defined
 * one take the first defined value (reading); with R = 0 every entry is 0. */
static int build_remap(orc_mphf *m, const uint8_t *taken, int want_clef) {
    const uint64_t n = m->L.n, total = m->L.P * m->L.S;
    m->remap_len = total - n;
    uint64_t *F = (uint64_t *)calloc(m->remap_len ? m->remap_len : 1, sizeof(uint64_t));
    if (!F) return ORC_ERR_OOM;
    uint64_t R_high = 0, R_low = 0;
    for (uint64_t q = n; q < total; q++) R_high += taken[q];
    for (uint64_t q = 0; q < n; q++) R_low += !taken[q];
    if (R_high != R_low) { free(F); return ORC_ERR_BUILD; }
    uint8_t *defined = (uint8_t *)calloc(m->remap_len ? m->remap_len : 1, 1);
    if (!defined) { free(F); return ORC_ERR_OOM; }
    uint64_t free_pos = 0;
    for (uint64_t q = n; q < total; q++) {
        if (!taken[q]) continue;
        while (taken[free_pos]) free_pos++;      /* next free slot below n */
        F[q - n] = free_pos;
        defined[q - n] = 1;
        free_pos++;
    }
    uint64_t first = 0;
    int have = 0;
    for (uint64_t j = 0; j < m->remap_len; j++) if (defined[j]) { first = F[j]; have = 1; break; }
    uint64_t prev = have ? first : 0;
    for (uint64_t j = 0; j < m->remap_len; j++) {
        if (defined[j]) prev = F[j];
        else F[j] = prev;
    }
    free(defined);

    int rc = ORC_OK;
    m->remap = ORC_REMAP_VEC;
    if (want_clef && m->remap_len > 0) {
        m->clef_lines = (m->remap_len + ORC_CLEF_PER_LINE - 1) / ORC_CLEF_PER_LINE;
        m->clef = (uint8_t *)calloc(m->clef_lines, 64);
        if (!m->clef) { free(F); return ORC_ERR_OOM; }
        rc = orc_clef_encode(F, m->remap_len, m->clef);
        if (rc == ORC_OK) m->remap = ORC_REMAP_CLEF;
        else if (rc == ORC_ERR_CLEF_SPAN) {   /* fall back to a plain array */
            free(m->clef); m->clef = NULL; m->clef_lines = 0; rc = ORC_OK;
        }
    } else if (want_clef) {
        m->remap = ORC_REMAP_CLEF;
        m->clef_lines = 0;
    }
    if (rc == ORC_OK && m->remap == ORC_REMAP_VEC) {
        m->vec = (uint64_t *)malloc((m->remap_len ? m->remap_len : 1) * sizeof(uint64_t));
        if (!m->vec) { free(F); return ORC_ERR_OOM; }
        for (uint64_t j = 0; j < m->remap_len; j++) m->vec[j] = F[j];
    }
    free(F);
    return rc;
}

/* Hash -> partition by part -> per-part pilot search -> remap
 * (Sec. 3.2 and Sec. 4.1.2 "time breakdown": hashing, sorting, pilots,
 * remapping).  For string keys the seed also enters the key hash, so a
 * failed attempt changes every hash; for integer keys h = C*k does not
 * depend on it and only hp() changes. */
static int build_common(const uint64_t *keys, const uint8_t *bytes, const uint64_t *offsets,
                        uint64_t n, const orc_params *prm, int key_kind, orc_mphf **out) {
    *out = NULL;
    if (!prm || !(prm->C & 1)) return ORC_ERR_ARG;
    if (prm->gamma != ORC_GAMMA_LINEAR && prm->gamma != ORC_GAMMA_CUBIC) return ORC_ERR_ARG;
    if (prm->remap != ORC_REMAP_CLEF && prm->remap != ORC_REMAP_VEC) return ORC_ERR_ARG;
    orc_layout L;
    int rc = orc_layout_for(n, prm->lambda, prm->alpha, prm->slots_override, &L);
    if (rc != ORC_OK) return rc;
    if (L.B > 0xFFFFFFFEull) return ORC_ERR_ARG;

    /* Byte keys take the 128-bit hash beyond 2^32 keys, or when asked to
     * (Sec. 3.1); u64 keys never need it (h = C k is injective). */
    const int h128 = key_kind == ORC_KEY_BYTES && (prm->hash128 || n > (1ull << 32));
    uint64_t *h = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *by_part = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *hh = h128 ? (uint64_t *)malloc(n * sizeof(uint64_t)) : NULL;
    uint64_t *by_part_hi = h128 ? (uint64_t *)malloc(n * sizeof(uint64_t)) : NULL;
    uint64_t *part_start = (uint64_t *)calloc(L.P + 1, sizeof(uint64_t));
    uint64_t *cursor = (uint64_t *)calloc(L.P, sizeof(uint64_t));
    uint8_t *taken = (uint8_t *)calloc(L.P * L.S, 1);
    if (!h || !by_part || !part_start || !cursor || !taken || (h128 && (!hh || !by_part_hi))) {
        free(h); free(by_part); free(hh); free(by_part_hi); free(part_start); free(cursor); free(taken);
        return ORC_ERR_OOM;
    }
    /* hb[i]: the hash that picks key i's part and bucket. */
    const uint64_t *hb = h128 ? hh : h;
    g_total_evictions = 0;
    rc = ORC_ERR_BUILD;
    for (int attempt = 0; attempt <= prm->max_reseeds; attempt++) {
        uint64_t seed = prm->seed + (uint64_t)attempt;
        orc_mphf *m = (orc_mphf *)calloc(1, sizeof(orc_mphf));
        if (!m) { rc = ORC_ERR_OOM; break; }
        m->L = L; m->gamma = prm->gamma; m->key_kind = key_kind; m->hash128 = h128;
        m->C = prm->C; m->seed = seed; m->lambda = prm->lambda; m->alpha = prm->alpha;
        m->pilots = (uint8_t *)calloc(L.P * L.B, 1);
        if (!m->pilots) { orc_free(m); rc = ORC_ERR_OOM; break; }

        for (uint64_t i = 0; i < n; i++) {
            if (key_kind == ORC_KEY_U64) h[i] = orc_hash_u64(prm->C, keys[i]);
            else if (h128) orc_hash_bytes128(bytes + offsets[i], offsets[i + 1] - offsets[i], seed, &hh[i], &h[i]);
            else h[i] = orc_hash_bytes(bytes + offsets[i], offsets[i + 1] - offsets[i], seed);
        }
        /* Counting sort of the hashes by part. */
        memset(part_start, 0, (L.P + 1) * sizeof(uint64_t));
        for (uint64_t i = 0; i < n; i++) part_start[orc_hi(L.P, hb[i]) + 1]++;
        for (uint64_t p = 0; p < L.P; p++) part_start[p + 1] += part_start[p];
        int overfull = 0;
        for (uint64_t p = 0; p < L.P; p++) if (part_start[p + 1] - part_start[p] > L.S) overfull = 1;
        if (overfull) {
            orc_free(m);
            rc = ORC_ERR_OVERFULL;
            if (key_kind == ORC_KEY_U64) break;   /* reseeding cannot move u64 keys */
            continue;
        }
        for (uint64_t p = 0; p < L.P; p++) cursor[p] = part_start[p];
        for (uint64_t i = 0; i < n; i++) {
            const uint64_t at = cursor[orc_hi(L.P, hb[i])]++;
            by_part[at] = h[i];
            if (h128) by_part_hi[at] = hh[i];
        }
        memset(taken, 0, L.P * L.S);

        build_ctx bc = {m, prm->evict_mult};   /* 0: pure greedy, no eviction allowed */
        build_pool bp;
        memset(&bp, 0, sizeof(bp));
        bp.bc = &bc; bp.by_part = by_part; bp.by_part_hi = by_part_hi; bp.part_start = part_start; bp.taken = taken;
        bp.rc = ORC_OK;
        pthread_mutex_init(&bp.lock, NULL);
        int threads = prm->threads < 1 ? 1 : (prm->threads > 256 ? 256 : prm->threads);
        if ((uint64_t)threads > L.P) threads = (int)L.P;
        if (threads == 1) build_worker(&bp);
        else {
            pthread_t tid[256];
            for (int t = 0; t < threads; t++) pthread_create(&tid[t], NULL, build_worker, &bp);
            for (int t = 0; t < threads; t++) pthread_join(tid[t], NULL);
        }
        pthread_mutex_destroy(&bp.lock);
        g_total_evictions += bp.evictions;
        rc = bp.rc;
        if (rc == ORC_OK) rc = build_remap(m, taken, prm->remap == ORC_REMAP_CLEF);
        if (rc == ORC_OK) { *out = m; break; }
        orc_free(m);
        if (rc == ORC_ERR_OOM) break;
        if (rc == ORC_ERR_DUP_KEYS && key_kind == ORC_KEY_U64) break;  /* h = C*k: true duplicates */
        /* ORC_ERR_BUILD, or equal string hashes: try the next seed. */
    }
    free(h); free(by_part); free(hh); free(by_part_hi); free(part_start); free(cursor); free(taken);
    return rc;
}

int orc_build_u64(const uint64_t *keys, uint64_t n, const orc_params *p, orc_mphf **out) {
    return build_common(keys, NULL, NULL, n, p, ORC_KEY_U64, out);
}

int orc_build_bytes(const uint8_t *bytes, const uint64_t *offsets, uint64_t n,
                    const orc_params *p, orc_mphf **out) {
    return build_common(NULL, bytes, offsets, n, p, ORC_KEY_BYTES, out);
}

void orc_free(orc_mphf *m) {
    if (!m) return;
    free(m->pilots); free(m->clef); free(m->vec);
    free(m);
}

/* ------------------------------------------------------------------ */
/* Serialized format (little-endian)                                   */
/* ------------------------------------------------------------------ */
/* 128-byte header:
 *   0 magic "PTRHASH1" | 8 u32 version=1 | 12 u32 key_kind | 16 u32 gamma
 *  20 u32 remap | 24 u32 reduce | 28 u32 flags (bit 0: 128-bit string hash)
 *  32 u64 n | 40 u64 P | 48 u64 S
 *  56 u64 B | 64 u64 C | 72 u64 seed | 80 u64 remap_len | 88 u64 remap_bytes
 *  96 f64 lambda | 104 f64 alpha | 112 u64 pilot_bytes (=P*B) | 120 u64 0
 * then the pilots (P*B bytes) zero-padded to a multiple of 64, then the
 * remap payload (CacheLineEF lines of 64 bytes, or plain entries: u32, or
 * u64 when n > 2^32 and the values no longer fit 32 bits). */

static uint64_t vec_width(uint64_t n) { return n > (1ull << 32) ? 8 : 4; }

static uint64_t pad64(uint64_t v) { return (v + 63) & ~63ull; }

static uint64_t remap_bytes_of(const orc_mphf *m) {
    return m->remap == ORC_REMAP_CLEF ? 64 * m->clef_lines : vec_width(m->L.n) * m->remap_len;
}

uint64_t orc_serialized_size(const orc_mphf *m) {
    return 128 + pad64(m->L.P * m->L.B) + remap_bytes_of(m);
}

int orc_serialize(const orc_mphf *m, uint8_t *buf, uint64_t cap) {
    uint64_t need = orc_serialized_size(m);
    if (cap < need) return ORC_ERR_ARG;
    memset(buf, 0, need);
    memcpy(buf, "PTRHASH1", 8);
    put_u32(buf + 8, 1);
    put_u32(buf + 12, (uint32_t)m->key_kind);
    put_u32(buf + 16, (uint32_t)m->gamma);
    put_u32(buf + 20, (uint32_t)m->remap);
    put_u32(buf + 24, (uint32_t)m->L.reduce);
    put_u32(buf + 28, m->hash128 ? 1u : 0u);
    put_u64(buf + 32, m->L.n);
    put_u64(buf + 40, m->L.P);
    put_u64(buf + 48, m->L.S);
    put_u64(buf + 56, m->L.B);
    put_u64(buf + 64, m->C);
    put_u64(buf + 72, m->seed);
    put_u64(buf + 80, m->remap_len);
    put_u64(buf + 88, remap_bytes_of(m));
    uint64_t lb, ab;
    memcpy(&lb, &m->lambda, 8); memcpy(&ab, &m->alpha, 8);
    put_u64(buf + 96, lb);
    put_u64(buf + 104, ab);
    put_u64(buf + 112, m->L.P * m->L.B);
    memcpy(buf + 128, m->pilots, m->L.P * m->L.B);
    uint8_t *rp = buf + 128 + pad64(m->L.P * m->L.B);
    if (m->remap == ORC_REMAP_CLEF) memcpy(rp, m->clef, 64 * m->clef_lines);
    else if (vec_width(m->L.n) == 8) for (uint64_t j = 0; j < m->remap_len; j++) put_u64(rp + 8 * j, m->vec[j]);
    else for (uint64_t j = 0; j < m->remap_len; j++) put_u32(rp + 4 * j, (uint32_t)m->vec[j]);
    return ORC_OK;
}

int orc_deserialize(const uint8_t *buf, uint64_t len, orc_mphf **out) {
    *out = NULL;
    if (len < 128 || memcmp(buf, "PTRHASH1", 8) != 0 || get_u32(buf + 8) != 1) return ORC_ERR_FORMAT;
    orc_mphf *m = (orc_mphf *)calloc(1, sizeof(orc_mphf));
    if (!m) return ORC_ERR_OOM;
    m->key_kind = (int)get_u32(buf + 12);
    m->gamma = (int)get_u32(buf + 16);
    m->remap = (int)get_u32(buf + 20);
    m->L.reduce = (int)get_u32(buf + 24);
    const uint32_t flags = get_u32(buf + 28);
    m->hash128 = (int)(flags & 1u);
    m->L.n = get_u64(buf + 32);
    m->L.P = get_u64(buf + 40);
    m->L.S = get_u64(buf + 48);
    m->L.B = get_u64(buf + 56);
    m->C = get_u64(buf + 64);
    m->seed = get_u64(buf + 72);
    m->remap_len = get_u64(buf + 80);
    uint64_t rbytes = get_u64(buf + 88);
    uint64_t lb = get_u64(buf + 96), ab = get_u64(buf + 104);
    memcpy(&m->lambda, &lb, 8); memcpy(&m->alpha, &ab, 8);
    uint64_t pb = get_u64(buf + 112);
    int bad = (m->gamma != ORC_GAMMA_LINEAR && m->gamma != ORC_GAMMA_CUBIC) ||
              (m->remap != ORC_REMAP_CLEF && m->remap != ORC_REMAP_VEC) ||
              (m->L.reduce != ORC_REDUCE_POW2 && m->L.reduce != ORC_REDUCE_MOD) ||
              m->L.n == 0 || m->L.P == 0 || m->L.S == 0 || m->L.B == 0 ||
              m->L.n > ORC_MAX_KEYS || m->L.S > 0xFFFFFFFFull || flags > 1u ||
              (m->hash128 && m->key_kind != ORC_KEY_BYTES) ||
              pb != m->L.P * m->L.B || m->L.P * m->L.S < m->L.n ||
              m->remap_len != m->L.P * m->L.S - m->L.n ||
              (m->L.reduce == ORC_REDUCE_POW2 && !is_pow2(m->L.S));
    if (!bad) {
        uint64_t want = m->remap == ORC_REMAP_CLEF
                            ? 64 * ((m->remap_len + ORC_CLEF_PER_LINE - 1) / ORC_CLEF_PER_LINE)
                            : vec_width(m->L.n) * m->remap_len;
        bad = rbytes != want || len < 128 + pad64(pb) + rbytes;
    }
    if (bad) { orc_free(m); return ORC_ERR_FORMAT; }
    m->pilots = (uint8_t *)malloc(pb);
    if (!m->pilots) { orc_free(m); return ORC_ERR_OOM; }
    memcpy(m->pilots, buf + 128, pb);
    const uint8_t *rp = buf + 128 + pad64(pb);
    if (m->remap == ORC_REMAP_CLEF) {
        m->clef_lines = rbytes / 64;
        m->clef = (uint8_t *)malloc(rbytes ? rbytes : 1);
        if (!m->clef) { orc_free(m); return ORC_ERR_OOM; }
        memcpy(m->clef, rp, rbytes);
    } else {
        m->vec = (uint64_t *)malloc((m->remap_len ? m->remap_len : 1) * 8);
        if (!m->vec) { orc_free(m); return ORC_ERR_OOM; }
        if (vec_width(m->L.n) == 8) for (uint64_t j = 0; j < m->remap_len; j++) m->vec[j] = get_u64(rp + 8 * j);
        else for (uint64_t j = 0; j < m->remap_len; j++) m->vec[j] = get_u32(rp + 4 * j);
    }
    *out = m;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Accessors                                                            */
/* ------------------------------------------------------------------ */

void orc_get_layout(const orc_mphf *m, orc_layout *L) { *L = m->L; }
const uint8_t *orc_pilots(const orc_mphf *m) { return m->pilots; }
uint64_t orc_remap_len(const orc_mphf *m) { return m->remap_len; }
void orc_remap_values(const orc_mphf *m, uint64_t *out) {
    for (uint64_t j = 0; j < m->remap_len; j++) out[j] = remap_get(m, j);
}
uint64_t orc_seed(const orc_mphf *m) { return m->seed; }
int orc_remap_kind(const orc_mphf *m) { return m->remap; }
int orc_gamma_kind(const orc_mphf *m) { return m->gamma; }
