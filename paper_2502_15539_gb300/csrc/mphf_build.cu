// GPU construction of a PtrHash structure (Sec. 3.2 and Sec. 3.4).
//
//   1. hash every key (hash_keys_kernel), or, in shards of whole parts, the
//      keys of one shard's parts (shard_hash_kernel); byte keys past 2^32
//      keys take the 128-bit hash, whose high half picks part and bucket
//   2. radix-sort the 64-bit hashes (CUB; 128-bit ones by (high, low));
//      sorted hashes are grouped by part and, inside a part, by bucket,
//      because part = hi(P h) and the bucket function are monotone in h
//   3. bucket boundaries, duplicate and part-size checks  (bucket_bounds_kernel)
//   4. pilot search, one CTA per part, the part's taken-slot bitvector in
//      shared memory: buckets in order of decreasing size, the smallest pilot
//      whose keys land on distinct free slots; else the pilot of least
//      weighted collisions (weight s^2 for a key of a bucket of size s),
//      evicting the colliding buckets, never one of the 16 most recently
//      placed unless that blocks every pilot; a part fails after
//      evict_mult * S evictions                              (pilot_search_kernel)
//   5. remap: the R taken slots >= n in order go to the R free slots < n in
//      order, F[q - n]; other entries repeat their predecessor; CacheLineEF
//      encoding of F, or a plain array (u32, u64 past 2^32 keys) if a line's
//      span does not fit.
// A failed part or equal string hashes restart from step 1 with seed + 1.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <atomic>
#include <mutex>
#include <vector>

#include "mphf_internal.cuh"

namespace ptrhash {

constexpr int kSearchThreads = 256;
constexpr int kMaxBucket = 2048;        // larger buckets fail the part
constexpr int kSmallBucket = 16;        // pilot-parallel search up to this size
constexpr int kPendingCap = 8192;       // deferred or evicted buckets waiting for a pilot
constexpr int kSetSize = 4096;          // slot set for self-collision checks
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint64_t kMaxSlots = 1ull << 20;   // bitvector in shared memory
constexpr uint64_t kMaxShardKeys = (1ull << 31) - 1;   // 32-bit bucket starts, int-sized sorts

enum : uint32_t { kPartOk = 0, kPartNoPilot = 1, kPartEvictCap = 2, kPartBigBucket = 3, kPartPendingFull = 4 };

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

// ---------------------------------------------------------- step 3: bounds
template <int GAMMA>
__device__ __forceinline__ uint64_t global_bucket(uint64_t h, uint64_t P, uint64_t B) {
    const uint64_t part = mul_hi(P, h);
    return part * B + mul_hi(B, bucket_fn<GAMMA>(P * h));
}

// The n sorted bucket hashes all lie in global buckets [gb_lo, gb_hi);
// bstart[b - gb_lo] = index of the first of them in bucket b, for gb_lo <= b
// <= gb_hi.  With 128-bit hashes, sorted_lo holds the low halves (the keys
// are sorted by (high, low)) and a duplicate is an equal pair.
template <int GAMMA>
__global__ void bucket_bounds_kernel(const uint64_t *__restrict__ sorted, const uint64_t *__restrict__ sorted_lo,
                                     uint64_t n, uint64_t P, uint64_t B, uint64_t gb_lo, uint64_t gb_hi,
                                     uint32_t *__restrict__ bstart, uint32_t *__restrict__ dup) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t hi_b = i < n ? global_bucket<GAMMA>(sorted[i], P, B) : gb_hi;
        const uint64_t lo_b = i > 0 ? global_bucket<GAMMA>(sorted[i - 1], P, B) + 1 : gb_lo;
        for (uint64_t b = lo_b; b <= hi_b; b++) bstart[b - gb_lo] = (uint32_t)i;
        if (i > 0 && i < n && sorted[i] == sorted[i - 1] && (!sorted_lo || sorted_lo[i] == sorted_lo[i - 1]))
            *dup = 1;
    }
}

// Parts [0, nparts) of the bstart array (relative to its first part).
__global__ void part_size_kernel(const uint32_t *__restrict__ bstart, uint64_t nparts, uint64_t B, uint64_t S,
                                 uint32_t *__restrict__ overfull) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nparts; p += (uint64_t)gridDim.x * blockDim.x)
        if (bstart[(p + 1) * B] - bstart[p * B] > S) *overfull = 1;
}

// One shard of the keys: the hashes of the keys whose part lies in
// [part_lo, part_hi), appended in any order (they are sorted next).  At
// most `cap` are stored; more raise *overflow (some part then holds more
// than S keys).  h = C k for u64 keys, the string hash for byte keys; with
// out_hi, the 128-bit string hash, whose high half (out_hi) picks the part.
__global__ void shard_hash_kernel(int key_kind, const void *__restrict__ keys, const uint64_t *__restrict__ offsets,
                                  uint64_t n, uint64_t C, uint64_t seed, uint64_t P, uint64_t part_lo,
                                  uint64_t part_hi, uint64_t *__restrict__ out, uint64_t *__restrict__ out_hi,
                                  uint64_t cap, unsigned long long *__restrict__ count,
                                  uint32_t *__restrict__ overflow) {
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // Every lane of a warp runs the same number of iterations.
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (uint64_t w = first; w < n; w += stride) {
        const uint64_t i = w + lane;
        uint64_t h[2] = {0, 0};
        bool keep = false;
        if (i < n) {
            if (key_kind == MPHF_KEY_U64) {
                h[0] = C * __ldg(static_cast<const uint64_t *>(keys) + i);
            } else {
                const uint64_t a = __ldg(offsets + i), e = __ldg(offsets + i + 1);
                if (out_hi) hash_string_global_n<true>(static_cast<const uint8_t *>(keys), a, e - a, seed, h);
                else hash_string_global_n<false>(static_cast<const uint8_t *>(keys), a, e - a, seed, h);
            }
            const uint64_t part = mul_hi(P, out_hi ? h[1] : h[0]);
            keep = part >= part_lo && part < part_hi;
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
        if (!m) continue;
        unsigned long long base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(0xFFFFFFFFu, base, __ffs(m) - 1);
        if (keep) {
            const uint64_t j = base + __popc(m & ((1u << lane) - 1));
            if (j < cap) {
                out[j] = h[0];
                if (out_hi) out_hi[j] = h[1];
            } else {
                *overflow = 1;
            }
        }
    }
}

// ------------------------------------------------------ step 4: the search
struct SearchArgs {
    const uint64_t *sorted;
    const uint32_t *bstart;
    uint8_t *pilots;
    uint32_t *taken;          // linear bitmap of P*S bits (zeroed)
    uint32_t *owner_scratch;  // gridDim.x * S
    uint64_t *order_scratch;  // gridDim.x * B packed descriptors (bucket | size | key offset)
    uint64_t *ohash_scratch;  // gridDim.x * S hashes in processing order
    uint32_t *status;         // per part
    unsigned long long *evictions;
    uint32_t *next_part;
    uint64_t P, S, B, C, seed, fm, s_mask, evict_cap;
    // Parts [part_begin, part_end) are searched; `sorted` holds their hashes
    // and bstart[b - bbase] indexes it for their global buckets b, with
    // bbase = part_begin * B (one shard of the parts, or all of them).
    uint64_t part_begin, part_end, bbase;
};

template <int REDUCE>
__device__ __forceinline__ uint32_t slot_in_part(const SearchArgs &a, uint64_t x) {
    if constexpr (REDUCE == kReducePow2) return (uint32_t)(mul_hi(a.C, x) & a.s_mask);
    else return (uint32_t)mod_barrett(x, a.fm, a.S);
}

__device__ __forceinline__ bool bit_of(const uint32_t *bits, uint32_t s) { return (bits[s >> 5] >> (s & 31)) & 1u; }

struct SearchShared {
    uint32_t *bits;     // S bits; during preparation, per-warp size counters
    uint32_t *hist;     // kMaxBucket + 1: first processing position of each size
    uint64_t *hcache;   // kMaxBucket hashes of the current bucket
    uint32_t *set;      // kSetSize slot-set entries (generation << 21 | slot);
                        // during preparation, first key offset of each size
    uint32_t *pend;     // kPendingCap waiting buckets (bucket | size << 20)
    uint32_t *np;       // how many
    uint32_t *recent;   // 16
    struct CoopReq *coop;   // block-cooperative pilot scoring (see below)
};

constexpr int kSearchWarps = kSearchThreads / 32;
// Slot owner entries and waiting buckets pack bucket | size << 20.
constexpr uint32_t kOwnerShift = 20, kOwnerMask = (1u << 20) - 1;
__device__ __forceinline__ uint32_t pack_owner(uint32_t b, uint32_t z) { return b | (z << kOwnerShift); }
constexpr uint64_t kPrepWords = (uint64_t)kSearchWarps * (kMaxBucket + 1);   // per-warp size counters

// Processing-order descriptor: bucket (32 bits) | size (12 bits) | offset of
// its first hash in the ordered hash array (20 bits; a part has <= 2^20 keys).
__device__ __forceinline__ uint64_t pack_desc(uint64_t b, uint64_t z, uint64_t koff) {
    return b | (z << 32) | (koff << 44);
}

// Inserts slot s for generation gen; false if it is already in the set.
__device__ __forceinline__ bool set_insert(uint32_t *set, uint32_t s, uint32_t gen) {
    const uint32_t key = (gen << 21) | s;
    uint32_t idx = (s * 2654435761u) & (kSetSize - 1);
    for (int probe = 0; probe < kSetSize; probe++) {
        uint32_t e = set[idx];
        while ((e >> 21) != gen) {               // stale entry of an older generation: free
            const uint32_t prev = atomicCAS(&set[idx], e, key);
            if (prev == e) return true;
            e = prev;
        }
        if ((e & 0x1FFFFFu) == s) return false;
        idx = (idx + 1) & (kSetSize - 1);
    }
    return false;                                 // cannot happen: load <= 1/2
}

__device__ __forceinline__ uint32_t bump_gen(uint32_t gen, uint32_t *set, int lane) {
    if (++gen < 2048) return gen;
    for (int i = lane; i < kSetSize; i += 32) set[i] = 0;
    __syncwarp();
    return 1;
}

__device__ __forceinline__ bool in_recent(const uint32_t *recent, uint32_t b) {
    bool r = false;
#pragma unroll
    for (int i = 0; i < 16; i++) r |= recent[i] == b;
    return r;
}

// Pilot-parallel greedy search for a bucket of s <= kSmallBucket keys: lane
// l tries pilot 32 r + l in round r; the smallest successful pilot wins.
// myh is key `lane`'s hash (lanes >= s hold anything).
template <int REDUCE>
__device__ int greedy_small(const SearchArgs &a, const uint32_t *bits, uint64_t myh, int s, int lane) {
    // s is warp-uniform, so the loops below stop at s for the whole warp
    // (the shuffles included) and sl stays in registers.
    for (int r = 0; r < 8; r++) {
        const uint64_t hp = a.C * ((uint64_t)(32 * r + lane) ^ a.seed);
        uint32_t sl[kSmallBucket];
        bool ok = true;
#pragma unroll
        for (int j = 0; j < kSmallBucket; j++) {
            if (j >= s) break;
            sl[j] = slot_in_part<REDUCE>(a, __shfl_sync(0xFFFFFFFFu, myh, j) ^ hp);
            ok &= !bit_of(bits, sl[j]);
#pragma unroll
            for (int k = 0; k < j; k++) ok &= sl[j] != sl[k];
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, ok);
        if (m) return 32 * r + __ffs(m) - 1;
    }
    return -1;
}

// Greedy search for a large bucket (hashes in sh.hcache).  Lane l tries
// pilot 32 r + l against the taken slots, key after key, until every lane
// has hit a taken slot; the surviving pilots, smallest first, are then
// checked for self-collisions key-parallel through the slot set.  The
// result is the smallest pilot whose keys land on distinct free slots.
template <int REDUCE>
__device__ int greedy_large(const SearchArgs &a, const SearchShared &sh, int s, uint32_t &gen, int lane) {
    for (int r = 0; r < 8; r++) {
        const uint64_t hp = a.C * ((uint64_t)(32 * r + lane) ^ a.seed);
        bool ok = true;
        for (int j = 0; j < s; j++) {
            if ((j & 3) == 0 && !__any_sync(0xFFFFFFFFu, ok)) break;
            if (ok) ok = !bit_of(sh.bits, slot_in_part<REDUCE>(a, sh.hcache[j] ^ hp));
        }
        for (unsigned m = __ballot_sync(0xFFFFFFFFu, ok); m; m &= m - 1) {
            const int p = 32 * r + __ffs(m) - 1;
            const uint64_t hpc = a.C * ((uint64_t)p ^ a.seed);
            gen = bump_gen(gen, sh.set, lane);
            bool bad = false;
            for (int j = lane; j < s; j += 32)
                if (!set_insert(sh.set, slot_in_part<REDUCE>(a, sh.hcache[j] ^ hpc), gen)) bad = true;
            if (!__any_sync(0xFFFFFFFFu, bad)) return p;
        }
    }
    return -1;
}

// Weighted-collision search of a small bucket (s <= MAXS keys, hashes in
// lane j's myh): lane l scores pilot 32 r + l, CH chunks of 32 pilots at a
// time so that the owner loads of CH chunks are in flight together.
// Chunks are taken in increasing pilot order and a later chunk needs a
// strictly lower cost, so ties go to the smaller pilot.
template <int REDUCE, int MAXS, int CH>
__device__ void evict_small(const SearchArgs &a, const SearchShared &sh, const uint32_t *owner, uint64_t myh, int s,
                            int lane, bool use_tabu, uint64_t &best_cost, int &best_p) {
    for (int r0 = 0; r0 < 8; r0 += CH) {
        uint32_t sl[CH][MAXS], oe[CH][MAXS];
        bool ok[CH];
#pragma unroll
        for (int c = 0; c < CH; c++) {
            const uint64_t hp = a.C * ((uint64_t)(32 * (r0 + c) + lane) ^ a.seed);
            ok[c] = true;
#pragma unroll
            for (int j = 0; j < MAXS; j++) {
                if (j >= s) break;
                sl[c][j] = slot_in_part<REDUCE>(a, __shfl_sync(0xFFFFFFFFu, myh, j) ^ hp);
                oe[c][j] = bit_of(sh.bits, sl[c][j]) ? owner[sl[c][j]] : kNone;
#pragma unroll
                for (int k = 0; k < j; k++) ok[c] &= sl[c][j] != sl[c][k];
            }
        }
#pragma unroll
        for (int c = 0; c < CH; c++) {
            uint64_t cost = 0;
#pragma unroll
            for (int j = 0; j < MAXS; j++) {
                if (j >= s) break;
                if (oe[c][j] == kNone) continue;
                if (use_tabu && in_recent(sh.recent, oe[c][j] & kOwnerMask)) ok[c] = false;
                const uint64_t z = oe[c][j] >> kOwnerShift;
                cost += z * z;
            }
            uint64_t cc = ok[c] ? cost : ~0ull;
            int pp = ok[c] ? 32 * (r0 + c) + lane : 0x7FFFFFFF;
            for (int off = 16; off; off >>= 1) {
                const uint64_t oc = __shfl_xor_sync(0xFFFFFFFFu, cc, off);
                const int op = __shfl_xor_sync(0xFFFFFFFFu, pp, off);
                if (oc < cc || (oc == cc && op < pp)) { cc = oc; pp = op; }
            }
            if (cc < best_cost) { best_cost = cc; best_p = pp; }
        }
    }
}

// Least weighted collisions (Sec. 3.2): cost = sum over the bucket's keys
// that hit a taken slot of size(owner)^2; pilots that self-collide or hit
// one of the 16 most recently placed buckets are not allowed.  Ties go to
// the smaller pilot.  Returns -1 if no pilot is allowed.
template <int REDUCE>
__device__ int evict_choice(const SearchArgs &a, const SearchShared &sh, const uint32_t *owner, uint64_t gb0,
                            uint64_t myh, int s, uint32_t &gen, int lane, bool use_tabu) {
    uint64_t best_cost = ~0ull;
    int best_p = -1;
    if (s <= 4) {
        evict_small<REDUCE, 4, 4>(a, sh, owner, myh, s, lane, use_tabu, best_cost, best_p);
        return best_p;
    }
    if (s <= kSmallBucket) {
        evict_small<REDUCE, kSmallBucket, 1>(a, sh, owner, myh, s, lane, use_tabu, best_cost, best_p);
        return best_p;
    }
    for (int p = 0; p < 256; p++) {
        const uint64_t hp = a.C * ((uint64_t)p ^ a.seed);
        gen = bump_gen(gen, sh.set, lane);
        bool bad = false;
        uint64_t cost = 0;
        for (int j = lane; j < s; j += 32) {
            const uint32_t sl = slot_in_part<REDUCE>(a, sh.hcache[j] ^ hp);
            if (!set_insert(sh.set, sl, gen)) bad = true;
            else if (bit_of(sh.bits, sl)) {
                const uint32_t oe = owner[sl];
                if (use_tabu && in_recent(sh.recent, oe & kOwnerMask)) bad = true;
                const uint64_t z = oe >> kOwnerShift;
                cost += z * z;
            }
        }
        bad = __any_sync(0xFFFFFFFFu, bad);
        for (int off = 16; off; off >>= 1) cost += __shfl_xor_sync(0xFFFFFFFFu, cost, off);
        if (!bad && cost < best_cost) { best_cost = cost; best_p = p; }
    }
    return best_p;
}

// ------------------------------------------- block-cooperative pilot scoring
// During the eviction drains between rounds, warp 0 places buckets one by
// one while the other warps would wait at a barrier.  Instead they score
// pilots for it: warp 0 posts a request (the bucket's hashes and what to
// compute) and warp w takes pilots 32 w .. 32 w + 31, so all 256 pilots of
// a greedy search or of a weighted-collision search are tried in one step.
// Warp 0 and the helpers meet at two named barriers per request (all
// threads of the block take part in both).  Warp 0 ends every drain with a
// kCoopDone request, on every return path, which releases the helpers.
// The results are those of greedy_small and evict_small: chunks are taken
// in pilot order and ties go to the smaller pilot.
enum : int { kCoopGreedy = 0, kCoopEvictTabu = 1, kCoopEvict = 2, kCoopLarge = 3, kCoopDone = 4 };
struct CoopReq {
    uint64_t h[kSmallBucket];                  // the bucket's hashes (large buckets: sh.hcache)
    int32_t s, kind;
    unsigned long long cost[kSearchWarps];     // per warp: best cost of its chunk
    int32_t pilot[kSearchWarps];               // per warp: best pilot of its chunk, or -1
    uint32_t mask[kSearchWarps];               // per warp: large-bucket pilots on free slots
};

// Barrier `id` (1 or 2; 0 is __syncthreads) of all kSearchThreads threads,
// entered by a converged warp.
__device__ __forceinline__ void named_barrier(int id) {
    __syncwarp();
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(kSearchThreads) : "memory");
}

// The smallest pilot of chunk w whose keys land on distinct free slots, or -1.
template <int REDUCE>
__device__ int coop_greedy_share(const SearchArgs &a, const uint32_t *bits, const CoopReq &q, int w, int lane) {
    const int s = q.s;
    const uint64_t hp = a.C * ((uint64_t)(32 * w + lane) ^ a.seed);
    uint32_t sl[kSmallBucket];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < kSmallBucket; j++) {
        if (j >= s) break;
        sl[j] = slot_in_part<REDUCE>(a, q.h[j] ^ hp);
        ok &= !bit_of(bits, sl[j]);
#pragma unroll
        for (int k = 0; k < j; k++) ok &= sl[j] != sl[k];
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, ok);
    return m ? 32 * w + __ffs(m) - 1 : -1;
}

// The least weighted-collision pilot of chunk w (cost ~0 if none allowed).
template <int REDUCE>
__device__ void coop_evict_share(const SearchArgs &a, const SearchShared &sh, const uint32_t *owner, const CoopReq &q,
                                 int w, int lane, bool use_tabu, unsigned long long &cost_out, int &pilot_out) {
    const int s = q.s;
    const int p = 32 * w + lane;
    const uint64_t hp = a.C * ((uint64_t)p ^ a.seed);
    uint32_t sl[kSmallBucket], oe[kSmallBucket];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < kSmallBucket; j++) {
        if (j >= s) break;
        sl[j] = slot_in_part<REDUCE>(a, q.h[j] ^ hp);
        oe[j] = bit_of(sh.bits, sl[j]) ? owner[sl[j]] : kNone;
#pragma unroll
        for (int k = 0; k < j; k++) ok &= sl[j] != sl[k];
    }
    uint64_t cost = 0;
#pragma unroll
    for (int j = 0; j < kSmallBucket; j++) {
        if (j >= s) break;
        if (oe[j] == kNone) continue;
        if (use_tabu && in_recent(sh.recent, oe[j] & kOwnerMask)) ok = false;
        const uint64_t z = oe[j] >> kOwnerShift;
        cost += z * z;
    }
    uint64_t cc = ok ? cost : ~0ull;
    int pp = ok ? p : 0x7FFFFFFF;
    for (int off = 16; off; off >>= 1) {
        const uint64_t oc = __shfl_xor_sync(0xFFFFFFFFu, cc, off);
        const int op = __shfl_xor_sync(0xFFFFFFFFu, pp, off);
        if (oc < cc || (oc == cc && op < pp)) { cc = oc; pp = op; }
    }
    cost_out = cc;
    pilot_out = pp;
}

// Large bucket (hashes in sh.hcache): bit l is set if pilot 32 w + l puts
// every key on a free slot (self-collisions are checked afterwards).
template <int REDUCE>
__device__ unsigned coop_large_share(const SearchArgs &a, const SearchShared &sh, int s, int w, int lane) {
    const uint64_t hp = a.C * ((uint64_t)(32 * w + lane) ^ a.seed);
    bool ok = true;
    for (int j = 0; j < s; j++) {
        if ((j & 3) == 0 && !__any_sync(0xFFFFFFFFu, ok)) break;
        if (ok) ok = !bit_of(sh.bits, slot_in_part<REDUCE>(a, sh.hcache[j] ^ hp));
    }
    return __ballot_sync(0xFFFFFFFFu, ok);
}

// Warps 1.. of a drain: score chunks until warp 0 posts kCoopDone.
template <int REDUCE>
__device__ void coop_helper(const SearchArgs &a, const SearchShared &sh, const uint32_t *owner, int warp, int lane) {
    CoopReq &q = *sh.coop;
    for (;;) {
        named_barrier(1);
        const int kind = q.kind;
        if (kind == kCoopDone) return;
        if (kind == kCoopGreedy) {
            const int pl = coop_greedy_share<REDUCE>(a, sh.bits, q, warp, lane);
            if (lane == 0) q.pilot[warp] = pl;
        } else if (kind == kCoopLarge) {
            const unsigned m = coop_large_share<REDUCE>(a, sh, q.s, warp, lane);
            if (lane == 0) q.mask[warp] = m;
        } else {
            unsigned long long c;
            int pl;
            coop_evict_share<REDUCE>(a, sh, owner, q, warp, lane, kind == kCoopEvictTabu, c, pl);
            if (lane == 0) { q.cost[warp] = c; q.pilot[warp] = pl; }
        }
        named_barrier(2);
    }
}

// Warp 0: posts the bucket (lane j holds key j's hash in myh) and a kind.
__device__ __forceinline__ void coop_post(const SearchShared &sh, uint64_t myh, int s, int kind, int lane) {
    CoopReq &q = *sh.coop;
    if (lane < s) q.h[lane] = myh;
    if (lane == 0) { q.s = s; q.kind = kind; }
    __syncwarp();
    named_barrier(1);
}

template <int REDUCE>
__device__ int coop_greedy(const SearchArgs &a, const SearchShared &sh, uint64_t myh, int s, int lane) {
    CoopReq &q = *sh.coop;
    coop_post(sh, myh, s, kCoopGreedy, lane);
    const int mine = coop_greedy_share<REDUCE>(a, sh.bits, q, 0, lane);
    if (lane == 0) q.pilot[0] = mine;
    named_barrier(2);
    for (int w = 0; w < kSearchWarps; w++)
        if (q.pilot[w] >= 0) return q.pilot[w];
    return -1;
}

template <int REDUCE>
__device__ int coop_evict(const SearchArgs &a, const SearchShared &sh, const uint32_t *owner, uint64_t myh, int s,
                          int lane, bool use_tabu) {
    CoopReq &q = *sh.coop;
    coop_post(sh, myh, s, use_tabu ? kCoopEvictTabu : kCoopEvict, lane);
    unsigned long long c;
    int pl;
    coop_evict_share<REDUCE>(a, sh, owner, q, 0, lane, use_tabu, c, pl);
    if (lane == 0) { q.cost[0] = c; q.pilot[0] = pl; }
    named_barrier(2);
    unsigned long long best = ~0ull;
    int best_p = -1;
    for (int w = 0; w < kSearchWarps; w++)
        if (q.cost[w] < best) { best = q.cost[w]; best_p = q.pilot[w]; }
    return best_p;
}

// Large bucket: all warps find the pilots on free slots; warp 0 then checks
// them for self-collisions, smallest first, through the slot set.
template <int REDUCE>
__device__ int coop_greedy_large(const SearchArgs &a, const SearchShared &sh, int s, uint32_t &gen, int lane) {
    CoopReq &q = *sh.coop;
    if (lane == 0) { q.s = s; q.kind = kCoopLarge; }
    named_barrier(1);
    const unsigned mine = coop_large_share<REDUCE>(a, sh, s, 0, lane);
    if (lane == 0) q.mask[0] = mine;
    named_barrier(2);
    for (int w = 0; w < kSearchWarps; w++) {
        for (unsigned m = q.mask[w]; m; m &= m - 1) {
            const int p = 32 * w + __ffs(m) - 1;
            const uint64_t hp = a.C * ((uint64_t)p ^ a.seed);
            gen = bump_gen(gen, sh.set, lane);
            bool bad = false;
            for (int j = lane; j < s; j += 32)
                if (!set_insert(sh.set, slot_in_part<REDUCE>(a, sh.hcache[j] ^ hp), gen)) bad = true;
            if (!__any_sync(0xFFFFFFFFu, bad)) return p;
        }
    }
    return -1;
}

__device__ __forceinline__ void coop_done(const SearchShared &sh, int lane) {
    if (lane == 0) sh.coop->kind = kCoopDone;
    __syncwarp();
    named_barrier(1);
}

// Greedy + hash-evict placement by one warp, over stream positions
// [first, last) and the waiting buckets in shared memory (deferred or
// evicted, largest first; ties go to the waiting bucket).  The hashes of
// the next bucket of the stream are requested while the current one is
// searched.  With COOP the other warps score pilots for buckets of up to
// kSmallBucket keys (they run coop_helper meanwhile).  Returns a status.
template <int REDUCE, bool COOP>
__device__ uint32_t search_serial_body(const SearchArgs &a, const SearchShared &sh, uint32_t *owner,
                                       const uint64_t *order, const uint64_t *ohash, uint32_t first, uint32_t last,
                                       uint64_t p, int lane, unsigned long long &evicted) {
    const uint64_t gb0 = p * a.B;
    uint32_t next = first, np = *sh.np, rpos = 0, gen = 0;
    if (np > (uint32_t)kPendingCap) return kPartPendingFull;
    uint32_t wbase = kNone;          // first position held in the descriptor window
    uint64_t wdesc = 0;              // lane l: descriptor of position wbase + l
    uint32_t pf_pos = kNone;         // position whose first 64 hashes were prefetched
    uint64_t pf_h = 0, pf_h2 = 0;    // lane l: hashes l and l + 32
    for (int i = lane; i < 16; i += 32) sh.recent[i] = kNone;
    for (int i = lane; i < kSetSize; i += 32) sh.set[i] = 0;
    __syncwarp();
    uint32_t status = kPartOk;
    for (;;) {
        if (next < last && (wbase == kNone || next >= wbase + 32)) {
            wbase = next;
            wdesc = next + lane < last ? order[next + lane] : 0;
        }
        const uint64_t od = next < last ? __shfl_sync(0xFFFFFFFFu, wdesc, (next - wbase) & 31) : 0;
        const uint32_t ord_z = (uint32_t)(od >> 32) & 0xFFFu;
        uint32_t best_z = 0, best_i = kNone;
        for (uint32_t i = lane; i < np; i += 32) {
            const uint32_t z = sh.pend[i] >> kOwnerShift;
            if (z > best_z || (z == best_z && i < best_i)) { best_z = z; best_i = i; }
        }
        for (int off = 16; off; off >>= 1) {
            const uint32_t oz = __shfl_xor_sync(0xFFFFFFFFu, best_z, off);
            const uint32_t oi = __shfl_xor_sync(0xFFFFFFFFu, best_i, off);
            if (oz > best_z || (oz == best_z && oi < best_i)) { best_z = oz; best_i = oi; }
        }
        if (next >= last && np == 0) break;
        uint32_t b;
        int s;
        uint64_t myh;
        if (np > 0 && best_z >= ord_z) {
            b = sh.pend[best_i] & kOwnerMask;
            s = (int)best_z;
            __syncwarp();
            if (lane == 0) sh.pend[best_i] = sh.pend[np - 1];
            np--;
            __syncwarp();
            const uint64_t kbase = a.bstart[gb0 - a.bbase + b];
            myh = lane < s ? a.sorted[kbase + lane] : 0;
            if (s > kSmallBucket) {
                for (int j = lane; j < s; j += 32) sh.hcache[j] = a.sorted[kbase + j];
                __syncwarp();
            }
        } else {
            b = (uint32_t)od;
            s = (int)ord_z;
            const uint64_t koff = od >> 44;
            const bool pf = pf_pos == next;
            myh = pf ? pf_h : (lane < s ? ohash[koff + lane] : 0);
            if (s > kSmallBucket) {   // the first 64 hashes may have been prefetched
                if (pf) {
                    if (lane < s) sh.hcache[lane] = pf_h;
                    if (lane + 32 < s) sh.hcache[lane + 32] = pf_h2;
                }
                for (int j = (pf ? 64 : 0) + lane; j < s; j += 32) sh.hcache[j] = ohash[koff + j];
                __syncwarp();
            }
            next++;
        }
        if (next < last && wbase != kNone && next < wbase + 32) {
            const uint64_t d2 = __shfl_sync(0xFFFFFFFFu, wdesc, (next - wbase) & 31);
            const uint32_t z2 = (uint32_t)(d2 >> 32) & 0xFFFu;
            pf_pos = next;
            pf_h = (uint32_t)lane < z2 ? ohash[(d2 >> 44) + lane] : 0;
            pf_h2 = (uint32_t)lane + 32 < z2 ? ohash[(d2 >> 44) + lane + 32] : 0;
        } else {
            pf_pos = kNone;
        }
        const bool coop = COOP && s <= kSmallBucket;
        int chosen = coop                   ? coop_greedy<REDUCE>(a, sh, myh, s, lane)
                     : s <= kSmallBucket    ? greedy_small<REDUCE>(a, sh.bits, myh, s, lane)
                     : COOP                 ? coop_greedy_large<REDUCE>(a, sh, s, gen, lane)
                                            : greedy_large<REDUCE>(a, sh, s, gen, lane);
        if (chosen < 0) {
            chosen = coop ? coop_evict<REDUCE>(a, sh, owner, myh, s, lane, true)
                          : evict_choice<REDUCE>(a, sh, owner, gb0, myh, s, gen, lane, true);
            // The tabu only breaks eviction cycles: when it blocks every pilot
            // that does not self-collide, it is ignored for this bucket.
            if (chosen < 0)
                chosen = coop ? coop_evict<REDUCE>(a, sh, owner, myh, s, lane, false)
                              : evict_choice<REDUCE>(a, sh, owner, gb0, myh, s, gen, lane, false);
            if (chosen < 0) { status = kPartNoPilot; break; }
            const uint64_t hp = a.C * ((uint64_t)chosen ^ a.seed);
            // Up to 32 keys: lane j reads the owner of key j's slot, and that
            // owner's first key and pilot, all at once.  While a slot's bit is
            // still set its owner is the one read here (nothing is placed in
            // this loop), so the evictions below use these values in key order.
            uint32_t sl_l = 0, oe_l = kNone;
            uint64_t ob_l = 0, ohp_l = 0;
            if (s <= 32 && lane < s) {
                sl_l = slot_in_part<REDUCE>(a, (s <= kSmallBucket ? myh : sh.hcache[lane]) ^ hp);
                if (bit_of(sh.bits, sl_l)) {
                    oe_l = owner[sl_l];
                    const uint32_t o = oe_l & kOwnerMask;
                    ob_l = a.bstart[gb0 - a.bbase + o];
                    ohp_l = a.C * ((uint64_t)a.pilots[gb0 + o] ^ a.seed);
                }
            }
            for (int j = 0; j < s; j++) {
                uint32_t sl, oe;
                uint64_t ob, ohp;
                if (s <= 32) {
                    sl = __shfl_sync(0xFFFFFFFFu, sl_l, j);
                    oe = __shfl_sync(0xFFFFFFFFu, oe_l, j);
                    ob = __shfl_sync(0xFFFFFFFFu, ob_l, j);
                    ohp = __shfl_sync(0xFFFFFFFFu, ohp_l, j);
                    if (!bit_of(sh.bits, sl)) continue;    // free, or its owner already evicted
                } else {
                    sl = slot_in_part<REDUCE>(a, sh.hcache[j] ^ hp);
                    if (!bit_of(sh.bits, sl)) continue;
                    oe = owner[sl];
                    ob = a.bstart[gb0 - a.bbase + (oe & kOwnerMask)];
                    ohp = a.C * ((uint64_t)a.pilots[gb0 + (oe & kOwnerMask)] ^ a.seed);
                }
                const uint64_t os = oe >> kOwnerShift;
                for (uint64_t k = lane; k < os; k += 32) {
                    const uint32_t osl = slot_in_part<REDUCE>(a, a.sorted[ob + k] ^ ohp);
                    atomicAnd(&sh.bits[osl >> 5], ~(1u << (osl & 31)));
                }
                if (np >= (uint32_t)kPendingCap) { status = kPartPendingFull; break; }
                if (lane == 0) sh.pend[np] = oe;
                np++;
                evicted++;
                __syncwarp();
            }
            if (status != kPartOk) break;
            if (evicted > a.evict_cap) { status = kPartEvictCap; break; }
        }
        const uint64_t hp = a.C * ((uint64_t)chosen ^ a.seed);
        for (int j = lane; j < s; j += 32) {
            const uint64_t hj = s <= kSmallBucket ? myh : sh.hcache[j];
            const uint32_t sl = slot_in_part<REDUCE>(a, hj ^ hp);
            atomicOr(&sh.bits[sl >> 5], 1u << (sl & 31));
            owner[sl] = pack_owner(b, (uint32_t)s);
        }
        if (lane == 0) {
            a.pilots[gb0 + b] = (uint8_t)chosen;
            sh.recent[rpos] = b;
        }
        rpos = (rpos + 1) & 15;
        __syncwarp();
    }
    __syncwarp();
    if (lane == 0) *sh.np = np;
    __syncwarp();
    return status;
}

template <int REDUCE, bool COOP>
__device__ uint32_t search_serial(const SearchArgs &a, const SearchShared &sh, uint32_t *owner, const uint64_t *order,
                                  const uint64_t *ohash, uint32_t first, uint32_t last, uint64_t p, int lane,
                                  unsigned long long &evicted) {
    const uint32_t st = search_serial_body<REDUCE, COOP>(a, sh, owner, order, ohash, first, last, p, lane, evicted);
    if (COOP) coop_done(sh, lane);   // releases the helpers, whatever the status
    return st;
}

// Greedy placement of small buckets (<= kSmallBucket keys) by every warp,
// in deterministic rounds of kRoundCands candidates (kRoundQ per warp).  In
// a round each candidate bucket finds its smallest free pilot on the same
// snapshot of the bitvector; then a candidate commits its slots only if no
// candidate of lower rank in the round picked any of them (the others
// retry in the next round on the updated bitvector).  The comparison goes
// through a claim table that keeps, per slot picked in the round, the
// smallest rank that picked it.  Buckets with no free pilot at all are
// placed by hash-evict (warp 0, serially, with their cascade) before the
// next round.  Finished candidates take the next buckets of the stream in
// rank order, so the outcome depends only on the input.
constexpr int kRoundQ = 4;                              // candidates per warp
constexpr int kRoundCands = kSearchWarps * kRoundQ;     // per round
constexpr int kClaimBits = kRoundQ <= 4 ? 10 : 11;      // claim table of 2^kClaimBits entries,
constexpr int kClaimSize = 1 << kClaimBits;             // at least twice the slots of a round
static_assert(kClaimSize >= 2 * kRoundCands * kSmallBucket && kRoundCands % 32 == 0, "round shape");

struct RoundShared {
    uint32_t slots[kRoundCands][kSmallBucket];
    int32_t chosen[kRoundCands];     // pilot, -1: none found, -2: no bucket
    uint32_t size[kRoundCands];
    uint32_t pos[kRoundCands];       // stream position of the candidate's bucket
    uint32_t done[kRoundCands];      // committed or deferred this round
    uint32_t claim_slot[kClaimSize]; // slot picked in this round, or kNone
    uint32_t claim_rank[kClaimSize]; // smallest rank that picked it
    uint32_t cursor;
};

// Claim-table entry of slot sl (inserted when `insert`, else looked up; a
// looked-up slot is always present).  The table is at most half full.
__device__ __forceinline__ uint32_t claim_index(RoundShared &rs, uint32_t sl, bool insert) {
    uint32_t idx = (sl * 2654435761u) >> (32 - kClaimBits);
    for (int probe = 0; probe < kClaimSize; probe++) {
        if (insert) {
            const uint32_t prev = atomicCAS(&rs.claim_slot[idx], kNone, sl);
            if (prev == kNone || prev == sl) return idx;
        } else if (rs.claim_slot[idx] == sl) {
            return idx;
        }
        idx = (idx + 1) & (kClaimSize - 1);
    }
    return idx;   // not reached: the table has free entries
}

template <int REDUCE>
__device__ void greedy_rounds(const SearchArgs &a, const SearchShared &sh, RoundShared &rs, uint32_t *owner,
                              const uint64_t *order, const uint64_t *ohash, uint32_t first, uint32_t last,
                              uint64_t p, int warp, int lane, unsigned long long &evicted, uint32_t *status) {
    const uint64_t gb0 = p * a.B;
    if (threadIdx.x == 0) {
        for (int c = 0; c < kRoundCands; c++) rs.pos[c] = first + c < last ? first + c : kNone;
        rs.cursor = first + kRoundCands < last ? first + kRoundCands : last;
    }
    for (int i = threadIdx.x; i < kClaimSize; i += blockDim.x) { rs.claim_slot[i] = kNone; rs.claim_rank[i] = kNone; }
    __syncthreads();
    for (;;) {
        // 1. Search: the warp's candidates, their descriptors and hashes
        //    requested together before any is searched.
        uint64_t d[kRoundQ], myh[kRoundQ];
#pragma unroll
        for (int q = 0; q < kRoundQ; q++) {
            const uint32_t pos = rs.pos[warp * kRoundQ + q];
            d[q] = pos != kNone ? order[pos] : 0;
        }
#pragma unroll
        for (int q = 0; q < kRoundQ; q++) {
            const uint32_t z = (uint32_t)(d[q] >> 32) & 0xFFFu;
            myh[q] = lane < (int)z ? ohash[(d[q] >> 44) + lane] : 0;
        }
#pragma unroll
        for (int q = 0; q < kRoundQ; q++) {
            const int c = warp * kRoundQ + q;
            const uint32_t z = (uint32_t)(d[q] >> 32) & 0xFFFu;
            int chosen = -2;
            if (rs.pos[c] != kNone) {
                chosen = greedy_small<REDUCE>(a, sh.bits, myh[q], (int)z, lane);
                if (chosen >= 0 && lane < (int)z)
                    rs.slots[c][lane] = slot_in_part<REDUCE>(a, myh[q] ^ (a.C * ((uint64_t)chosen ^ a.seed)));
            }
            if (lane == 0) { rs.chosen[c] = chosen; rs.size[c] = z; }
        }
        __syncthreads();
        // No candidate has a bucket left: the phase is over.
        bool any = false;
        for (int c = 0; c < kRoundCands; c++) any |= rs.chosen[c] != -2;
        if (!any) break;
        // 2. Claims: the smallest rank that picked each slot.
#pragma unroll
        for (int q = 0; q < kRoundQ; q++) {
            const int c = warp * kRoundQ + q;
            if (rs.chosen[c] >= 0 && lane < (int)rs.size[c])
                atomicMin(&rs.claim_rank[claim_index(rs, rs.slots[c][lane], true)], (uint32_t)c);
        }
        __syncthreads();
        // 3. Commit the candidates that own every slot they picked.
#pragma unroll
        for (int q = 0; q < kRoundQ; q++) {
            const int c = warp * kRoundQ + q;
            const int chosen = rs.chosen[c];
            const uint32_t z = rs.size[c];
            uint32_t done = 0;
            if (chosen >= 0) {
                const bool mine = lane >= (int)z || rs.claim_rank[claim_index(rs, rs.slots[c][lane], false)] == (uint32_t)c;
                if (__all_sync(0xFFFFFFFFu, mine)) {
                    const uint32_t b = (uint32_t)d[q];
                    if (lane < (int)z) {
                        const uint32_t sl = rs.slots[c][lane];
                        atomicOr(&sh.bits[sl >> 5], 1u << (sl & 31));
                        owner[sl] = pack_owner(b, z);
                    }
                    if (lane == 0) a.pilots[gb0 + b] = (uint8_t)chosen;
                    done = 1;
                }
            } else if (chosen == -1) {
                done = 1;   // deferred below, in rank order
            }
            if (lane == 0) rs.done[c] = done;
        }
        __syncthreads();
        // 4. Deferrals and refills in rank order (warp 0, 32 candidates per
        //    step, ranks from ballots); the claim table is emptied.
        if (warp == 0) {
            for (int c0 = 0; c0 < kRoundCands; c0 += 32) {
                const int c = c0 + lane;
                const bool done = rs.done[c] != 0, deferred = done && rs.chosen[c] == -1;
                const unsigned lt = (1u << lane) - 1;
                const unsigned dm = __ballot_sync(0xFFFFFFFFu, done), fm = __ballot_sync(0xFFFFFFFFu, deferred);
                const uint32_t np0 = *sh.np, cur0 = rs.cursor;
                if (deferred) {
                    const uint32_t i = np0 + __popc(fm & lt);
                    if (i < (uint32_t)kPendingCap) sh.pend[i] = pack_owner((uint32_t)order[rs.pos[c]], rs.size[c]);
                }
                if (done) {
                    const uint64_t nx = (uint64_t)cur0 + __popc(dm & lt);
                    rs.pos[c] = nx < last ? (uint32_t)nx : kNone;
                }
                __syncwarp();
                if (lane == 0) {
                    *sh.np = np0 + __popc(fm);
                    const uint64_t nc = (uint64_t)cur0 + __popc(dm);
                    rs.cursor = nc < last ? (uint32_t)nc : last;
                }
                __syncwarp();
            }
        }
        for (int i = threadIdx.x; i < kClaimSize; i += blockDim.x) { rs.claim_slot[i] = kNone; rs.claim_rank[i] = kNone; }
        __syncthreads();
        // A bucket without a free pilot is placed now, by hash-evict, with
        // the whole cascade of evicted buckets, before the next round.
        if (*sh.np > 0) {
            if (warp == 0) {
                const uint32_t st = search_serial<REDUCE, true>(a, sh, owner, order, ohash, 0, 0, p, lane, evicted);
                if (lane == 0 && st != kPartOk) *status = st;
            } else {
                coop_helper<REDUCE>(a, sh, owner, warp, lane);
            }
            __syncthreads();
            if (*status != kPartOk) break;
        }
    }
    __syncthreads();
}

template <int REDUCE>
__global__ void __launch_bounds__(kSearchThreads, 1) pilot_search_kernel(SearchArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint64_t words = (a.S + 31) / 32;
    const uint64_t bits_words = words > kPrepWords ? words : kPrepWords;
    SearchShared sh;
    sh.hcache = reinterpret_cast<uint64_t *>(smem);
    sh.bits = reinterpret_cast<uint32_t *>(sh.hcache + kMaxBucket);
    sh.hist = sh.bits + bits_words;
    sh.set = sh.hist + (kMaxBucket + 1);
    sh.pend = sh.set + kSetSize;
    sh.recent = sh.pend + kPendingCap;
    __shared__ uint32_t s_part, s_flag, s_nb, s_status, s_np;
    __shared__ RoundShared rs;
    __shared__ CoopReq s_coop;
    sh.np = &s_np;
    sh.coop = &s_coop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *owner = a.owner_scratch + (uint64_t)blockIdx.x * a.S;
    uint64_t *order = a.order_scratch + (uint64_t)blockIdx.x * a.B;
    uint64_t *ohash = a.ohash_scratch + (uint64_t)blockIdx.x * a.S;
    uint32_t *cnt = sh.bits;      // [kSearchWarps][kMaxBucket + 1] during preparation
    uint32_t *kbase = sh.set;     // [kMaxBucket + 1] during preparation
    const uint64_t chunk = (a.B + kSearchWarps - 1) / kSearchWarps;
    for (;;) {
        if (tid == 0) { s_part = atomicAdd(a.next_part, 1u); s_flag = 0; }
        __syncthreads();
        const uint64_t p = a.part_begin + s_part;
        if (p >= a.part_end) break;
        const uint64_t gb0 = p * a.B;
        // 1. Bucket sizes, counted per warp over its own range of buckets.
        for (uint64_t w = tid; w < kPrepWords; w += blockDim.x) cnt[w] = 0;
        __syncthreads();
        const uint64_t lo = warp * chunk, hi = (lo + chunk < a.B ? lo + chunk : a.B);
        for (uint64_t b = lo + lane; b < hi; b += 32) {
            const uint32_t z = a.bstart[gb0 - a.bbase + b + 1] - a.bstart[gb0 - a.bbase + b];
            if (z > (uint32_t)kMaxBucket) s_flag = 1;
            else if (z) atomicAdd(&cnt[warp * (kMaxBucket + 1) + z], 1u);
        }
        __syncthreads();
        if (s_flag) {
            if (tid == 0) a.status[p] = kPartBigBucket;
            __syncthreads();
            continue;
        }
        // 2. Processing order: sizes decreasing; inside a size, warp ranges in
        //    order.  Position and first key offset of every (size, warp).
        if (warp == 0) {
            uint32_t carry_pos = 0, carry_keys = 0;
            for (int c = 0; c * 32 < kMaxBucket; c++) {
                const int z = kMaxBucket - 32 * c - lane;   // >= 1 for every chunk and lane
                uint32_t tot = 0;
                for (int w = 0; w < kSearchWarps; w++) tot += cnt[w * (kMaxBucket + 1) + z];
                uint32_t keys = tot * (uint32_t)z, ip = tot, ik = keys;
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t tp = __shfl_up_sync(0xFFFFFFFFu, ip, off);
                    const uint32_t tk = __shfl_up_sync(0xFFFFFFFFu, ik, off);
                    if (lane >= off) { ip += tp; ik += tk; }
                }
                const uint32_t pos0 = carry_pos + ip - tot, key0 = carry_keys + ik - keys;
                sh.hist[z] = pos0;
                kbase[z] = key0;
                uint32_t run = pos0;
                for (int w = 0; w < kSearchWarps; w++) {
                    const uint32_t cw = cnt[w * (kMaxBucket + 1) + z];
                    cnt[w * (kMaxBucket + 1) + z] = run;
                    run += cw;
                }
                carry_pos += __shfl_sync(0xFFFFFFFFu, ip, 31);
                carry_keys += __shfl_sync(0xFFFFFFFFu, ik, 31);
            }
            if (lane == 0) s_nb = carry_pos;
        }
        __syncthreads();
        // 3. Stable scatter of the descriptors, every warp over its range.
        for (uint64_t base = lo; base < hi; base += 32) {
            const uint64_t b = base + lane;
            const uint32_t z = b < hi ? a.bstart[gb0 - a.bbase + b + 1] - a.bstart[gb0 - a.bbase + b] : 0;
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, z);
            const unsigned rank = __popc(peers & ((1u << lane) - 1));
            uint32_t pos = 0;
            if (z) pos = cnt[warp * (kMaxBucket + 1) + z] + rank;
            __syncwarp();
            if (z) {
                order[pos] = pack_desc(b, z, kbase[z] + (uint64_t)(pos - sh.hist[z]) * z);
                if (rank == 0) cnt[warp * (kMaxBucket + 1) + z] += __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        // 4. The part's hashes in processing order.
        const uint32_t nb = s_nb;
        for (uint32_t pos = tid; pos < nb; pos += blockDim.x) {
            const uint64_t d = order[pos];
            const uint32_t b = (uint32_t)d, z = (uint32_t)(d >> 32) & 0xFFFu;
            const uint64_t koff = d >> 44, src = a.bstart[gb0 - a.bbase + b];
            for (uint32_t k = 0; k < z; k++) ohash[koff + k] = a.sorted[src + k];
        }
        const uint32_t n_large = sh.hist[kSmallBucket];   // positions of buckets > kSmallBucket keys
        for (uint64_t w = tid; w < bits_words; w += blockDim.x) sh.bits[w] = 0;
        if (tid == 0) { s_np = 0; s_status = kPartOk; }
        __syncthreads();
        // Phase 1: the large buckets, serially (warp 0, the other warps
        // scoring pilots for it), with hash-evict.
        unsigned long long ev = 0;
        if (warp == 0) {
            const uint32_t st = search_serial<REDUCE, true>(a, sh, owner, order, ohash, 0, n_large, p, lane, ev);
            if (lane == 0) s_status = st;
        } else {
            coop_helper<REDUCE>(a, sh, owner, warp, lane);
        }
        __syncthreads();
        // Phase 2: the small buckets, every warp, greedy; failures wait.
        if (s_status == kPartOk)
            greedy_rounds<REDUCE>(a, sh, rs, owner, order, ohash, n_large, nb, p, warp, lane, ev, &s_status);
        __syncthreads();
        // Phase 3: what waits, serially, with hash-evict.
        if (s_status == kPartOk) {
            if (warp == 0) {
                const uint32_t st = search_serial<REDUCE, true>(a, sh, owner, order, ohash, nb, nb, p, lane, ev);
                if (lane == 0) s_status = st;
            } else {
                coop_helper<REDUCE>(a, sh, owner, warp, lane);
            }
        }
        if (warp == 0 && lane == 0) {
            a.status[p] = s_status;
            atomicAdd(a.evictions, ev);
        }
        __syncthreads();
        if (s_status == kPartOk) {   // publish the part's slots into the global bitmap
            for (uint64_t w = tid; w < words; w += blockDim.x) {
                const uint32_t word = sh.bits[w];
                if (!word) continue;
                const uint64_t g = p * a.S + 32 * w;
                const uint32_t sh_ = (uint32_t)(g & 31);
                atomicOr(&a.taken[g >> 5], word << sh_);
                if (sh_) atomicOr(&a.taken[(g >> 5) + 1], word >> (32 - sh_));
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ step 5: remap
// Word w of the bitmap covers slots [32 w, 32 w + 32).
__device__ __forceinline__ uint32_t low_mask(uint64_t w, uint64_t n) {   // bits of slots < n
    const uint64_t a = 32 * w;
    if (a + 32 <= n) return 0xFFFFFFFFu;
    if (a >= n) return 0;
    return (1u << (n - a)) - 1;
}
__device__ __forceinline__ uint32_t range_mask(uint64_t w, uint64_t lo, uint64_t hi) {  // slots in [lo, hi)
    const uint64_t a = 32 * w;
    uint32_t m = 0xFFFFFFFFu;
    if (lo > a) m &= lo - a >= 32 ? 0 : ~((1u << (lo - a)) - 1);
    if (hi < a + 32) m &= hi <= a ? 0 : (1u << (hi - a)) - 1;
    return m;
}

__global__ void remap_count_kernel(const uint32_t *__restrict__ taken, uint64_t words, uint64_t n, uint64_t total,
                                   uint32_t *__restrict__ free_cnt, uint32_t *__restrict__ high_cnt) {
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = taken[w];
        free_cnt[w] = __popc(~t & low_mask(w, n));
        high_cnt[w] = __popc(t & range_mask(w, n, total));
    }
}

// L[r] = position of the r-th free slot below n (positions may pass 2^32).
__global__ void free_list_kernel(const uint32_t *__restrict__ taken, uint64_t words, uint64_t n,
                                 const uint32_t *__restrict__ free_rank, uint64_t *__restrict__ L) {
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t m = ~taken[w] & low_mask(w, n);
        uint32_t r = free_rank[w];
        while (m) {
            const int bpos = __ffs(m) - 1;
            L[r++] = 32 * w + bpos;
            m &= m - 1;
        }
    }
}

// F[j] = L[t - 1] with t the number of taken slots in [n, n + j]; entries
// before the first taken slot take L[0]; all zero when R = 0.
__global__ void remap_values_kernel(const uint32_t *__restrict__ taken, const uint32_t *__restrict__ high_rank,
                                    const uint64_t *__restrict__ L, uint64_t n, uint64_t total, uint64_t R,
                                    uint64_t *__restrict__ F) {
    const uint64_t len = total - n;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = n + j, w = q >> 5;
        const uint32_t upto = (q & 31) == 31 ? 0xFFFFFFFFu : (2u << (q & 31)) - 1;
        const uint64_t t = high_rank[w] + __popc(taken[w] & range_mask(w, n, total) & upto);
        F[j] = R ? L[t ? t - 1 : 0] : 0;
    }
}

// One CacheLineEF line per thread (Sec. 3.4, Eq. clef).  Values are below
// 2^40 (the 32-bit offset counts units of 256).
__global__ void clef_encode_kernel(const uint64_t *__restrict__ F, uint64_t len, uint64_t lines,
                                   uint8_t *__restrict__ out, uint32_t *__restrict__ span_fail) {
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < lines; c += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i0 = c * kClefPerLine;
        const uint64_t v0 = F[i0];
        const uint64_t offset = v0 >> 8;
        uint32_t words[4] = {0, 0, 0, 0};
        uint8_t *line = out + 64 * c;
        for (int i = 0; i < kClefPerLine; i++) {
            const uint64_t idx = i0 + i < len ? i0 + i : len - 1;
            const uint64_t v = F[idx];
            const uint64_t bit = i + ((v >> 8) - offset);
            if (bit >= 128) { *span_fail = 1; break; }
            words[bit >> 5] |= 1u << (bit & 31);
            line[20 + i] = (uint8_t)v;
        }
        reinterpret_cast<uint4 *>(line)[0] = make_uint4(words[0], words[1], words[2], words[3]);
        reinterpret_cast<uint32_t *>(line)[4] = (uint32_t)offset;
    }
}

// The plain remap array: u32 entries, or u64 once values reach 2^32.
__global__ void narrow_kernel(const uint64_t *__restrict__ F, uint64_t len, uint32_t *__restrict__ out) {
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += (uint64_t)gridDim.x * blockDim.x)
        out[j] = (uint32_t)F[j];
}

// ------------------------------------------------------------ orchestration
// The builder's own stream-ordered memory pool, one per device.  It keeps
// freed memory while any build runs (so concurrent and back-to-back builds
// reuse it instead of mapping and unmapping pages at every synchronization)
// and is trimmed when the last running build ends.
struct BuildPool {
    std::mutex mu;
    cudaMemPool_t pool[64] = {};
    int active[64] = {};
};
static BuildPool g_build_pool;

static cudaError_t build_pool_enter(int dev, cudaMemPool_t *out) {
    std::lock_guard<std::mutex> lock(g_build_pool.mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_build_pool.pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&g_build_pool.pool[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(g_build_pool.pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
    }
    g_build_pool.active[dev]++;
    *out = g_build_pool.pool[dev];
    return cudaSuccess;
}

// Called once the build's stream is idle (its last synchronization).
static void build_pool_leave(int dev) {
    std::lock_guard<std::mutex> lock(g_build_pool.mu);
    if (--g_build_pool.active[dev] == 0) cudaMemPoolTrimTo(g_build_pool.pool[dev], 0);
}

struct PoolGuard {   // leaves the pool on every return path, after its buffers
    int dev = -1;
    cudaStream_t s = nullptr;
    ~PoolGuard() {
        if (dev < 0) return;
        cudaStreamSynchronize(s);
        build_pool_leave(dev);
    }
};

// Device memory of one build, taken from and returned to the pool on the
// build's stream: neither step synchronizes the device, so builds on
// different streams (from different host threads) overlap.
struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    cudaMemPool_t pool = nullptr;
    DevBuf(cudaStream_t st, cudaMemPool_t pl) : s(st), pool(pl) {}
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { if (p) cudaFreeAsync(p, s); }
    template <class T> T *as() const { return static_cast<T *>(p); }
    cudaError_t alloc(size_t bytes) {   // pool NULL: the device's default pool
        return pool ? cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, pool, s) : cudaMallocAsync(&p, bytes ? bytes : 16, s);
    }
    void *release() { void *q = p; p = nullptr; return q; }
};

struct EventPair {   // timing events of a build, destroyed on every return path
    cudaEvent_t t0 = nullptr, t1 = nullptr;   // the whole build
    cudaEvent_t a = nullptr, b = nullptr;     // one phase
    ~EventPair() {
        for (cudaEvent_t e : {t0, t1, a, b})
            if (e) cudaEventDestroy(e);
    }
    // Milliseconds between a and b, once b has completed.
    double phase_ms() const {
        float ms = 0;
        return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? ms : 0.0;
    }
};

// Dynamic shared memory of pilot_search_kernel for S slots per part.
static size_t search_smem_bytes(uint64_t S) {
    const uint64_t words = (S + 31) / 32;
    const uint64_t bits_words = words > kPrepWords ? words : kPrepWords;
    return kMaxBucket * 8 + bits_words * 4 + (kMaxBucket + 1) * 4 + kSetSize * 4 + kPendingCap * 4 + 16 * 4;
}

static unsigned grid_for(uint64_t work, int sms) {
    const uint64_t want = (work + 255) / 256;
    const uint64_t cap = (uint64_t)sms * 32;
    return (unsigned)(want == 0 ? 1 : (want < cap ? want : cap));
}

// The dynamic shared-memory limit of the search kernel is raised once per
// device, to what the largest part (S = kMaxSlots) needs, so that builds of
// different S running from several threads never lower it under each other.
template <int REDUCE>
static cudaError_t launch_search(const SearchArgs &a, unsigned grid, size_t smem, cudaStream_t s) {
    static std::atomic<uint64_t> opted{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(opted.load() & bit)) {
        e = cudaFuncSetAttribute(pilot_search_kernel<REDUCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)search_smem_bytes(kMaxSlots));
        if (e != cudaSuccess) return e;
        opted.fetch_or(bit);
    }
    pilot_search_kernel<REDUCE><<<grid, kSearchThreads, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

int build_structure(const mphf_params &prm, int key_kind, const void *keys, const uint64_t *offsets, uint64_t n,
                    cudaStream_t s, BuildResult *out) {
    if (!(prm.C & 1)) { set_error("mixing constant C must be odd"); return MPHF_ERR_ARG; }
    if (prm.gamma != MPHF_GAMMA_LINEAR && prm.gamma != MPHF_GAMMA_CUBIC) { set_error("bad gamma"); return MPHF_ERR_ARG; }
    if (prm.remap != MPHF_REMAP_CLEF && prm.remap != MPHF_REMAP_VEC) { set_error("bad remap kind"); return MPHF_ERR_ARG; }
    uint64_t P, S, B;
    int reduce;
    int rc = choose_layout(n, prm.lambda, prm.alpha, prm.slots_override, &P, &S, &B, &reduce);
    if (rc) return rc;
    if (S > kMaxSlots) { set_error("S=%llu above the %llu slots a part can hold", (unsigned long long)S, (unsigned long long)kMaxSlots); return MPHF_ERR_CAPACITY; }
    if (B > kOwnerMask) { set_error("B=%llu buckets per part: lambda too small", (unsigned long long)B); return MPHF_ERR_ARG; }
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    EventPair ev;
    CK(cudaEventCreate(&ev.t0));
    CK(cudaEventCreate(&ev.t1));
    CK(cudaEventCreate(&ev.a));
    CK(cudaEventCreate(&ev.b));
    CK(cudaEventRecord(ev.t0, s));
    double hash_sort_ms = 0, search_ms = 0;

    const uint64_t total = P * S, nbkt = P * B, words = (total + 31) / 32;
    // Shards of whole parts (the in-memory sharding of Appendix B): every
    // shard hashes all keys and keeps, sorts and searches only the hashes of
    // its parts, so the working memory follows the shard, not n.  A part's
    // search sees only its own keys, so the structure does not depend on the
    // sharding.
    uint64_t shard_keys = prm.shard_keys;
    if (shard_keys == 0) {   // automatic: a quarter of the free memory at 24 bytes per key
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        shard_keys = free_b / 4 / 24;
    }
    uint64_t parts_per_shard = (uint64_t)((double)shard_keys * (double)P / (double)n);
    if (parts_per_shard > kMaxShardKeys / S) parts_per_shard = kMaxShardKeys / S;
    if (parts_per_shard < 1) parts_per_shard = 1;
    if (parts_per_shard > P) parts_per_shard = P;
    const uint64_t shards = (P + parts_per_shard - 1) / parts_per_shard;
    const uint64_t max_parts = (P + shards - 1) / shards;    // shard i: parts [P i / shards, P (i+1) / shards)
    const uint64_t cap = shards == 1 ? n : max_parts * S;    // hashes a valid shard can hold
    if (cap > kMaxShardKeys) { set_error("%llu keys in one shard", (unsigned long long)cap); return MPHF_ERR_CAPACITY; }
    const unsigned search_grid = (unsigned)(max_parts < (uint64_t)sms ? max_parts : (uint64_t)sms);
    // Byte keys take the 128-bit hash beyond 2^32 keys or when asked to
    // (Sec. 3.1): its high half picks part and bucket, its low half the slot,
    // and the keys are sorted by (high, low) with two stable radix passes.
    const bool h128 = key_kind == MPHF_KEY_BYTES && (prm.hash128 != 0 || n > (1ull << 32));
    PoolGuard guard;
    cudaMemPool_t pool = nullptr;
    CK(build_pool_enter(dev, &pool));
    guard.dev = dev;
    guard.s = s;
    DevBuf hash(s, pool), sorted(s, pool), hash_hi(s, pool), sorted_hi(s, pool), bstart(s, pool), taken(s, pool),
        owner(s, pool), order(s, pool), ohash(s, pool), status(s, pool), flags(s, pool), cub_tmp(s, pool);
    // The structure's own arrays outlive the build: the default allocator.
    DevBuf pilots(s, nullptr);
    CK(hash.alloc(cap * 8));
    CK(sorted.alloc(cap * 8));
    if (h128) {
        CK(hash_hi.alloc(cap * 8));
        CK(sorted_hi.alloc(cap * 8));
    }
    CK(bstart.alloc((max_parts * B + 1) * 4));
    CK(pilots.alloc((nbkt + 63) & ~63ull));
    CK(taken.alloc((words + 1) * 4));
    CK(owner.alloc((uint64_t)search_grid * S * 4));
    CK(order.alloc((uint64_t)search_grid * B * 8));
    CK(ohash.alloc((uint64_t)search_grid * S * 8));
    CK(status.alloc(P * 4));
    CK(flags.alloc(64));
    size_t sort_tmp = 0;
    if (h128)
        CK(cub::DeviceRadixSort::SortPairs(nullptr, sort_tmp, hash.as<uint64_t>(), sorted.as<uint64_t>(),
                                           hash_hi.as<uint64_t>(), sorted_hi.as<uint64_t>(), cap, 0, 64, s));
    else
        CK(cub::DeviceRadixSort::SortKeys(nullptr, sort_tmp, hash.as<uint64_t>(), sorted.as<uint64_t>(), cap, 0, 64, s));
    CK(cub_tmp.alloc(sort_tmp));
    // [0] dup, [1] overfull, [2] next part, [3] span, [4..5] evictions, [6] shard overflow, [8..9] shard count
    uint32_t *d_flags = flags.as<uint32_t>();

    const size_t smem = search_smem_bytes(S);
    Header h;
    h.n = n; h.P = P; h.S = S; h.B = B; h.C = prm.C; h.gamma = prm.gamma; h.reduce = reduce;
    h.key_kind = key_kind; h.lambda = prm.lambda; h.alpha = prm.alpha; h.remap_len = total - n;
    h.hash128 = h128 ? 1 : 0;
    uint64_t evictions_total = 0;
    bool built = false;
    int last_fail = MPHF_ERR_BUILD_FAILED;
    const int attempts = prm.max_reseeds < 0 ? 1 : prm.max_reseeds + 1;
    for (int attempt = 0; attempt < attempts && !built; attempt++) {
        const uint64_t seed = prm.seed + (uint64_t)attempt;
        h.seed = seed;
        CK(cudaMemsetAsync(taken.p, 0, (words + 1) * 4, s));
        CK(cudaMemsetAsync(pilots.p, 0, nbkt, s));
        bool ok = true;
        for (uint64_t sh = 0; sh < shards && ok; sh++) {
            const uint64_t p_lo = P * sh / shards, p_hi = P * (sh + 1) / shards;
            CK(cudaEventRecord(ev.a, s));
            CK(cudaMemsetAsync(d_flags, 0, 64, s));
            uint64_t m = n;
            if (shards == 1) {
                rc = launch_hash_keys(key_kind, keys, offsets, n, prm.C, seed, hash.as<uint64_t>(),
                                      h128 ? hash_hi.as<uint64_t>() : nullptr, sms, s);
                if (rc) return rc;
            } else {
                shard_hash_kernel<<<grid_for(n, sms), 256, 0, s>>>(
                    key_kind, keys, offsets, n, prm.C, seed, P, p_lo, p_hi, hash.as<uint64_t>(),
                    h128 ? hash_hi.as<uint64_t>() : nullptr, cap,
                    reinterpret_cast<unsigned long long *>(d_flags + 8), d_flags + 6);
                count_launch();
                CK(cudaGetLastError());
                uint32_t fl[4];
                CK(cudaMemcpyAsync(fl, d_flags + 6, 16, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                m = (uint64_t)fl[2] | ((uint64_t)fl[3] << 32);
                if (fl[0]) m = cap + 1;   // too many keys for the shard's parts: reported below as overfull
            }
            uint32_t hf[2] = {0, 0};
            // slot_h: the sorted slot hashes the search reads; bucket_h: the
            // sorted hashes that pick part and bucket (the same array unless 128-bit).
            const uint64_t *slot_h = sorted.as<uint64_t>(), *bucket_h = sorted.as<uint64_t>();
            if (m <= cap) {
                if (h128) {   // by low half, then stably by high half: sorted by (high, low)
                    CK(cub::DeviceRadixSort::SortPairs(cub_tmp.p, sort_tmp, hash.as<uint64_t>(), sorted.as<uint64_t>(),
                                                       hash_hi.as<uint64_t>(), sorted_hi.as<uint64_t>(), m, 0, 64, s));
                    CK(cub::DeviceRadixSort::SortPairs(cub_tmp.p, sort_tmp, sorted_hi.as<uint64_t>(), hash_hi.as<uint64_t>(),
                                                       sorted.as<uint64_t>(), hash.as<uint64_t>(), m, 0, 64, s));
                    count_launch(8);
                    slot_h = hash.as<uint64_t>();
                    bucket_h = hash_hi.as<uint64_t>();
                } else {
                    CK(cub::DeviceRadixSort::SortKeys(cub_tmp.p, sort_tmp, hash.as<uint64_t>(), sorted.as<uint64_t>(), m, 0, 64, s));
                    count_launch(4);
                }
                const uint64_t gb_lo = p_lo * B, gb_hi = p_hi * B;
                const uint64_t *dup_lo = h128 ? slot_h : nullptr;
                if (prm.gamma == MPHF_GAMMA_CUBIC)
                    bucket_bounds_kernel<MPHF_GAMMA_CUBIC><<<grid_for(m + 1, sms), 256, 0, s>>>(
                        bucket_h, dup_lo, m, P, B, gb_lo, gb_hi, bstart.as<uint32_t>(), d_flags);
                else
                    bucket_bounds_kernel<MPHF_GAMMA_LINEAR><<<grid_for(m + 1, sms), 256, 0, s>>>(
                        bucket_h, dup_lo, m, P, B, gb_lo, gb_hi, bstart.as<uint32_t>(), d_flags);
                part_size_kernel<<<grid_for(p_hi - p_lo, sms), 256, 0, s>>>(bstart.as<uint32_t>(), p_hi - p_lo, B, S, d_flags + 1);
                count_launch(2);
                CK(cudaGetLastError());
                CK(cudaEventRecord(ev.b, s));
                CK(cudaMemcpyAsync(hf, d_flags, 8, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                hash_sort_ms += ev.phase_ms();
            } else {
                hf[1] = 1;
            }
            if (hf[0]) {
                last_fail = MPHF_ERR_DUP_KEYS;
                set_error("equal key hashes (duplicate keys)");
                if (key_kind == MPHF_KEY_U64) return MPHF_ERR_DUP_KEYS;   // h = C k: duplicates for sure
                ok = false;
                break;
            }
            if (hf[1]) {
                last_fail = MPHF_ERR_OVERFULL;
                set_error("a part holds more than S=%llu keys", (unsigned long long)S);
                if (key_kind == MPHF_KEY_U64) return MPHF_ERR_OVERFULL;   // the seed does not move u64 keys
                ok = false;
                break;
            }
            SearchArgs a;
            a.sorted = slot_h; a.bstart = bstart.as<uint32_t>(); a.pilots = pilots.as<uint8_t>();
            a.taken = taken.as<uint32_t>(); a.owner_scratch = owner.as<uint32_t>(); a.order_scratch = order.as<uint64_t>();
            a.ohash_scratch = ohash.as<uint64_t>();
            a.status = status.as<uint32_t>();
            a.evictions = reinterpret_cast<unsigned long long *>(d_flags + 4);
            a.next_part = d_flags + 2;
            a.P = P; a.S = S; a.B = B; a.C = prm.C; a.seed = seed; a.s_mask = S - 1;
            a.fm = reduce == kReduceMod ? barrett_constant(S) : 0;
            a.evict_cap = (uint64_t)prm.evict_mult * S;
            a.part_begin = p_lo; a.part_end = p_hi; a.bbase = p_lo * B;
            const unsigned grid = (unsigned)(p_hi - p_lo < (uint64_t)search_grid ? p_hi - p_lo : (uint64_t)search_grid);
            CK(cudaEventRecord(ev.a, s));
            CK(reduce == kReducePow2 ? launch_search<kReducePow2>(a, grid, smem, s)
                                     : launch_search<kReduceMod>(a, grid, smem, s));
            CK(cudaEventRecord(ev.b, s));
            std::vector<uint32_t> st(p_hi - p_lo);
            unsigned long long nev = 0;
            CK(cudaMemcpyAsync(st.data(), status.as<uint32_t>() + p_lo, (p_hi - p_lo) * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(&nev, d_flags + 4, 8, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            search_ms += ev.phase_ms();
            evictions_total += nev;
            uint64_t failed = 0, first_bad = 0;
            for (uint64_t q = 0; q < p_hi - p_lo; q++) if (st[q] != kPartOk) { if (!failed) first_bad = p_lo + q; failed++; }
            if (failed) {
                last_fail = MPHF_ERR_BUILD_FAILED;
                set_error("%llu part(s) failed (first: part %llu, status %u) with seed %llu", (unsigned long long)failed,
                          (unsigned long long)first_bad, st[first_bad - p_lo], (unsigned long long)seed);
                ok = false;
            }
        }
        built = ok;
    }
    if (!built) {
        if (last_fail == MPHF_ERR_BUILD_FAILED && key_kind == MPHF_KEY_U64) {
            // h = C k keeps the structure of lattice-like key sets (arithmetic
            // progressions, multiples of a power of two), which can defeat the
            // search under every seed; random-looking keys do not.
            char msg[512];
            snprintf(msg, sizeof(msg), "%s; every reseed failed: structured u64 keys should first go through "
                     "a bijective 64-bit mixer", mphf_last_error());
            set_error("%s", msg);
        }
        return last_fail;
    }

    // Remap (Sec. 3.4).
    CK(cudaEventRecord(ev.a, s));
    const uint64_t len = total - n;
    DevBuf free_cnt(s, pool), high_cnt(s, pool), free_rank(s, pool), high_rank(s, pool), L(s, pool), F(s, nullptr),
        remap(s, nullptr);
    CK(free_cnt.alloc(words * 4));
    CK(high_cnt.alloc(words * 4));
    CK(free_rank.alloc((words + 1) * 4));
    CK(high_rank.alloc((words + 1) * 4));
    remap_count_kernel<<<grid_for(words, sms), 256, 0, s>>>(taken.as<uint32_t>(), words, n, total,
                                                            free_cnt.as<uint32_t>(), high_cnt.as<uint32_t>());
    count_launch();
    size_t scan_tmp = 0;
    CK(cub::DeviceScan::ExclusiveSum(nullptr, scan_tmp, free_cnt.as<uint32_t>(), free_rank.as<uint32_t>(), words, s));
    DevBuf scan_buf(s, pool);
    CK(scan_buf.alloc(scan_tmp));
    CK(cub::DeviceScan::ExclusiveSum(scan_buf.p, scan_tmp, free_cnt.as<uint32_t>(), free_rank.as<uint32_t>(), words, s));
    CK(cub::DeviceScan::ExclusiveSum(scan_buf.p, scan_tmp, high_cnt.as<uint32_t>(), high_rank.as<uint32_t>(), words, s));
    count_launch(2);
    uint32_t tail[4];
    CK(cudaMemcpyAsync(&tail[0], free_rank.as<uint32_t>() + words - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&tail[1], free_cnt.as<uint32_t>() + words - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&tail[2], high_rank.as<uint32_t>() + words - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&tail[3], high_cnt.as<uint32_t>() + words - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t R_low = (uint64_t)tail[0] + tail[1], R_high = (uint64_t)tail[2] + tail[3];
    if (R_low != R_high) {
        set_error("internal: %llu free slots below n but %llu keys at or above n", (unsigned long long)R_low,
                  (unsigned long long)R_high);
        return MPHF_ERR_BUILD_FAILED;
    }
    CK(L.alloc(R_low * 8));
    CK(F.alloc(len * 8));
    free_list_kernel<<<grid_for(words, sms), 256, 0, s>>>(taken.as<uint32_t>(), words, n, free_rank.as<uint32_t>(), L.as<uint64_t>());
    remap_values_kernel<<<grid_for(len, sms), 256, 0, s>>>(taken.as<uint32_t>(), high_rank.as<uint32_t>(), L.as<uint64_t>(),
                                                           n, total, R_low, F.as<uint64_t>());
    count_launch(2);
    int remap_kind = prm.remap;
    if (remap_kind == MPHF_REMAP_CLEF && len > 0) {
        const uint64_t lines = clef_lines_for(len);
        CK(remap.alloc(lines * 64));
        clef_encode_kernel<<<grid_for(lines, sms), 256, 0, s>>>(F.as<uint64_t>(), len, lines, remap.as<uint8_t>(), d_flags + 3);
        count_launch();
        uint32_t span_fail = 0;
        CK(cudaMemcpyAsync(&span_fail, d_flags + 3, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (span_fail) {               // a line's values span too far: plain array instead
            cudaFreeAsync(remap.release(), s);
            remap_kind = MPHF_REMAP_VEC;
        } else {
            h.remap_bytes = lines * 64;
        }
    } else if (remap_kind == MPHF_REMAP_CLEF) {
        h.remap_bytes = 0;
    }
    if (remap_kind == MPHF_REMAP_VEC) {
        const uint64_t width = vec_entry_bytes(n);
        if (width == 8) {
            remap.p = F.release();
        } else {
            CK(remap.alloc(len * 4));
            narrow_kernel<<<grid_for(len, sms), 256, 0, s>>>(F.as<uint64_t>(), len, remap.as<uint32_t>());
            count_launch();
        }
        h.remap_bytes = len * width;
    }
    h.remap = remap_kind;
    CK(cudaGetLastError());
    CK(cudaEventRecord(ev.t1, s));
    CK(cudaEventSynchronize(ev.t1));
    float ms = 0, remap_ms = 0;
    cudaEventElapsedTime(&ms, ev.t0, ev.t1);
    cudaEventElapsedTime(&remap_ms, ev.a, ev.t1);
    out->hdr = h;
    out->d_pilots = static_cast<uint8_t *>(pilots.release());
    out->d_remap = static_cast<uint8_t *>(remap.p ? remap.release() : nullptr);
    if (!out->d_remap) {
        cudaError_t e = cudaMalloc(&out->d_remap, 64);
        if (e != cudaSuccess) { cudaFree(out->d_pilots); return cuda_fail(e, "remap placeholder"); }
    }
    out->evictions = evictions_total;
    out->build_ms = ms;
    out->hash_sort_ms = hash_sort_ms;
    out->search_ms = search_ms;
    out->remap_ms = remap_ms;
    return MPHF_OK;
}

}  // namespace ptrhash

// ------------------------------------------------- build without allocating
// mphf_build_u64_noalloc: the same construction for small key sets, with all
// device working memory carved out of one fixed, file-scope device array
// instead of cudaMalloc.  The array belongs to this translation unit's
// device module: the CUDA runtime gives it device memory when it loads that
// module on a device, which under lazy module loading (the default) is the
// first call into the builder on that device (this entry point or
// mphf_build), and eagerly at context creation with CUDA_MODULE_LOADING=EAGER.
// From then on the device holds the 8 MiB until its context is destroyed.
#include <string.h>

#include <mutex>

namespace ptrhash {

constexpr uint64_t kNoAllocScratchBytes = 8ull << 20;   // 8 MiB per device
constexpr uint64_t kNoAllocMaxKeys = 65536;
constexpr uint64_t kNoAllocMaxParts = 1024;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
struct NoAllocSlot {
    unsigned long long ctx_id = 0;   // context the address belongs to (0: none yet)
    uint8_t *base = nullptr;
};
static NoAllocSlot g_noalloc[64];

// cuCtxGetId through the runtime's driver entry point, so the library does
// not link libcuda directly.
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

static unsigned long long current_context_id() {
    static CtxGetIdFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<CtxGetIdFn>(p);
    }();
    unsigned long long id = 0;
    if (!fn || fn(nullptr, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array on device `dev`, which must be current
// with its primary context initialized.  In host code the array's name is
// only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device and context and cached; a new context
// on the device (after cudaDeviceReset) gets a fresh lookup.
static int noalloc_scratch(int dev, uint8_t **out) {
    if (dev < 0 || dev >= 64) { set_error("device ordinal %d out of range", dev); return MPHF_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long ctx = current_context_id();
    NoAllocSlot &slot = g_noalloc[dev];
    if (!slot.base || ctx == 0 || ctx != slot.ctx_id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        slot.base = static_cast<uint8_t *>(p);
        slot.ctx_id = ctx;
    }
    *out = slot.base;
    return MPHF_OK;
}

struct Carve {   // bump allocation inside the scratch array
    uint8_t *base;
    uint64_t used = 0, cap;
    template <class T> T *take(uint64_t bytes) {
        const uint64_t off = (used + 255) & ~255ull;
        if (off + bytes > cap) return nullptr;
        used = off + (bytes ? bytes : 1);
        return reinterpret_cast<T *>(base + off);
    }
};

static void put64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void put32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }

static int build_noalloc(const mphf_params &prm, const uint64_t *keys, uint64_t n, cudaStream_t s,
                         uint8_t *out, uint64_t cap, uint64_t *needed) {
    if (n > kNoAllocMaxKeys) {
        set_error("n=%llu is above the %llu keys this entry point supports", (unsigned long long)n,
                  (unsigned long long)kNoAllocMaxKeys);
        return MPHF_ERR_CAPACITY;
    }
    if (!(prm.C & 1)) { set_error("mixing constant C must be odd"); return MPHF_ERR_ARG; }
    if (prm.gamma != MPHF_GAMMA_LINEAR && prm.gamma != MPHF_GAMMA_CUBIC) { set_error("bad gamma"); return MPHF_ERR_ARG; }
    if (prm.remap != MPHF_REMAP_CLEF && prm.remap != MPHF_REMAP_VEC) { set_error("bad remap kind"); return MPHF_ERR_ARG; }
    uint64_t P, S, B;
    int reduce;
    int rc = choose_layout(n, prm.lambda, prm.alpha, prm.slots_override, &P, &S, &B, &reduce);
    if (rc) return rc;
    if (S > kMaxSlots || P > kNoAllocMaxParts || B > kOwnerMask) {
        set_error("layout P=%llu S=%llu exceeds this entry point's limits", (unsigned long long)P, (unsigned long long)S);
        return MPHF_ERR_CAPACITY;
    }
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaSetDevice(dev));   // initializes the device's primary context if needed
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint8_t *base = nullptr;
    rc = noalloc_scratch(dev, &base);
    if (rc) return rc;

    const uint64_t total = P * S, nbkt = P * B, words = (total + 31) / 32, len = total - n;
    const uint64_t lines = clef_lines_for(len);
    const unsigned search_grid = (unsigned)(P < (uint64_t)sms ? P : (uint64_t)sms);
    size_t sort_tmp = 0, scan_tmp = 0;
    CK(cub::DeviceRadixSort::SortKeys(nullptr, sort_tmp, (const uint64_t *)nullptr, (uint64_t *)nullptr, n, 0, 64, s));
    CK(cub::DeviceScan::ExclusiveSum(nullptr, scan_tmp, (const uint32_t *)nullptr, (uint32_t *)nullptr, words, s));
    Carve c{base, 0, kNoAllocScratchBytes};
    uint64_t *hash = c.take<uint64_t>(n * 8), *sorted = c.take<uint64_t>(n * 8);
    void *sort_buf = c.take<void>(sort_tmp), *scan_buf = c.take<void>(scan_tmp);
    uint32_t *bstart = c.take<uint32_t>((nbkt + 1) * 4);
    uint8_t *pilots = c.take<uint8_t>(nbkt);
    uint32_t *taken = c.take<uint32_t>((words + 1) * 4);
    uint32_t *owner = c.take<uint32_t>((uint64_t)search_grid * S * 4);
    uint64_t *order = c.take<uint64_t>((uint64_t)search_grid * B * 8);
    uint64_t *ohash = c.take<uint64_t>((uint64_t)search_grid * S * 8);
    uint32_t *status = c.take<uint32_t>(P * 4);
    uint32_t *flags = c.take<uint32_t>(64);
    uint32_t *free_cnt = c.take<uint32_t>(words * 4), *high_cnt = c.take<uint32_t>(words * 4);
    uint32_t *free_rank = c.take<uint32_t>((words + 1) * 4), *high_rank = c.take<uint32_t>((words + 1) * 4);
    uint64_t *L = c.take<uint64_t>(len * 8), *F = c.take<uint64_t>(len * 8);
    uint32_t *F32 = c.take<uint32_t>(len * 4);
    uint8_t *lines_buf = c.take<uint8_t>(lines * 64);
    if (!lines_buf || !F32 || !F || !L || !high_rank || !free_rank || !high_cnt || !free_cnt || !flags || !status || !order ||
        !ohash || !owner || !taken || !pilots || !bstart || !scan_buf || !sort_buf || !sorted || !hash) {
        set_error("this layout needs more than the %llu-byte scratch array", (unsigned long long)kNoAllocScratchBytes);
        return MPHF_ERR_CAPACITY;
    }

    const size_t smem = search_smem_bytes(S);
    Header h;
    h.n = n; h.P = P; h.S = S; h.B = B; h.C = prm.C; h.gamma = prm.gamma; h.reduce = reduce;
    h.key_kind = MPHF_KEY_U64; h.lambda = prm.lambda; h.alpha = prm.alpha; h.remap_len = len;
    bool built = false;
    int last_fail = MPHF_ERR_BUILD_FAILED;
    const int attempts = prm.max_reseeds < 0 ? 1 : prm.max_reseeds + 1;
    uint32_t st[kNoAllocMaxParts];
    for (int attempt = 0; attempt < attempts && !built; attempt++) {
        const uint64_t seed = prm.seed + (uint64_t)attempt;
        h.seed = seed;
        CK(cudaMemsetAsync(flags, 0, 64, s));
        rc = launch_hash_keys(MPHF_KEY_U64, keys, nullptr, n, prm.C, seed, hash, nullptr, sms, s);
        if (rc) return rc;
        CK(cub::DeviceRadixSort::SortKeys(sort_buf, sort_tmp, hash, sorted, n, 0, 64, s));
        count_launch(4);
        if (prm.gamma == MPHF_GAMMA_CUBIC)
            bucket_bounds_kernel<MPHF_GAMMA_CUBIC><<<grid_for(n + 1, sms), 256, 0, s>>>(sorted, nullptr, n, P, B, 0, P * B, bstart, flags);
        else
            bucket_bounds_kernel<MPHF_GAMMA_LINEAR><<<grid_for(n + 1, sms), 256, 0, s>>>(sorted, nullptr, n, P, B, 0, P * B, bstart, flags);
        part_size_kernel<<<grid_for(P, sms), 256, 0, s>>>(bstart, P, B, S, flags + 1);
        count_launch(2);
        CK(cudaGetLastError());
        uint32_t hf[2];
        CK(cudaMemcpyAsync(hf, flags, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hf[0]) { set_error("equal key hashes (duplicate keys)"); return MPHF_ERR_DUP_KEYS; }
        if (hf[1]) { set_error("a part holds more than S=%llu keys", (unsigned long long)S); return MPHF_ERR_OVERFULL; }
        CK(cudaMemsetAsync(taken, 0, (words + 1) * 4, s));
        CK(cudaMemsetAsync(pilots, 0, nbkt, s));
        SearchArgs a;
        a.sorted = sorted; a.bstart = bstart; a.pilots = pilots; a.taken = taken; a.owner_scratch = owner;
        a.order_scratch = order; a.ohash_scratch = ohash; a.status = status;
        a.evictions = reinterpret_cast<unsigned long long *>(flags + 4);
        a.next_part = flags + 2;
        a.part_begin = 0; a.part_end = P; a.bbase = 0;
        a.P = P; a.S = S; a.B = B; a.C = prm.C; a.seed = seed; a.s_mask = S - 1;
        a.fm = reduce == kReduceMod ? barrett_constant(S) : 0;
        a.evict_cap = (uint64_t)prm.evict_mult * S;
        CK(reduce == kReducePow2 ? launch_search<kReducePow2>(a, search_grid, smem, s)
                                 : launch_search<kReduceMod>(a, search_grid, smem, s));
        CK(cudaMemcpyAsync(st, status, P * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        uint64_t failed = 0;
        for (uint64_t p = 0; p < P; p++) failed += st[p] != kPartOk;
        if (failed) {
            set_error("%llu part(s) failed with seed %llu", (unsigned long long)failed, (unsigned long long)seed);
            continue;
        }
        built = true;
    }
    if (!built) return last_fail;

    remap_count_kernel<<<grid_for(words, sms), 256, 0, s>>>(taken, words, n, total, free_cnt, high_cnt);
    count_launch();
    CK(cub::DeviceScan::ExclusiveSum(scan_buf, scan_tmp, free_cnt, free_rank, words, s));
    CK(cub::DeviceScan::ExclusiveSum(scan_buf, scan_tmp, high_cnt, high_rank, words, s));
    count_launch(2);
    uint32_t tail[4];
    CK(cudaMemcpyAsync(&tail[0], free_rank + words - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&tail[1], free_cnt + words - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&tail[2], high_rank + words - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&tail[3], high_cnt + words - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t R = (uint64_t)tail[0] + tail[1];
    if (R != (uint64_t)tail[2] + tail[3]) { set_error("internal: remap counts differ"); return MPHF_ERR_BUILD_FAILED; }
    free_list_kernel<<<grid_for(words, sms), 256, 0, s>>>(taken, words, n, free_rank, L);
    remap_values_kernel<<<grid_for(len, sms), 256, 0, s>>>(taken, high_rank, L, n, total, R, F);
    count_launch(2);
    narrow_kernel<<<grid_for(len, sms), 256, 0, s>>>(F, len, F32);   // n < 2^32 here: u32 entries
    count_launch();
    h.remap = prm.remap;
    const uint8_t *remap_src = reinterpret_cast<const uint8_t *>(F32);
    h.remap_bytes = len * 4;
    if (prm.remap == MPHF_REMAP_CLEF) {
        h.remap_bytes = lines * 64;
        remap_src = lines_buf;
        if (len > 0) {
            clef_encode_kernel<<<grid_for(lines, sms), 256, 0, s>>>(F, len, lines, lines_buf, flags + 3);
            count_launch();
            uint32_t span_fail = 0;
            CK(cudaMemcpyAsync(&span_fail, flags + 3, 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (span_fail) { h.remap = MPHF_REMAP_VEC; h.remap_bytes = len * 4; remap_src = reinterpret_cast<const uint8_t *>(F32); }
        }
    }
    CK(cudaGetLastError());
    const uint64_t pad_pilots = (nbkt + 63) & ~63ull;
    const uint64_t need = 128 + pad_pilots + h.remap_bytes;
    if (needed) *needed = need;
    if (!out || cap < need) { set_error("output buffer of %llu bytes, %llu needed", (unsigned long long)cap, (unsigned long long)need); return MPHF_ERR_ARG; }
    memset(out, 0, 128 + pad_pilots);
    memcpy(out, "PTRHASH1", 8);
    put32(out + 8, 1);
    put32(out + 12, MPHF_KEY_U64);
    put32(out + 16, (uint32_t)h.gamma);
    put32(out + 20, (uint32_t)h.remap);
    put32(out + 24, (uint32_t)h.reduce);
    put64(out + 32, n); put64(out + 40, P); put64(out + 48, S); put64(out + 56, B);
    put64(out + 64, h.C); put64(out + 72, h.seed); put64(out + 80, len); put64(out + 88, h.remap_bytes);
    uint64_t lb, ab;
    memcpy(&lb, &h.lambda, 8); memcpy(&ab, &h.alpha, 8);
    put64(out + 96, lb); put64(out + 104, ab); put64(out + 112, nbkt);
    CK(cudaMemcpyAsync(out + 128, pilots, nbkt, cudaMemcpyDeviceToHost, s));
    if (h.remap_bytes) CK(cudaMemcpyAsync(out + 128 + pad_pilots, remap_src, h.remap_bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MPHF_OK;
}

}  // namespace ptrhash

extern "C" int mphf_build_u64_noalloc(const mphf_params *params, const uint64_t *keys_dev, uint64_t n,
                                      void *out_host, size_t cap, size_t *needed, void *stream) {
    if (!params || !keys_dev || ((uintptr_t)keys_dev & 7)) {
        ptrhash::set_error("NULL params or keys, or keys not 8-byte aligned");
        return MPHF_ERR_ARG;
    }
    uint64_t need = 0;
    int rc = ptrhash::build_noalloc(*params, keys_dev, n, (cudaStream_t)stream, static_cast<uint8_t *>(out_host),
                                    cap, &need);
    if (needed) *needed = need;
    return rc;
}
