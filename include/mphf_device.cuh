/*
 * mphf_device.cuh -- evaluate a PtrHash structure inside your own kernels.
 *
 * Header-only CUDA device code.  Get a structure's view on the host with
 * mphf_device_view() (include/mphf.h), pass it to your kernel by value, and
 * call mphf_dev::eval_u64 / eval_bytes / eval_hash per key: the result is the
 * same as mphf_query_u64 / mphf_query_bytes on that key, so an application
 * can fuse the lookup into the kernel that produces or consumes its keys
 * (streaming queries inside an application, the direction the paper's
 * conclusion proposes).  The view's device memory belongs to the structure:
 * keep the structure alive while kernels use the view.  The same arithmetic
 * is what libmphf's own kernels run (Sec. 3.1 Eq. partbucket / Eq. slot,
 * Sec. 3.3 gamma, Sec. 3.4 CacheLineEF).
 */
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mphf.h"

namespace mphf_dev {

__device__ __forceinline__ uint64_t mul_hi(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// The high and low halves of the 128-bit product a b for a < 2^32, from two
// 32 x 32 -> 64-bit products: a b = A + Bv 2^32 with A = a lo32(b) and Bv =
// a hi32(b), so the high half is floor((Bv + floor(A / 2^32)) / 2^32), and
// Bv + floor(A / 2^32) < 2^64 because Bv <= (2^32 - 1)^2.  Every structure the
// library builds or loads has P, B < 2^32 (mphf_deserialize rejects others),
// so Eq. partbucket's products hi(P h) and hi(B gamma) take this form.
__device__ __forceinline__ uint64_t mul_hi_lo_32x64(uint32_t a, uint64_t b, uint64_t &lo) {
    const uint64_t A = (uint64_t)a * (uint32_t)b, Bv = (uint64_t)a * (uint32_t)(b >> 32);
    lo = (Bv << 32) + A;
    return (Bv + (A >> 32)) >> 32;
}

// gamma on 64-bit fixed point (Sec. 3.3): gamma_1(x) = x, gamma_3(x) =
// 255/256 (x^2 + x^3)/2 + x/256 with x^2 = hi(x x), x^3 = hi(x^2 x), floors.
template <int GAMMA>
__device__ __forceinline__ uint64_t bucket_fn(uint64_t x) {
    if constexpr (GAMMA == MPHF_GAMMA_LINEAR) {
        return x;
    } else {
        uint64_t sq = mul_hi(x, x);
        uint64_t cube = mul_hi(sq, x);
        uint64_t half = (sq >> 1) + (cube >> 1);
        return half - (half >> 8) + (x >> 8);
    }
}

// x mod S for 2 <= S < 2^32 by Barrett reduction: with M = floor(2^64 / S),
// q = hi(x M) is floor(x / S) or one less (x M / 2^64 > x / S - 1), so
// x - q S lies in [0, 2S) and one conditional subtraction makes it exact.
__device__ __forceinline__ uint64_t mod_barrett(uint64_t x, uint64_t M, uint64_t S) {
    const uint64_t q = mul_hi(x, M);
    uint64_t r = x - q * S;
    if (r >= S) r -= S;
    return r;
}

// Position of the i-th (0-based) set bit of a 32-bit word that has > i set bits.
__device__ __forceinline__ uint32_t select32(uint32_t w, uint32_t i) {
    uint32_t pos = 0, c;
    c = __popc(w & 0xFFFFu); if (i >= c) { i -= c; w >>= 16; pos += 16; }
    c = __popc(w & 0xFFu);   if (i >= c) { i -= c; w >>= 8;  pos += 8; }
    c = __popc(w & 0xFu);    if (i >= c) { i -= c; w >>= 4;  pos += 4; }
    c = __popc(w & 0x3u);    if (i >= c) { i -= c; w >>= 2;  pos += 2; }
    c = w & 1u;              if (i >= c) { pos += 1; }
    return pos;
}

// CacheLineEF lookup (Sec. 3.4): v = 256 (offset + select(i) - i) + low[i].
// Line layout: bytes 0..15 the 128-bit bitmap (two little-endian words),
// 16..19 the offset, 20..63 the low bytes.
__device__ __forceinline__ uint32_t clef_get(const uint8_t *lines, uint32_t j) {
    uint32_t line = j / 44u;
    uint32_t i = j - line * 44u;
    const uint8_t *L = lines + (uint64_t)line * 64;
    uint4 head = __ldg(reinterpret_cast<const uint4 *>(L));        // bitmap words
    uint32_t offset = __ldg(reinterpret_cast<const uint32_t *>(L + 16));
    uint32_t low = __ldg(L + 20 + i);
    uint32_t words[4] = {head.x, head.y, head.z, head.w};
    uint32_t sel = 0, k = i;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        uint32_t c = __popc(words[q]);
        if (k < c) { sel = 32 * q + select32(words[q], k); break; }
        k -= c;
    }
    return 256u * (offset + sel - i) + low;
}

// The same lookup with 64-bit arithmetic, for structures of more than 2^32
// keys (values up to 2^40, remap positions past 2^32).
__device__ __forceinline__ uint64_t clef_get64(const uint8_t *lines, uint64_t j) {
    const uint64_t line = j / 44u;
    const uint32_t i = (uint32_t)(j - line * 44u);
    const uint8_t *L = lines + line * 64;
    const uint4 head = __ldg(reinterpret_cast<const uint4 *>(L));
    const uint64_t offset = __ldg(reinterpret_cast<const uint32_t *>(L + 16));
    const uint64_t low = __ldg(L + 20 + i);
    const uint32_t words[4] = {head.x, head.y, head.z, head.w};
    uint32_t sel = 0, k = i;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const uint32_t c = __popc(words[q]);
        if (k < c) { sel = 32 * q + select32(words[q], k); break; }
        k -= c;
    }
    return 256ull * (offset + sel - i) + low;
}

// ------------------------------------------------------------ string keys
// Project string hash (the paper's GxHash is not specified in it):
//   w_j = little-endian u64 of bytes [8j, 8j+8) zero-padded past len,
//   acc = sum_j fold(w_j xor (seed + j K1)),  h = mix(acc xor len K2 xor seed),
// fold(x) = hi(x K3) xor lo(x K3) of the 128-bit product, mix = splitmix64
// finalizer.  The sum lets every word be hashed on its own.
__device__ __forceinline__ uint64_t str_mix(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}
constexpr uint64_t kStrK1 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStrK2 = 0xC2B2AE3D27D4EB4Full;
constexpr uint64_t kStrK3 = 0xA173621FA8385BE3ull;

__device__ __forceinline__ uint64_t str_fold(uint64_t x) { return mul_hi(x, kStrK3) ^ (x * kStrK3); }

__device__ __forceinline__ uint64_t str_finish(uint64_t acc, uint64_t len, uint64_t seed) {
    return str_mix(acc ^ (len * kStrK2) ^ seed);
}

// 128-bit variant (beyond 2^32 keys, Sec. 3.1): the low half is the hash
// above, the high half the same construction with seed xor K4 and the fold
// constant K5; the high half picks the part and bucket, the low half the slot.
constexpr uint64_t kStrK4 = 0x47523634D9D6709Bull;
constexpr uint64_t kStrK5 = 0x2EF8175451B07575ull;
__device__ __forceinline__ uint64_t str_fold_hi(uint64_t x) { return mul_hi(x, kStrK5) ^ (x * kStrK5); }

// The string hash over 32-bit little-endian words W[0], W[1], ... that hold
// the string from bit `sh` (0, 8, 16 or 24) of W[0] on.  Word j of the
// string is bits [64 j + sh, 64 j + sh + 64) of that sequence: two funnel
// shifts of W[2j], W[2j+1], W[2j+2].  fetch(k) returns W[k]; it is called
// for every k <= 2 ceil(len / 8).  out[0] gets the 64-bit hash and, with
// H128, out[1] the high half of the 128-bit one.  Len is the integer type
// of the length and word indexes (32 bits where the string is known to be
// short).
template <bool H128, class Fetch, class Len>
__device__ __forceinline__ void hash_string_words_n(Fetch fetch, uint32_t sh, Len len, uint64_t seed,
                                                    uint64_t *out) {
    const uint64_t seed_hi = seed ^ kStrK4;
    uint64_t acc = 0, acc_hi = 0, tweak = seed, tweak_hi = seed_hi;
    uint32_t cur = fetch(Len(0));
    const Len full = len >> 3;
    for (Len j = 0; j < full; j++, tweak += kStrK1, tweak_hi += kStrK1) {
        const uint32_t m1 = fetch(2 * j + 1), m2 = fetch(2 * j + 2);
        const uint64_t w = ((uint64_t)__funnelshift_r(m1, m2, sh) << 32) | __funnelshift_r(cur, m1, sh);
        acc += str_fold(w ^ tweak);
        if (H128) acc_hi += str_fold_hi(w ^ tweak_hi);
        cur = m2;
    }
    const uint32_t rem = (uint32_t)len & 7u;
    if (rem) {   // the last, partial word: zero past the end of the string
        const uint32_t m1 = fetch(2 * full + 1), m2 = fetch(2 * full + 2);
        uint64_t w = ((uint64_t)__funnelshift_r(m1, m2, sh) << 32) | __funnelshift_r(cur, m1, sh);
        w &= (1ull << (8 * rem)) - 1;
        acc += str_fold(w ^ tweak);
        if (H128) acc_hi += str_fold_hi(w ^ tweak_hi);
    }
    out[0] = str_finish(acc, (uint64_t)len, seed);
    if (H128) out[1] = str_finish(acc_hi, (uint64_t)len, seed_hi);
}

template <class Fetch, class Len>
__device__ __forceinline__ uint64_t hash_string_words(Fetch fetch, uint32_t sh, Len len, uint64_t seed) {
    uint64_t h[1];
    hash_string_words_n<false>(fetch, sh, len, seed, h);
    return h[0];
}

// The string hash of bytes[a, a + len) in global memory, read as aligned
// 32-bit words; words that hold no byte of the string are not read.
// out[0] = the 64-bit hash; with H128 out[1] = the high half.
template <bool H128>
__device__ __forceinline__ void hash_string_global_n(const uint8_t *bytes, uint64_t a, uint64_t len, uint64_t seed,
                                                     uint64_t *out) {
    const uintptr_t addr = reinterpret_cast<uintptr_t>(bytes + a);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(addr & ~(uintptr_t)3);
    const uint64_t lead = addr & 3;   // bytes of W[0] before the string
    hash_string_words_n<H128>([&](uint64_t k) { return 4 * k < lead + len ? __ldg(w + k) : 0u; },
                              (uint32_t)(8 * lead), len, seed, out);
}

__device__ __forceinline__ uint64_t hash_string_global(const uint8_t *bytes, uint64_t a, uint64_t len,
                                                       uint64_t seed) {
    uint64_t h[1];
    hash_string_global_n<false>(bytes, a, len, seed, h);
    return h[0];
}

// The non-minimal slot (Eq. slot): part S + reduce(hs xor hp(p), S), with
// the part and bucket taken from hb (Eq. partbucket).  hb = hs except for
// 128-bit string hashes.
// The two halves of that: the bucket of hb (and its part), and the slot
// that hs reaches with the bucket's pilot.  Between them sits the one random
// memory access, pilots[bucket].
__device__ __forceinline__ uint64_t bucket_index(const mphf_view_t &v, uint64_t hb, uint64_t &part) {
    uint64_t x, unused;
    part = mul_hi_lo_32x64((uint32_t)v.P, hb, x);   // x: position inside the part, as a fraction of 2^64
    const uint64_t g = v.gamma == MPHF_GAMMA_CUBIC ? bucket_fn<MPHF_GAMMA_CUBIC>(x) : x;
    return part * v.B + mul_hi_lo_32x64((uint32_t)v.B, g, unused);
}

__device__ __forceinline__ uint64_t slot_of_pilot(const mphf_view_t &v, uint64_t hs, uint64_t part, uint32_t pilot) {
    const uint64_t xp = hs ^ (v.C * ((uint64_t)pilot ^ v.seed));
    const uint64_t r = v.reduce == 0 ? (mul_hi(v.C, xp) & v.s_mask) : mod_barrett(xp, v.barrett, v.S);
    return part * v.S + r;
}

__device__ __forceinline__ uint64_t slot_hash2(const mphf_view_t &v, uint64_t hb, uint64_t hs) {
    uint64_t part;
    const uint64_t b = bucket_index(v, hb, part);
    return slot_of_pilot(v, hs, part, __ldg(v.pilots + b));
}

__device__ __forceinline__ uint64_t slot_hash(const mphf_view_t &v, uint64_t h) { return slot_hash2(v, h, h); }

// The MPHF value of a slot: itself, or its remap entry when >= n.
// The 32-bit forms need n <= 2^32; the _wide forms take any structure.
__device__ __forceinline__ uint32_t eval_slot(const mphf_view_t &v, uint64_t s) {
    if (s < v.n) return (uint32_t)s;
    const uint32_t j = (uint32_t)(s - v.n);
    if (v.remap_kind == MPHF_REMAP_CLEF) return clef_get(static_cast<const uint8_t *>(v.remap), j);
    return __ldg(static_cast<const uint32_t *>(v.remap) + j);
}

__device__ __forceinline__ uint64_t eval_slot_wide(const mphf_view_t &v, uint64_t s) {
    if (s < v.n) return s;
    const uint64_t j = s - v.n;
    if (v.remap_kind == MPHF_REMAP_CLEF) return clef_get64(static_cast<const uint8_t *>(v.remap), j);
    if (v.n > (1ull << 32)) return __ldg(static_cast<const unsigned long long *>(v.remap) + j);
    return __ldg(static_cast<const uint32_t *>(v.remap) + j);
}

// The value of a key hash (u64 keys, and strings with the 64-bit hash).
__device__ __forceinline__ uint32_t eval_hash(const mphf_view_t &v, uint64_t h) { return eval_slot(v, slot_hash(v, h)); }
__device__ __forceinline__ uint64_t eval_hash_wide(const mphf_view_t &v, uint64_t h) {
    return eval_slot_wide(v, slot_hash(v, h));
}

// A u64 key (structures built with MPHF_KEY_U64).
__device__ __forceinline__ uint32_t eval_u64(const mphf_view_t &v, uint64_t key) { return eval_hash(v, v.C * key); }

__device__ __forceinline__ uint64_t eval_u64_wide(const mphf_view_t &v, uint64_t key) {
    return eval_hash_wide(v, v.C * key);
}

// K u64 keys at once, for kernels that want several pilot gathers in flight
// per thread: all K buckets are computed, then all K pilots requested, and
// only then are the slots and remap entries resolved.  One key at a time
// leaves a single random access in flight per thread, since each remap
// branch ends the compiler's scheduling region.  Results equal eval_u64
// (eval_u64_wide) key by key.
template <int K>
__device__ __forceinline__ void eval_u64_n(const mphf_view_t &v, const uint64_t (&keys)[K], uint32_t (&out)[K]) {
    uint64_t h[K], part[K], b[K];
    uint32_t p[K];
#pragma unroll
    for (int q = 0; q < K; q++) {
        h[q] = v.C * keys[q];
        b[q] = bucket_index(v, h[q], part[q]);
    }
#pragma unroll
    for (int q = 0; q < K; q++) p[q] = __ldg(v.pilots + b[q]);
#pragma unroll
    for (int q = 0; q < K; q++) out[q] = eval_slot(v, slot_of_pilot(v, h[q], part[q], p[q]));
}

template <int K>
__device__ __forceinline__ void eval_u64_wide_n(const mphf_view_t &v, const uint64_t (&keys)[K], uint64_t (&out)[K]) {
    uint64_t h[K], part[K], b[K];
    uint32_t p[K];
#pragma unroll
    for (int q = 0; q < K; q++) {
        h[q] = v.C * keys[q];
        b[q] = bucket_index(v, h[q], part[q]);
    }
#pragma unroll
    for (int q = 0; q < K; q++) p[q] = __ldg(v.pilots + b[q]);
#pragma unroll
    for (int q = 0; q < K; q++) out[q] = eval_slot_wide(v, slot_of_pilot(v, h[q], part[q], p[q]));
}

// A byte-string key (structures built with MPHF_KEY_BYTES), with the
// structure's 64- or 128-bit string hash.
__device__ __forceinline__ uint64_t slot_bytes(const mphf_view_t &v, const uint8_t *s, uint64_t len) {
    uint64_t h[2];
    if (v.hash128) {
        hash_string_global_n<true>(s, 0, len, v.seed, h);
        return slot_hash2(v, h[1], h[0]);
    }
    hash_string_global_n<false>(s, 0, len, v.seed, h);
    return slot_hash(v, h[0]);
}
__device__ __forceinline__ uint32_t eval_bytes(const mphf_view_t &v, const uint8_t *s, uint64_t len) {
    return eval_slot(v, slot_bytes(v, s, len));
}
__device__ __forceinline__ uint64_t eval_bytes_wide(const mphf_view_t &v, const uint8_t *s, uint64_t len) {
    return eval_slot_wide(v, slot_bytes(v, s, len));
}

}  // namespace mphf_dev
