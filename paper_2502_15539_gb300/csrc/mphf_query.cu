// Query kernels: MPHF evaluation over device-resident keys.
//
// Per key (Sec. 3.1, Eq. partbucket / Eq. slot; Sec. 3.4):
//   h = C k (u64 keys) or the string hash (byte keys)
//   part = hi(P h), x = lo(P h), b = part B + hi(B gamma(x))
//   p = pilots[b]                       <- the one random HBM access per key
//   s = part S + reduce(h xor C (p xor seed), S)
//   out = s < n ? s : F[s - n]          <- CacheLineEF line, ~1% of keys
//
// Each thread owns K keys of a tile: all K keys are loaded (streaming,
// evict-first), all K bucket indexes computed, then all K pilot bytes are
// requested before any is used, so K gathers per thread are in flight.
#include "mphf_internal.cuh"

namespace ptrhash {

constexpr int kThreads = 256;
constexpr int kKeysPerThread = 8;

// A launch of `blocks` 256-thread CTAs that would not fill one wave at 4
// CTAs per SM runs as twice as many 128-thread CTAs instead.
static bool small_batch(uint64_t blocks) {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        sms[dev] = 0;
        return false;
    }
    return blocks < (uint64_t)sms[dev] * 4;
}

// Eq. partbucket with P, B < 2^32 (true of every structure): 32 x 64-bit products.
template <int GAMMA>
__device__ __forceinline__ uint64_t bucket_of(const View &v, uint64_t h, uint64_t &part) {
    uint64_t x, unused;
    part = mul_hi_lo_32x64((uint32_t)v.P, h, x);   // x = lo(P h): position inside the part
    return part * v.B + mul_hi_lo_32x64((uint32_t)v.B, bucket_fn<GAMMA>(x), unused);
}

template <int REDUCE, int REMAP, bool PHF>
__device__ __forceinline__ uint32_t slot_value(const View &v, uint64_t h, uint64_t part, uint32_t pilot) {
    const uint64_t x = h ^ (v.C * ((uint64_t)pilot ^ v.seed));   // h xor hp(p)
    const uint64_t s = part * v.S + reduce_slot<REDUCE>(v, x);
    if (PHF || s < v.n) return (uint32_t)s;
    const uint32_t j = (uint32_t)(s - v.n);
    if constexpr (REMAP == kRemapClef) return clef_get(static_cast<const uint8_t *>(v.remap), j);
    else return __ldg(static_cast<const uint32_t *>(v.remap) + j);
}

// 64-bit results (any structure; needed once n > 2^32).  The plain remap
// array holds u64 entries exactly when n > 2^32.
template <int REDUCE, int REMAP>
__device__ __forceinline__ uint64_t slot_value_wide(const View &v, uint64_t h, uint64_t part, uint32_t pilot) {
    const uint64_t x = h ^ (v.C * ((uint64_t)pilot ^ v.seed));
    const uint64_t s = part * v.S + reduce_slot<REDUCE>(v, x);
    if (s < v.n) return s;
    const uint64_t j = s - v.n;
    if constexpr (REMAP == kRemapClef) return clef_get64(static_cast<const uint8_t *>(v.remap), j);
    else if (v.n > (1ull << 32)) return __ldg(static_cast<const unsigned long long *>(v.remap) + j);
    else return __ldg(static_cast<const uint32_t *>(v.remap) + j);
}

template <int GAMMA, int REDUCE, int REMAP>
__global__ void __launch_bounds__(kThreads)
query_u64_wide_kernel(const View v, const uint64_t *__restrict__ keys, const uint64_t count,
                      uint64_t *__restrict__ out) {
    constexpr int K = kKeysPerThread;
    const uint64_t tile = (uint64_t)blockIdx.x * (kThreads * K);
    uint64_t h[K], part[K], b[K];
    uint32_t p[K];
#pragma unroll
    for (int q = 0; q < K; q++) {
        const uint64_t i = tile + (uint64_t)q * kThreads + threadIdx.x;
        h[q] = v.C * (i < count ? __ldcs(keys + i) : 0ull);
        b[q] = bucket_of<GAMMA>(v, h[q], part[q]);
    }
#pragma unroll
    for (int q = 0; q < K; q++) {
        const uint64_t i = tile + (uint64_t)q * kThreads + threadIdx.x;
        p[q] = i < count ? __ldg(v.pilots + b[q]) : 0u;
    }
#pragma unroll
    for (int q = 0; q < K; q++) {
        const uint64_t i = tile + (uint64_t)q * kThreads + threadIdx.x;
        if (i < count) __stcs(reinterpret_cast<unsigned long long *>(out) + i,
                              (unsigned long long)slot_value_wide<REDUCE, REMAP>(v, h[q], part[q], p[q]));
    }
}

// VEC: keys 16-byte and out 8-byte aligned; pairs of keys per load / store.
// TPB threads per CTA: 256, or 128 for batches that do not fill one wave of
// 256-thread CTAs (the same 8 K gathers in flight per SM, spread over twice
// as many CTAs, so the SMs share the one wave more evenly).
template <int GAMMA, int REDUCE, int REMAP, bool PHF, bool VEC, int TPB = kThreads>
__global__ void __launch_bounds__(TPB, 1024 / TPB)
query_u64_kernel(const View v, const uint64_t *__restrict__ keys, const uint64_t count,
                 uint32_t *__restrict__ out) {
    constexpr int K = kKeysPerThread;
    const uint64_t tile = (uint64_t)blockIdx.x * (TPB * K);
    uint64_t h[K], part[K], b[K];
    uint32_t p[K];
    if (VEC && tile + TPB * K <= count) {
#pragma unroll
        for (int j = 0; j < K / 2; j++) {
            const uint64_t i = tile + (uint64_t)j * 2 * TPB + 2 * threadIdx.x;
            const uint4 kk = __ldcs(reinterpret_cast<const uint4 *>(keys + i));
            h[2 * j] = v.C * (((uint64_t)kk.y << 32) | kk.x);
            h[2 * j + 1] = v.C * (((uint64_t)kk.w << 32) | kk.z);
        }
#pragma unroll
        for (int q = 0; q < K; q++) b[q] = bucket_of<GAMMA>(v, h[q], part[q]);
#pragma unroll
        for (int q = 0; q < K; q++) p[q] = __ldg(v.pilots + b[q]);
#pragma unroll
        for (int j = 0; j < K / 2; j++) {
            const uint64_t i = tile + (uint64_t)j * 2 * TPB + 2 * threadIdx.x;
            uint2 o;
            o.x = slot_value<REDUCE, REMAP, PHF>(v, h[2 * j], part[2 * j], p[2 * j]);
            o.y = slot_value<REDUCE, REMAP, PHF>(v, h[2 * j + 1], part[2 * j + 1], p[2 * j + 1]);
            __stcs(reinterpret_cast<uint2 *>(out + i), o);
        }
    } else {
#pragma unroll
        for (int q = 0; q < K; q++) {
            const uint64_t i = tile + (uint64_t)q * TPB + threadIdx.x;
            h[q] = v.C * (i < count ? __ldcs(keys + i) : 0ull);
            b[q] = bucket_of<GAMMA>(v, h[q], part[q]);
        }
#pragma unroll
        for (int q = 0; q < K; q++) {
            const uint64_t i = tile + (uint64_t)q * TPB + threadIdx.x;
            p[q] = i < count ? __ldg(v.pilots + b[q]) : 0u;
        }
#pragma unroll
        for (int q = 0; q < K; q++) {
            const uint64_t i = tile + (uint64_t)q * TPB + threadIdx.x;
            if (i < count) out[i] = slot_value<REDUCE, REMAP, PHF>(v, h[q], part[q], p[q]);
        }
    }
}

template <int GAMMA, int REDUCE, int REMAP, bool PHF>
static int launch_u64_t(const View &v, const uint64_t *keys, uint64_t count, uint32_t *out, cudaStream_t s) {
    const uint64_t per_block = (uint64_t)kThreads * kKeysPerThread;
    const uint64_t blocks = (count + per_block - 1) / per_block;
    if (blocks > 0x7FFFFFFFull) { set_error("too many keys for one launch"); return MPHF_ERR_ARG; }
    const bool vec = ((uintptr_t)keys % 16 == 0) && ((uintptr_t)out % 8 == 0);
    if (small_batch(blocks)) {
        const unsigned b2 = (unsigned)(2 * blocks);   // 128-thread CTAs of half the keys
        if (vec) query_u64_kernel<GAMMA, REDUCE, REMAP, PHF, true, 128><<<b2, 128, 0, s>>>(v, keys, count, out);
        else query_u64_kernel<GAMMA, REDUCE, REMAP, PHF, false, 128><<<b2, 128, 0, s>>>(v, keys, count, out);
    } else if (vec) {
        query_u64_kernel<GAMMA, REDUCE, REMAP, PHF, true><<<(unsigned)blocks, kThreads, 0, s>>>(v, keys, count, out);
    } else {
        query_u64_kernel<GAMMA, REDUCE, REMAP, PHF, false><<<(unsigned)blocks, kThreads, 0, s>>>(v, keys, count, out);
    }
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPHF_OK : cuda_fail(e, "query_u64 launch");
}

template <int GAMMA, int REDUCE>
static int dispatch_remap(const Header &h, const View &v, const uint64_t *keys, uint64_t count,
                          uint32_t *out, bool phf, cudaStream_t s) {
    if (phf) return launch_u64_t<GAMMA, REDUCE, kRemapNone, true>(v, keys, count, out, s);
    if (h.remap == MPHF_REMAP_VEC) return launch_u64_t<GAMMA, REDUCE, kRemapVec, false>(v, keys, count, out, s);
    return launch_u64_t<GAMMA, REDUCE, kRemapClef, false>(v, keys, count, out, s);
}

template <int GAMMA, int REDUCE, int REMAP>
static int launch_u64_wide_t(const View &v, const uint64_t *keys, uint64_t count, uint64_t *out, cudaStream_t s) {
    const uint64_t per_block = (uint64_t)kThreads * kKeysPerThread;
    const uint64_t blocks = (count + per_block - 1) / per_block;
    if (blocks > 0x7FFFFFFFull) { set_error("too many keys for one launch"); return MPHF_ERR_ARG; }
    query_u64_wide_kernel<GAMMA, REDUCE, REMAP><<<(unsigned)blocks, kThreads, 0, s>>>(v, keys, count, out);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPHF_OK : cuda_fail(e, "query_u64_wide launch");
}

int launch_query_u64_wide(const Header &h, const View &v, const uint64_t *keys, uint64_t count, uint64_t *out,
                          cudaStream_t s) {
    const bool cubic = h.gamma == MPHF_GAMMA_CUBIC, pow2 = h.reduce == kReducePow2;
    const bool vec = h.remap == MPHF_REMAP_VEC;
#define MPHF_WIDE_CASE(G, R)                                                         \
    return vec ? launch_u64_wide_t<G, R, kRemapVec>(v, keys, count, out, s)      \
               : launch_u64_wide_t<G, R, kRemapClef>(v, keys, count, out, s);
    if (cubic && pow2) { MPHF_WIDE_CASE(MPHF_GAMMA_CUBIC, kReducePow2) }
    if (cubic) { MPHF_WIDE_CASE(MPHF_GAMMA_CUBIC, kReduceMod) }
    if (pow2) { MPHF_WIDE_CASE(MPHF_GAMMA_LINEAR, kReducePow2) }
    MPHF_WIDE_CASE(MPHF_GAMMA_LINEAR, kReduceMod)
#undef MPHF_WIDE_CASE
}

int launch_query_u64(const Header &h, const View &v, const uint64_t *keys, uint64_t count,
                     uint32_t *out, bool phf, cudaStream_t s) {
    const bool cubic = h.gamma == MPHF_GAMMA_CUBIC;
    const bool pow2 = h.reduce == kReducePow2;
    if (cubic && pow2) return dispatch_remap<MPHF_GAMMA_CUBIC, kReducePow2>(h, v, keys, count, out, phf, s);
    if (cubic) return dispatch_remap<MPHF_GAMMA_CUBIC, kReduceMod>(h, v, keys, count, out, phf, s);
    if (pow2) return dispatch_remap<MPHF_GAMMA_LINEAR, kReducePow2>(h, v, keys, count, out, phf, s);
    return dispatch_remap<MPHF_GAMMA_LINEAR, kReduceMod>(h, v, keys, count, out, phf, s);
}

// ------------------------------------------------------------ string keys
constexpr int kStrThreads = 128;                     // strings per tile and threads per block
constexpr int kBlkStage = kStrThreads * 64 + 64;     // staged bytes per block

// One string per thread.  The block's kStrThreads contiguous strings are staged
// through shared memory with 16-byte loads (every byte below the end of the
// whole key buffer may be read; only the chunk crossing that end is read
// byte by byte), then each thread hashes its string from the stage.  A
// block whose bytes do not fit the stage hashes from global memory.
// 16 resident blocks of 128 threads per SM (32 registers, a few bytes
// spilled): many small blocks hide the stage-then-hash latency of each
// block (6 blocks of 256 threads were 26 % slower, 8 of 256 5 % slower).
template <int GAMMA, int REDUCE, int REMAP, bool WIDE, bool H128>
__global__ void __launch_bounds__(kStrThreads, 16)
query_bytes_kernel(const View v, const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                   const uint64_t count, void *__restrict__ out) {
    __shared__ __align__(16) uint8_t stage[kBlkStage];
    const int t = threadIdx.x;
    const uint64_t i0 = (uint64_t)blockIdx.x * kStrThreads;
    const uint64_t last = i0 + kStrThreads < count ? i0 + kStrThreads : count;
    const uint64_t lo = __ldg(offsets + i0), hi = __ldg(offsets + last);
    const uint64_t i = i0 + t;
    const uint64_t a = i < count ? __ldg(offsets + i) : hi;
    const uint64_t e = i < count ? __ldg(offsets + i + 1) : hi;
    const uint64_t base = lo & ~15ull;
    const bool staged = hi - base + 32 <= (uint64_t)kBlkStage;   // + one zeroed chunk
    if (staged) {
        const uint64_t end_all = last < count ? __ldg(offsets + count) : hi;
        const uint32_t nvec = (uint32_t)((hi - base + 15) / 16);
        uint4 *dst = reinterpret_cast<uint4 *>(stage);
        for (uint32_t q = t; q < nvec; q += kStrThreads) {
            const uint64_t c0 = base + 16ull * q;
            if (c0 + 16 <= end_all) {
                dst[q] = __ldcs(reinterpret_cast<const uint4 *>(bytes + c0));
            } else {   // the chunk crossing the end of the key buffer
                uint8_t *d8 = stage + 16 * q;
                for (int k = 0; k < 16; k++) d8[k] = c0 + k < hi ? __ldg(bytes + c0 + k) : 0;
            }
        }
        if (t == 0) dst[nvec] = make_uint4(0, 0, 0, 0);   // words past the last string may be read
        __syncthreads();
    }
    if (i >= count) return;
    uint64_t h[2];   // [0] the slot hash; with H128, [1] the high half, which picks part and bucket
    if (staged) {
        const uint32_t st = (uint32_t)(a - base);
        const uint32_t *w = reinterpret_cast<const uint32_t *>(stage) + (st >> 2);
        hash_string_words_n<H128>([&](uint32_t k) { return w[k]; }, 8 * (st & 3u), (uint32_t)(e - a), v.seed, h);
    } else {
        hash_string_global_n<H128>(bytes, a, e - a, v.seed, h);
    }
    uint64_t part;
    const uint64_t b = bucket_of<GAMMA>(v, H128 ? h[1] : h[0], part);
    const uint32_t p = __ldg(v.pilots + b);
    if constexpr (WIDE) static_cast<uint64_t *>(out)[i] = slot_value_wide<REDUCE, REMAP>(v, h[0], part, p);
    else static_cast<uint32_t *>(out)[i] = slot_value<REDUCE, REMAP, false>(v, h[0], part, p);
}

template <int GAMMA, int REDUCE, int REMAP, bool WIDE>
static int launch_bytes_t(const View &v, bool h128, const uint8_t *bytes, const uint64_t *offsets, uint64_t count,
                          void *out, cudaStream_t s) {
    const uint64_t blocks = (count + kStrThreads - 1) / kStrThreads;
    if (blocks > 0x7FFFFFFFull) { set_error("too many keys for one launch"); return MPHF_ERR_ARG; }
    if ((uintptr_t)bytes % 16) {
        set_error("byte keys need a 16-byte aligned buffer");
        return MPHF_ERR_ARG;
    }
    if (h128)
        query_bytes_kernel<GAMMA, REDUCE, REMAP, WIDE, true><<<(unsigned)blocks, kStrThreads, 0, s>>>(v, bytes, offsets, count, out);
    else
        query_bytes_kernel<GAMMA, REDUCE, REMAP, WIDE, false><<<(unsigned)blocks, kStrThreads, 0, s>>>(v, bytes, offsets, count, out);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPHF_OK : cuda_fail(e, "query_bytes launch");
}

template <bool WIDE>
static int dispatch_bytes(const Header &h, const View &v, const uint8_t *bytes, const uint64_t *offsets,
                          uint64_t count, void *out, cudaStream_t s) {
    const bool cubic = h.gamma == MPHF_GAMMA_CUBIC, pow2 = h.reduce == kReducePow2;
    const bool vec = h.remap == MPHF_REMAP_VEC, h128 = h.hash128 != 0;
#define MPHF_BYTES_CASE(G, R)                                                                  \
    return vec ? launch_bytes_t<G, R, kRemapVec, WIDE>(v, h128, bytes, offsets, count, out, s)     \
               : launch_bytes_t<G, R, kRemapClef, WIDE>(v, h128, bytes, offsets, count, out, s);
    if (cubic && pow2) { MPHF_BYTES_CASE(MPHF_GAMMA_CUBIC, kReducePow2) }
    if (cubic) { MPHF_BYTES_CASE(MPHF_GAMMA_CUBIC, kReduceMod) }
    if (pow2) { MPHF_BYTES_CASE(MPHF_GAMMA_LINEAR, kReducePow2) }
    MPHF_BYTES_CASE(MPHF_GAMMA_LINEAR, kReduceMod)
#undef MPHF_BYTES_CASE
}

int launch_query_bytes(const Header &h, const View &v, const uint8_t *bytes, const uint64_t *offsets,
                       uint64_t count, uint32_t *out, cudaStream_t s) {
    return dispatch_bytes<false>(h, v, bytes, offsets, count, out, s);
}

int launch_query_bytes_wide(const Header &h, const View &v, const uint8_t *bytes, const uint64_t *offsets,
                            uint64_t count, uint64_t *out, cudaStream_t s) {
    return dispatch_bytes<true>(h, v, bytes, offsets, count, out, s);
}

// Key hashes for the builder: h = C k for u64 keys, the string hash above
// for byte keys (one thread per key).
__global__ void hash_keys_kernel(int key_kind, const void *__restrict__ keys,
                                 const uint64_t *__restrict__ offsets, uint64_t n, uint64_t C,
                                 uint64_t seed, uint64_t *__restrict__ out, uint64_t *__restrict__ out_hi) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (key_kind == MPHF_KEY_U64) {
            out[i] = C * __ldg(static_cast<const uint64_t *>(keys) + i);
        } else {
            const uint64_t a = __ldg(offsets + i), e = __ldg(offsets + i + 1);
            uint64_t h[2];
            if (out_hi) {
                hash_string_global_n<true>(static_cast<const uint8_t *>(keys), a, e - a, seed, h);
                out_hi[i] = h[1];
            } else {
                hash_string_global_n<false>(static_cast<const uint8_t *>(keys), a, e - a, seed, h);
            }
            out[i] = h[0];
        }
    }
}

int launch_hash_keys(int key_kind, const void *keys, const uint64_t *offsets, uint64_t n, uint64_t C,
                     uint64_t seed, uint64_t *out, uint64_t *out_hi, int sm_count, cudaStream_t s) {
    const uint64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < (uint64_t)sm_count * 16 ? (want ? want : 1) : (uint64_t)sm_count * 16);
    hash_keys_kernel<<<blocks, 256, 0, s>>>(key_kind, keys, offsets, n, C, seed, out, out_hi);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPHF_OK : cuda_fail(e, "hash keys launch");
}

// ----------------------------------------------------- gather roofline probe
// The same tile shape and key stream as query_u64_kernel; each key picks a
// uniformly random byte of the table by fast range of a mixed key.
template <int TPB>
__global__ void __launch_bounds__(TPB)
gather_probe_kernel(const uint64_t *__restrict__ keys, const uint64_t count, const uint8_t *__restrict__ table,
                    const uint64_t table_bytes, uint32_t *__restrict__ out) {
    constexpr int K = kKeysPerThread;
    constexpr uint64_t kMix = 0x9E3779B97F4A7C15ull;
    const uint64_t tile = (uint64_t)blockIdx.x * (TPB * K);
    uint64_t idx[K];
    uint32_t p[K];
    if (tile + TPB * K <= count) {
#pragma unroll
        for (int j = 0; j < K / 2; j++) {
            const uint64_t i = tile + (uint64_t)j * 2 * TPB + 2 * threadIdx.x;
            const uint4 kk = __ldcs(reinterpret_cast<const uint4 *>(keys + i));
            idx[2 * j] = mul_hi(kMix * (((uint64_t)kk.y << 32) | kk.x), table_bytes);
            idx[2 * j + 1] = mul_hi(kMix * (((uint64_t)kk.w << 32) | kk.z), table_bytes);
        }
#pragma unroll
        for (int q = 0; q < K; q++) p[q] = __ldg(table + idx[q]);
#pragma unroll
        for (int j = 0; j < K / 2; j++) {
            const uint64_t i = tile + (uint64_t)j * 2 * TPB + 2 * threadIdx.x;
            __stcs(reinterpret_cast<uint2 *>(out + i), make_uint2(p[2 * j], p[2 * j + 1]));
        }
    } else {
        for (uint64_t i = tile + threadIdx.x; i < count; i += TPB)
            out[i] = __ldg(table + mul_hi(kMix * __ldcs(keys + i), table_bytes));
    }
}

// The probe matched to the query's own access pattern: keys are replaced by
// precomputed table indexes (the query's bucket indexes for the same key
// stream, mphf_bucket_u64), so the gathers hit the same addresses with the
// same skew; 8 index bytes in and 4 result bytes out per key, as the query.
// An index outside the table reads nothing and gives 0.
template <int TPB>
__global__ void __launch_bounds__(TPB)
gather_probe_at_kernel(const uint64_t *__restrict__ idx, const uint64_t count, const uint8_t *__restrict__ table,
                       const uint64_t table_bytes, uint32_t *__restrict__ out) {
    constexpr int K = kKeysPerThread;
    const uint64_t tile = (uint64_t)blockIdx.x * (TPB * K);
    uint64_t b[K];
    uint32_t p[K];
    if (tile + TPB * K <= count) {
#pragma unroll
        for (int j = 0; j < K / 2; j++) {
            const uint64_t i = tile + (uint64_t)j * 2 * TPB + 2 * threadIdx.x;
            const uint4 kk = __ldcs(reinterpret_cast<const uint4 *>(idx + i));
            b[2 * j] = ((uint64_t)kk.y << 32) | kk.x;
            b[2 * j + 1] = ((uint64_t)kk.w << 32) | kk.z;
        }
#pragma unroll
        for (int q = 0; q < K; q++) p[q] = b[q] < table_bytes ? (uint32_t)__ldg(table + b[q]) : 0u;
#pragma unroll
        for (int j = 0; j < K / 2; j++) {
            const uint64_t i = tile + (uint64_t)j * 2 * TPB + 2 * threadIdx.x;
            __stcs(reinterpret_cast<uint2 *>(out + i), make_uint2(p[2 * j], p[2 * j + 1]));
        }
    } else {
        for (uint64_t i = tile + threadIdx.x; i < count; i += TPB) {
            const uint64_t bi = __ldcs(idx + i);
            out[i] = bi < table_bytes ? (uint32_t)__ldg(table + bi) : 0u;
        }
    }
}

// Global bucket index part B + bucket of each u64 key (Eq. partbucket).
template <int GAMMA>
__global__ void bucket_u64_kernel(const View v, const uint64_t *__restrict__ keys, const uint64_t count,
                                  uint64_t *__restrict__ out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t part;
        __stcs(out + i, (unsigned long long)bucket_of<GAMMA>(v, v.C * __ldcs(keys + i), part));
    }
}

int launch_bucket_u64(const Header &h, const View &v, const uint64_t *keys, uint64_t count, uint64_t *out,
                      int sm_count, cudaStream_t s) {
    const uint64_t want = (count + 255) / 256;
    const unsigned blocks = (unsigned)(want < (uint64_t)sm_count * 16 ? want : (uint64_t)sm_count * 16);
    if (h.gamma == MPHF_GAMMA_CUBIC)
        bucket_u64_kernel<MPHF_GAMMA_CUBIC><<<blocks, 256, 0, s>>>(v, keys, count, out);
    else
        bucket_u64_kernel<MPHF_GAMMA_LINEAR><<<blocks, 256, 0, s>>>(v, keys, count, out);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPHF_OK : cuda_fail(e, "bucket_u64 launch");
}

}  // namespace ptrhash

using namespace ptrhash;

extern "C" int mphf_gather_probe_at(const uint64_t *idx_dev, uint64_t count, const uint8_t *table_dev,
                                    uint64_t table_bytes, uint32_t *out_dev, void *stream) {
    if (count == 0) return MPHF_OK;
    if (!idx_dev || !table_dev || !out_dev || table_bytes == 0 || ((uintptr_t)idx_dev % 16) ||
        ((uintptr_t)out_dev % 8)) {
        set_error("gather probe: indexes 16-byte aligned, out 8-byte aligned, table non-empty");
        return MPHF_ERR_ARG;
    }
    const uint64_t per_block = (uint64_t)kThreads * kKeysPerThread;
    const uint64_t blocks = (count + per_block - 1) / per_block;
    if (blocks > 0x7FFFFFFFull) { set_error("too many keys for one launch"); return MPHF_ERR_ARG; }
    if (small_batch(blocks))
        gather_probe_at_kernel<128><<<(unsigned)(2 * blocks), 128, 0, (cudaStream_t)stream>>>(idx_dev, count, table_dev,
                                                                                          table_bytes, out_dev);
    else
        gather_probe_at_kernel<kThreads><<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(idx_dev, count,
                                                                                            table_dev, table_bytes,
                                                                                            out_dev);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPHF_OK : cuda_fail(e, "gather probe launch");
}

extern "C" int mphf_gather_probe(const uint64_t *keys_dev, uint64_t count, const uint8_t *table_dev,
                                 uint64_t table_bytes, uint32_t *out_dev, void *stream) {
    if (count == 0) return MPHF_OK;
    if (!keys_dev || !table_dev || !out_dev || table_bytes == 0 || ((uintptr_t)keys_dev % 16) ||
        ((uintptr_t)out_dev % 8)) {
        set_error("gather probe: keys 16-byte aligned, out 8-byte aligned, table non-empty");
        return MPHF_ERR_ARG;
    }
    const uint64_t per_block = (uint64_t)kThreads * kKeysPerThread;
    const uint64_t blocks = (count + per_block - 1) / per_block;
    if (blocks > 0x7FFFFFFFull) { set_error("too many keys for one launch"); return MPHF_ERR_ARG; }
    if (small_batch(blocks))
        gather_probe_kernel<128><<<(unsigned)(2 * blocks), 128, 0, (cudaStream_t)stream>>>(keys_dev, count, table_dev,
                                                                                       table_bytes, out_dev);
    else
        gather_probe_kernel<kThreads><<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(keys_dev, count,
                                                                                         table_dev, table_bytes,
                                                                                         out_dev);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPHF_OK : cuda_fail(e, "gather probe launch");
}
