// Windowed query: large batches of u64 keys against a pilot array larger
// than the L2 cache.
//
// The single-pass kernel (mphf_query.cu) makes one random pilot read per key
// (Sec. 3.1: the one cache line a query touches); past the L2 size nearly
// every such read goes to DRAM, and the query runs at the device's random
// DRAM access rate.  Here the pilot array is cut into W byte ranges
// ("windows") small enough to stay resident in L2, and the keys are streamed
// once per window; a key reads its pilot in the pass of the window that holds
// it, so every pilot read after the first touch of its line is an L2 hit.
// The results are those of Eq. partbucket and Eq. slot, key by key, exactly.
//
//   pass 0      keys -> bucket index b (u32 stream, when a later pass reads
//               it) and the pilot of keys in window 0 (u8 stream)
//   pass 1..W-2 (b, carried pilot) -> carried pilot, filling in window w
//   pass W-1    (key, b, carried pilot) -> the MPHF value (slot, remap)
//
// Sequential traffic per key: 13 B in pass 0, 6 B in each middle pass and
// 17 B in the last, against one random DRAM access in the single pass.
// The last pass reads the key anyway (Eq. slot needs h), so it can compute
// the part and bucket again instead of reading b: 4 B per key less in the
// last pass, and 4 B less in pass 0 when W = 2 (no middle pass reads b).
// That pays where the bucket arithmetic is cheap or hidden: gamma_1 (the
// identity; Fast parameters at n = 1e9, 4 windows: 9.92 against 10.46 ms on
// one GPU) and the fused lookup, whose last pass waits on random table reads
// (27.88 against 28.39 ms).  With gamma_3 the two dependent 64-bit high products sit
// between the key load and the pilot read of a pass that already runs at the
// DRAM limit: 9.71 against 9.19 ms at n = 1e9 (3 windows), 2.02 against 1.85
// ms at n = 3e8 (2 windows), and 40 registers or 8 keys per thread were
// slower still.
// Keys are processed in chunks of at most 2^28, so the scratch streams (6 B
// per key of a chunk, 1.6 GB) are bounded; every chunk re-reads the pilot
// windows once (286 MB per 2^28 keys at n = 1e9, about 1 B per key).
#include "mphf_internal.cuh"

namespace ptrhash {

// Launch shapes (measured at n = 1e9, one 2^28-key chunk per pass: keys per
// thread / resident CTAs per SM): the first pass 8 / 5 (0.77 ms; 8 / 4 took
// 0.81, 4 / 8 0.83), the last pass 4 / 8 (0.95 ms; 8 / 4 took 1.13, 8 / 5
// 1.03).  The last pass has the most arithmetic per key and the most
// streams; more resident warps hide its load latency better than more keys
// per thread.  The middle passes take 8 keys per thread (27 registers, 8 CTAs
// per SM): the same time as 16 or 32 at n = 1e9 (3 windows), 14.84 ms
// against 15.20 (16) and 15.30 (32) at n = 1.4e9 (5 windows).  (With 16 keys
// per thread the middle pass's top stall was a full queue of memory
// instructions.)
constexpr int kWinThreads = 256;
constexpr int kWinFirstKeys = 8;    // keys per thread in the first pass
constexpr int kWinMidKeys = 8;      // keys per thread in the middle passes
constexpr int kWinLastKeys = 4;     // keys per thread in the last pass
constexpr uint64_t kWindowChunkDefault = 1ull << 28;
constexpr uint64_t kWindowMinKeys = 1ull << 24;

// The part and bucket index of Eq. partbucket (32 x 64-bit products, P, B < 2^32).
template <int GAMMA>
__device__ __forceinline__ uint64_t window_bucket(const View &v, uint64_t h, uint64_t &part) {
    uint64_t x, unused;
    part = mul_hi_lo_32x64((uint32_t)v.P, h, x);
    return part * v.B + mul_hi_lo_32x64((uint32_t)v.B, bucket_fn<GAMMA>(x), unused);
}

template <int GAMMA>
__device__ __forceinline__ uint64_t window_bucket(const View &v, uint64_t h) {
    uint64_t part;
    return window_bucket<GAMMA>(v, h, part);
}

__device__ __forceinline__ bool in_window(uint64_t b, uint64_t lo, uint64_t hi) { return b >= lo && b < hi; }

// Pass 0: the pilot of the keys in [blo, bhi), and the bucket index of every
// key when STORE_B.
template <int GAMMA, bool STORE_B>
__global__ void __launch_bounds__(kWinThreads, 5)
window_first_kernel(const View v, const uint64_t *__restrict__ keys, const uint64_t count,
                    uint32_t *__restrict__ b32, uint8_t *__restrict__ q, const uint64_t blo, const uint64_t bhi) {
    constexpr int K = kWinFirstKeys;
    const uint64_t tile = (uint64_t)blockIdx.x * (kWinThreads * K);
    if (tile + kWinThreads * K > count) {
        for (uint64_t i = tile + threadIdx.x; i < count; i += kWinThreads) {
            const uint64_t b = window_bucket<GAMMA>(v, v.C * __ldcs(keys + i));
            if (STORE_B) b32[i] = (uint32_t)b;
            q[i] = in_window(b, blo, bhi) ? __ldg(v.pilots + b) : 0;
        }
        return;
    }
    uint64_t b[K];
    uint32_t p[K];
#pragma unroll
    for (int j = 0; j < K / 2; j++) {
        const uint64_t i = tile + (uint64_t)j * 2 * kWinThreads + 2 * threadIdx.x;
        const uint4 kk = __ldcs(reinterpret_cast<const uint4 *>(keys + i));
        b[2 * j] = window_bucket<GAMMA>(v, v.C * (((uint64_t)kk.y << 32) | kk.x));
        b[2 * j + 1] = window_bucket<GAMMA>(v, v.C * (((uint64_t)kk.w << 32) | kk.z));
    }
#pragma unroll
    for (int k = 0; k < K; k++) p[k] = in_window(b[k], blo, bhi) ? (uint32_t)__ldg(v.pilots + b[k]) : 0u;
#pragma unroll
    for (int j = 0; j < K / 2; j++) {
        const uint64_t i = tile + (uint64_t)j * 2 * kWinThreads + 2 * threadIdx.x;
        if (STORE_B) __stcs(reinterpret_cast<uint2 *>(b32 + i), make_uint2((uint32_t)b[2 * j], (uint32_t)b[2 * j + 1]));
        __stcs(reinterpret_cast<unsigned short *>(q + i), (unsigned short)(p[2 * j] | (p[2 * j + 1] << 8)));
    }
}

// Middle passes: the carried pilot, with the keys of window [blo, bhi) filled in.
__global__ void __launch_bounds__(kWinThreads, 4)
window_mid_kernel(const uint8_t *__restrict__ pilots, const uint32_t *__restrict__ b32, const uint64_t count,
                  const uint8_t *__restrict__ qin, uint8_t *__restrict__ qout, const uint64_t blo, const uint64_t bhi) {
    constexpr int K = kWinMidKeys;
    const uint64_t tile = (uint64_t)blockIdx.x * (kWinThreads * K);
    if (tile + kWinThreads * K > count) {
        for (uint64_t i = tile + threadIdx.x; i < count; i += kWinThreads) {
            const uint32_t b = b32[i];
            qout[i] = in_window(b, blo, bhi) ? __ldg(pilots + b) : qin[i];
        }
        return;
    }
    // Thread t takes keys tile + 4 kWinThreads j + 4 t + e (e < 4): per j one
    // 16-byte bucket load, one 4-byte carried-pilot load and one 4-byte
    // store, each warp access 512 or 128 contiguous bytes.  The carried
    // pilot streams are 16-byte aligned (run_windows lays them out so).
    uint32_t b[K], c[K / 4];
#pragma unroll
    for (int j = 0; j < K / 4; j++) {
        const uint64_t i = tile + (uint64_t)j * 4 * kWinThreads + 4 * threadIdx.x;
        const uint4 bb = __ldcs(reinterpret_cast<const uint4 *>(b32 + i));
        b[4 * j] = bb.x;
        b[4 * j + 1] = bb.y;
        b[4 * j + 2] = bb.z;
        b[4 * j + 3] = bb.w;
        c[j] = __ldcs(reinterpret_cast<const uint32_t *>(qin + i));
    }
    uint32_t o[K / 4] = {};
#pragma unroll
    for (int k = 0; k < K; k++) {
        const uint32_t carried = (c[k >> 2] >> (8 * (k & 3))) & 0xFFu;
        const uint32_t p = in_window(b[k], blo, bhi) ? (uint32_t)__ldg(pilots + b[k]) : carried;
        o[k >> 2] |= p << (8 * (k & 3));
    }
#pragma unroll
    for (int j = 0; j < K / 4; j++) {
        const uint64_t i = tile + (uint64_t)j * 4 * kWinThreads + 4 * threadIdx.x;
        __stcs(reinterpret_cast<uint32_t *>(qout + i), o[j]);
    }
}

// Last pass: the value of every key (Eq. slot, Sec. 3.4 remap), written in
// one of the output forms below.  With RECOMPUTE the part and bucket come
// from the key (Eq. partbucket) and b32 is not read; otherwise the part is
// b / B, taken as hi(b M) with
// M = ceil(2^64 / B), exact for b, B < 2^32 (the error b (M - 2^64 / B) /
// 2^64 < 2^-32 < 1 / B cannot carry the quotient over an integer).
// hp(p) = C (p xor seed) comes from a table of the 256 pilot values in
// shared memory.
//   kOutMphf32  u32 MPHF values (n <= 2^32)
//   kOutPhf32   u32 slots, no remap (P S <= 2^32)
//   kOutWide64  u64 MPHF values (any n)
//   kOutTable4 / kOutTable8  out[i] = table[value]: the fused lookup, with
//               4- or 8-byte table elements; the table is read evict-first
//               (each read touches a line of a table far larger than L2 once,
//               and would otherwise displace the pilot window's lines)
enum : int { kOutMphf32 = 0, kOutPhf32 = 1, kOutWide64 = 2, kOutTable4 = 3, kOutTable8 = 4 };

template <int OUT> struct WindowOut { using T = uint32_t; };
template <> struct WindowOut<kOutWide64> { using T = unsigned long long; };
template <> struct WindowOut<kOutTable8> { using T = unsigned long long; };

// Whether the last pass computes the bucket again (see the traffic note at
// the top of this file).
template <int GAMMA, int OUT>
constexpr bool kRecomputeBucket = GAMMA == MPHF_GAMMA_LINEAR || OUT == kOutTable4 || OUT == kOutTable8;

// 8 resident CTAs (32 registers) for 32-bit values; the 64-bit and table
// forms keep more live values per key and take 6 (40 registers, no spill).
template <int GAMMA, int REDUCE, int REMAP, int OUT>
__global__ void __launch_bounds__(kWinThreads, OUT == kOutMphf32 || OUT == kOutPhf32 ? 8 : 6)
window_last_kernel(const View v, const uint64_t *__restrict__ keys, const uint64_t count,
                   const uint32_t *__restrict__ b32, const uint8_t *__restrict__ qin,
                   typename WindowOut<OUT>::T *__restrict__ out, const uint64_t blo, const uint64_t bhi,
                   const uint64_t part_magic, const typename WindowOut<OUT>::T *__restrict__ table) {
    using T = typename WindowOut<OUT>::T;
    constexpr bool kWideValue = OUT == kOutWide64 || OUT == kOutTable4 || OUT == kOutTable8;
    constexpr int K = kWinLastKeys;
    __shared__ uint64_t hp[256];
    hp[threadIdx.x] = v.C * ((uint64_t)threadIdx.x ^ v.seed);   // kWinThreads == 256
    __syncthreads();
    constexpr bool kRecompute = kRecomputeBucket<GAMMA, OUT>;
    auto value = [&](uint64_t h, uint64_t part, uint32_t pilot) -> uint64_t {
        const uint64_t s = part * v.S + reduce_slot<REDUCE>(v, h ^ hp[pilot]);
        if (OUT == kOutPhf32 || s < v.n) return s;
        const uint64_t j = s - v.n;
        if constexpr (REMAP == kRemapClef) {
            if constexpr (kWideValue) return clef_get64(static_cast<const uint8_t *>(v.remap), j);
            else return clef_get(static_cast<const uint8_t *>(v.remap), (uint32_t)j);
        } else {
            if (kWideValue && v.n > (1ull << 32)) return __ldg(static_cast<const unsigned long long *>(v.remap) + j);
            return __ldg(static_cast<const uint32_t *>(v.remap) + j);
        }
    };
    auto emit = [&](uint64_t val) -> T {
        if constexpr (OUT == kOutTable4 || OUT == kOutTable8) return __ldcs(table + val);
        else return (T)val;
    };
    // The part of bucket b (b < 2^32), from the bucket stream's value.
    auto part_of = [&](uint64_t b) -> uint64_t {
        uint64_t unused;
        return v.B == 1 ? b : mul_hi_lo_32x64((uint32_t)b, part_magic, unused);
    };
    const uint64_t tile = (uint64_t)blockIdx.x * (kWinThreads * K);
    if (tile + kWinThreads * K > count) {
        for (uint64_t i = tile + threadIdx.x; i < count; i += kWinThreads) {
            const uint64_t h = v.C * __ldcs(keys + i);
            uint64_t part, b;
            if constexpr (kRecompute) b = window_bucket<GAMMA>(v, h, part);
            else { b = b32[i]; part = part_of(b); }
            out[i] = emit(value(h, part, in_window(b, blo, bhi) ? __ldg(v.pilots + b) : qin[i]));
        }
        return;
    }
    // kh holds h = C k when the bucket is computed again (it is needed ahead
    // of the pilot reads), else the key, whose product is formed after them
    // (measured: each order is the faster one for its form).
    uint64_t kh[K], part[K], b[K];
    uint32_t p[K], c[K / 2];
    const uint64_t mul = kRecompute ? v.C : 1;
#pragma unroll
    for (int j = 0; j < K / 2; j++) {
        const uint64_t i = tile + (uint64_t)j * 2 * kWinThreads + 2 * threadIdx.x;
        const uint4 kk = __ldcs(reinterpret_cast<const uint4 *>(keys + i));
        kh[2 * j] = mul * (((uint64_t)kk.y << 32) | kk.x);
        kh[2 * j + 1] = mul * (((uint64_t)kk.w << 32) | kk.z);
        if constexpr (!kRecompute) {
            const uint2 bb = __ldcs(reinterpret_cast<const uint2 *>(b32 + i));
            b[2 * j] = bb.x;
            b[2 * j + 1] = bb.y;
        }
        c[j] = __ldcs(reinterpret_cast<const unsigned short *>(qin + i));
    }
    if constexpr (kRecompute) {
#pragma unroll
        for (int q = 0; q < K; q++) b[q] = window_bucket<GAMMA>(v, kh[q], part[q]);
    }
#pragma unroll
    for (int q = 0; q < K; q++)
        p[q] = in_window(b[q], blo, bhi) ? (uint32_t)__ldg(v.pilots + b[q]) : (c[q >> 1] >> (8 * (q & 1))) & 0xFFu;
    if constexpr (!kRecompute) {
#pragma unroll
        for (int q = 0; q < K; q++) part[q] = part_of(b[q]);
    }
    T r[K];
#pragma unroll
    for (int q = 0; q < K; q++) r[q] = emit(value(kRecompute ? kh[q] : v.C * kh[q], part[q], p[q]));
#pragma unroll
    for (int j = 0; j < K / 2; j++) {
        const uint64_t i = tile + (uint64_t)j * 2 * kWinThreads + 2 * threadIdx.x;
        if constexpr (sizeof(T) == 4) __stcs(reinterpret_cast<uint2 *>(out + i), make_uint2(r[2 * j], r[2 * j + 1]));
        else __stcs(reinterpret_cast<ulonglong2 *>(out + i), make_ulonglong2(r[2 * j], r[2 * j + 1]));
    }
}

static_assert(kWinThreads == 256, "the last pass fills its 256-entry hp table with one thread per pilot value");

template <int GAMMA, int REDUCE, int REMAP, int OUT>
static int run_windows(const View &v, const uint64_t *keys, uint64_t count, void *out_v, const void *table_v,
                       uint64_t W, uint64_t chunk, uint64_t part_magic, uint8_t *scratch, cudaStream_t s) {
    using T = typename WindowOut<OUT>::T;
    T *out = static_cast<T *>(out_v);
    const T *table = static_cast<const T *>(table_v);
    const uint64_t nbkt = v.P * v.B;
    uint32_t *b32 = reinterpret_cast<uint32_t *>(scratch);
    const uint64_t cp = window_stream_keys(chunk);   // 16-byte aligned carried-pilot streams
    uint8_t *qa = scratch + 4 * cp, *qb = qa + cp;
    for (uint64_t c0 = 0; c0 < count; c0 += chunk) {
        const uint64_t cnt = count - c0 < chunk ? count - c0 : chunk;
        const unsigned first_blocks = (unsigned)((cnt + kWinThreads * kWinFirstKeys - 1) / (kWinThreads * kWinFirstKeys));
        const unsigned mid_blocks = (unsigned)((cnt + kWinThreads * kWinMidKeys - 1) / (kWinThreads * kWinMidKeys));
        const unsigned last_blocks = (unsigned)((cnt + kWinThreads * kWinLastKeys - 1) / (kWinThreads * kWinLastKeys));
        uint8_t *qi = qa, *qo = qb;
        for (uint64_t w = 0; w < W; w++) {
            const uint64_t blo = nbkt * w / W, bhi = nbkt * (w + 1) / W;
            if (w == 0 && (W > 2 || !kRecomputeBucket<GAMMA, OUT>))
                window_first_kernel<GAMMA, true><<<first_blocks, kWinThreads, 0, s>>>(v, keys + c0, cnt, b32, qo, blo, bhi);
            else if (w == 0)
                window_first_kernel<GAMMA, false><<<first_blocks, kWinThreads, 0, s>>>(v, keys + c0, cnt, b32, qo, blo, bhi);
            else if (w + 1 < W)
                window_mid_kernel<<<mid_blocks, kWinThreads, 0, s>>>(v.pilots, b32, cnt, qi, qo, blo, bhi);
            else
                window_last_kernel<GAMMA, REDUCE, REMAP, OUT><<<last_blocks, kWinThreads, 0, s>>>(
                    v, keys + c0, cnt, b32, qi, out + c0, blo, bhi, part_magic, table);
            count_launch();
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "windowed query launch");
            uint8_t *t = qi;
            qi = qo;
            qo = t;
        }
    }
    return MPHF_OK;
}

// The automatic window count (measured on GB300, all keys of a structure
// queried in a random order, per query of n keys):
//   pilots   86 MB (n = 3e8):   single 1.97 ms, W = 2 1.86
//           143 MB (n = 5e8):   single 4.07, W = 2 3.50, W = 3 3.74
//           200 MB (n = 7e8):   single 6.84, W = 2 5.87, W = 3 5.69, W = 4 6.10
//           286 MB (n = 1e9):   single 12.54, W = 3 9.17, W = 4 9.38, W = 5 9.89
//           400 MB (n = 1.4e9): single 18.79, W = 3 15.51, W = 4 14.71, W = 5 15.24
//           572 MB (n = 2e9):   single 30.08, W = 4 24.94, W = 5 24.43, W = 6 25.17, W = 8 27.55
//          1.29 GB (n = 4.5e9): single 82.8, W = 18 (72 MB windows) 112
// The best windows hold 70-115 MB, growing with the pilot array (larger
// arrays pay more middle passes per window saved).  W = ceil(pilots / 100
// MB), at least 2, is within 3 % of the best at every size above; the
// rounding rule round(pilots / 110 MB) was 7-16 % slower on the Compact
// (250 MB, 2 windows of 125 MB: 9.72 ms against 9.05 in 4 windows) and Fast
// (334 MB of uniformly used buckets, 3 windows of 111 MB: 11.83 against
// 10.07-10.22) structures at n = 1e9.  Past 6 windows the middle passes' 6
// bytes per key outweigh the random reads they replace, and at or below
// 72 MiB the single pass keeps most pilots in L2.
constexpr uint64_t kWindowAutoMin = 72ull << 20;
constexpr uint64_t kWindowAutoBytes = 100000000ull;
constexpr uint64_t kWindowMaxAuto = 6;

uint64_t window_count_for(uint64_t nbkt, uint64_t window_bytes) {
    if (window_bytes) return (nbkt + window_bytes - 1) / window_bytes;
    if (nbkt <= kWindowAutoMin) return 1;
    uint64_t W = (nbkt + kWindowAutoBytes - 1) / kWindowAutoBytes;
    if (W < 2) W = 2;
    return W > kWindowMaxAuto ? 1 : W;
}

uint64_t window_plan(const Header &h, uint64_t count) {
    return count >= kWindowMinKeys ? window_count_for(h.P * h.B, 0) : 1;
}

uint64_t window_stream_keys(uint64_t chunk) { return (chunk + 15) & ~15ull; }

uint64_t window_chunk_for(uint64_t count, uint64_t chunk_keys) {
    uint64_t chunk = chunk_keys ? chunk_keys : kWindowChunkDefault;
    const uint64_t even = count + (count & 1);
    return chunk < even ? chunk : even;
}

bool window_supported(const Header &h, const uint64_t *keys, const void *out, int out_bytes) {
    const uint64_t nbkt = h.P * h.B;
    return h.B > 0 && h.P < (1ull << 32) && h.B < (1ull << 32) && nbkt < (1ull << 32) && ((uintptr_t)keys % 16) == 0 &&
           ((uintptr_t)out % (2 * out_bytes)) == 0;
}

template <int GAMMA, int REDUCE, int OUT>
static int run_windows_remap(const Header &h, const View &v, const uint64_t *keys, uint64_t count, void *out,
                             const void *table, uint64_t W, uint64_t chunk, uint64_t part_magic, uint8_t *scratch,
                             cudaStream_t s) {
    if (OUT == kOutPhf32)
        return run_windows<GAMMA, REDUCE, kRemapNone, OUT>(v, keys, count, out, table, W, chunk, part_magic, scratch, s);
    if (h.remap == MPHF_REMAP_VEC)
        return run_windows<GAMMA, REDUCE, kRemapVec, OUT>(v, keys, count, out, table, W, chunk, part_magic, scratch, s);
    return run_windows<GAMMA, REDUCE, kRemapClef, OUT>(v, keys, count, out, table, W, chunk, part_magic, scratch, s);
}

template <int OUT>
static int run_windows_layout(const Header &h, const View &v, const uint64_t *keys, uint64_t count, void *out,
                              const void *table, uint64_t W, uint64_t chunk, uint64_t part_magic, uint8_t *scratch,
                              cudaStream_t s) {
    const bool cubic = h.gamma == MPHF_GAMMA_CUBIC, pow2 = h.reduce == kReducePow2;
    if (cubic && pow2)
        return run_windows_remap<MPHF_GAMMA_CUBIC, kReducePow2, OUT>(h, v, keys, count, out, table, W, chunk, part_magic, scratch, s);
    if (cubic)
        return run_windows_remap<MPHF_GAMMA_CUBIC, kReduceMod, OUT>(h, v, keys, count, out, table, W, chunk, part_magic, scratch, s);
    if (pow2)
        return run_windows_remap<MPHF_GAMMA_LINEAR, kReducePow2, OUT>(h, v, keys, count, out, table, W, chunk, part_magic, scratch, s);
    return run_windows_remap<MPHF_GAMMA_LINEAR, kReduceMod, OUT>(h, v, keys, count, out, table, W, chunk, part_magic, scratch, s);
}

int window_out_bytes(int mode) { return mode == kWinWide64 || mode == kWinTable8 ? 8 : 4; }

// scratch: 6 window_stream_keys(chunk) bytes of device memory (the bucket
// stream and two carried-pilot streams of one chunk), 16-byte aligned.
int launch_query_u64_windowed(const Header &h, const View &v, const uint64_t *keys, uint64_t count, void *out,
                              int mode, const void *table, uint64_t W, uint64_t chunk, uint8_t *scratch,
                              cudaStream_t s) {
    if (W < 2 || chunk < 2 || chunk % 2 || chunk > (1ull << 31) ||
        !window_supported(h, keys, out, window_out_bytes(mode))) {
        set_error("windowed query: W >= 2, an even chunk of at most 2^31 keys, P B < 2^32, aligned buffers");
        return MPHF_ERR_ARG;
    }
    // M = ceil(2^64 / B) gives the part of a bucket index (B >= 2).
    const uint64_t part_magic = h.B == 1 ? 0 : (uint64_t)((((unsigned __int128)1 << 64) + h.B - 1) / h.B);
    switch (mode) {
        case kWinMphf32: return run_windows_layout<kOutMphf32>(h, v, keys, count, out, table, W, chunk, part_magic, scratch, s);
        case kWinPhf32: return run_windows_layout<kOutPhf32>(h, v, keys, count, out, table, W, chunk, part_magic, scratch, s);
        case kWinWide64: return run_windows_layout<kOutWide64>(h, v, keys, count, out, table, W, chunk, part_magic, scratch, s);
        case kWinTable4: return run_windows_layout<kOutTable4>(h, v, keys, count, out, table, W, chunk, part_magic, scratch, s);
        case kWinTable8: return run_windows_layout<kOutTable8>(h, v, keys, count, out, table, W, chunk, part_magic, scratch, s);
        default: set_error("windowed query: unknown output form"); return MPHF_ERR_ARG;
    }
}

}  // namespace ptrhash
