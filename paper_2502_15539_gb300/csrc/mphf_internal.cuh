// Internal declarations shared by the library's translation units.
//
// Device-side view of a PtrHash structure and the exact 64-bit integer
// arithmetic of the query (Sec. 3.1 Eq. partbucket and Eq. slot, Sec. 3.3
// gamma, Sec. 3.4 Eq. clef).  Everything here is integer and exact.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/mphf.h"
#include "../../include/mphf_device.cuh"

namespace ptrhash {

enum : int { kReducePow2 = 0, kReduceMod = 1 };
enum : int { kRemapClef = MPHF_REMAP_CLEF, kRemapVec = MPHF_REMAP_VEC, kRemapNone = 2 };
constexpr int kClefPerLine = 44;   // values per 64-byte CacheLineEF line (Sec. 3.4)

// Everything a query kernel needs, passed by value as a kernel argument.
struct View {
    const uint8_t *pilots;   // P*B bytes
    const void *remap;       // CacheLineEF lines (64 B each) or u32 entries
    uint64_t n, P, S, B, C, seed;
    uint64_t fm, fm_unused;  // floor(2^64 / S) for reduce = x mod S
    uint64_t s_mask;         // S - 1 for power-of-two S
};

// ---------------------------------------------------------------- host side
struct Header {
    uint64_t n = 0, P = 0, S = 0, B = 0, C = 0, seed = 0;
    int32_t gamma = MPHF_GAMMA_CUBIC, remap = MPHF_REMAP_CLEF, reduce = kReducePow2;
    int32_t key_kind = MPHF_KEY_U64;
    int32_t hash128 = 0;       // byte keys hashed to 128 bits (high: part and bucket, low: slot)
    double lambda = 3.5, alpha = 0.99;
    uint64_t remap_len = 0;    // P*S - n
    uint64_t remap_bytes = 0;  // bytes of the remap payload
};

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
void count_launch(uint64_t k = 1);

// Layout rule of Sec. 3.1 "Parameter values" (library's own implementation).
int choose_layout(uint64_t n, double lambda, double alpha, uint64_t slots_override,
                  uint64_t *P, uint64_t *S, uint64_t *B, int *reduce);
uint64_t barrett_constant(uint64_t S);
uint64_t clef_lines_for(uint64_t remap_len);

// Keys a structure may hold: CacheLineEF stores values below 2^40 (a 32-bit
// offset in units of 256).  Values pass 32 bits once n > 2^32; the plain
// remap array then holds u64 entries, and the results need 64-bit outputs.
constexpr uint64_t kMaxKeys = 1ull << 40;
inline bool wide_values(uint64_t n) { return n > (1ull << 32); }
inline uint64_t vec_entry_bytes(uint64_t n) { return wide_values(n) ? 8 : 4; }

View make_view(const Header &h, const uint8_t *pilots, const void *remap);

// Query launchers (mphf_query.cu).
int launch_query_u64(const Header &h, const View &v, const uint64_t *keys, uint64_t count,
                     uint32_t *out, bool phf, cudaStream_t s);
int launch_query_bytes(const Header &h, const View &v, const uint8_t *bytes,
                       const uint64_t *offsets, uint64_t count, uint32_t *out, cudaStream_t s);
int launch_query_u64_wide(const Header &h, const View &v, const uint64_t *keys, uint64_t count, uint64_t *out,
                          cudaStream_t s);
int launch_query_bytes_wide(const Header &h, const View &v, const uint8_t *bytes, const uint64_t *offsets,
                            uint64_t count, uint64_t *out, cudaStream_t s);

// Windowed query (mphf_window.cu): the pilot array in W byte ranges that stay
// L2-resident, the keys streamed once per range.  window_count_for gives W
// for a window size (0: the automatic count for the pilot array, 1 meaning
// the single pass); window_plan the W the automatic path uses for a batch.
// The output forms: u32 MPHF values, u32 slots (PHF), u64 values, and the
// fused lookup out[i] = table[value] with 4- or 8-byte elements.
enum : int { kWinMphf32 = 0, kWinPhf32 = 1, kWinWide64 = 2, kWinTable4 = 3, kWinTable8 = 4 };
uint64_t window_count_for(uint64_t nbkt, uint64_t window_bytes);
uint64_t window_plan(const Header &h, uint64_t count);
uint64_t window_chunk_for(uint64_t count, uint64_t chunk_keys);
// Keys per scratch stream for a chunk: the chunk rounded up to 16, so that
// every stream of the scratch starts 16-byte aligned.
uint64_t window_stream_keys(uint64_t chunk);
int window_out_bytes(int mode);
// Keys 16-byte aligned, out aligned to two elements, P B < 2^32.
bool window_supported(const Header &h, const uint64_t *keys, const void *out, int out_bytes);
int launch_query_u64_windowed(const Header &h, const View &v, const uint64_t *keys, uint64_t count, void *out,
                              int mode, const void *table, uint64_t W, uint64_t chunk, uint8_t *scratch,
                              cudaStream_t s);
// The windowed query on a structure's own scratch (mphf_api.cu): W >= 2
// windows, chunk_keys 0 for the default.  MPHF_ERR_OOM (no CUDA error left
// pending) if the scratch cannot be allocated.
int handle_windowed_query(const mphf *m, const uint64_t *keys, uint64_t count, void *out, int mode,
                          const void *table, uint64_t W, uint64_t chunk_keys, cudaStream_t s);
// The automatic choice of the query entry points: runs the windowed path and
// returns 1 (its result in *rc) for a batch of at least 2^24 keys against a
// pilot array of 2 to 6 automatic windows with aligned buffers; else returns 0 and the
// caller runs the single pass (also when the scratch cannot be allocated).
int try_windowed(const mphf *m, const uint64_t *keys, uint64_t count, void *out, int mode, const void *table,
                 cudaStream_t s, int *rc);

// Global bucket index of each u64 key (mphf_query.cu).
int launch_bucket_u64(const Header &h, const View &v, const uint64_t *keys, uint64_t count, uint64_t *out,
                      int sm_count, cudaStream_t s);

// Key hashes for the builder (mphf_query.cu); out_hi (high halves of the
// 128-bit string hash) may be NULL.
int launch_hash_keys(int key_kind, const void *keys, const uint64_t *offsets, uint64_t n, uint64_t C,
                     uint64_t seed, uint64_t *out, uint64_t *out_hi, int sm_count, cudaStream_t s);

// Builder (mphf_build.cu).  Fills header, pilots and remap on the device.
struct BuildResult {
    Header hdr;
    uint8_t *d_pilots = nullptr;
    uint8_t *d_remap = nullptr;
    uint64_t evictions = 0;
    double build_ms = 0.0;
    double hash_sort_ms = 0.0, search_ms = 0.0, remap_ms = 0.0;   // phases, summed over shards and seeds
};
int build_structure(const mphf_params &p, int key_kind, const void *keys, const uint64_t *offsets,
                    uint64_t n, cudaStream_t s, BuildResult *out);

// ------------------------------------------------------------- device side
// The exact arithmetic of the query lives in the public device header;
// the kernels here use it with compile-time layouts.
using namespace mphf_dev;

template <int REDUCE>
__device__ __forceinline__ uint64_t reduce_slot(const View &v, uint64_t x) {
    if constexpr (REDUCE == kReducePow2) {
        return mul_hi(v.C, x) & v.s_mask;      // hi(C x) mod S, S = 2^k
    } else {
        return mod_barrett(x, v.fm, v.S);
    }
}

constexpr int kStrStage = 2048 + 32;   // staged bytes per warp (32 strings)

// Hashes the strings [w0, min(w0 + 32, count)) of a warp: lane l returns the
// hash of string w0 + l (any value for lanes past count).  Their contiguous
// byte range is staged into `stage` (kStrStage bytes, 16-byte aligned,
// private to the warp) with 16-byte loads; every byte below the end of the
// whole key buffer may be read, only a chunk crossing it is read byte by
// byte.  A warp whose range does not fit the stage reads from global memory.
// All lanes of the warp must call it.
__device__ __forceinline__ uint64_t warp_hash_strings(const uint8_t *bytes, const uint64_t *offsets, uint64_t w0,
                                                      uint64_t count, uint8_t *stage, uint64_t seed, int lane) {
    const uint64_t i = w0 + lane;
    const uint64_t last = (w0 + 32 < count ? w0 + 32 : count);
    const uint64_t lo = __ldg(offsets + w0), hi = __ldg(offsets + last);
    const uint64_t a = i < count ? __ldg(offsets + i) : hi;
    const uint64_t e = i < count ? __ldg(offsets + i + 1) : hi;
    const uint64_t base = lo & ~15ull;
    if (hi - base + 32 > kStrStage) return hash_string_global(bytes, a, e - a, seed);   // + one zeroed chunk
    const uint64_t end_all = last < count ? __ldg(offsets + count) : hi;
    const uint32_t nvec = (uint32_t)((hi - base + 15) / 16);
    uint4 *dst = reinterpret_cast<uint4 *>(stage);
    __syncwarp();   // the stage may still be read from a previous call
    for (uint32_t q = lane; q < nvec; q += 32) {
        const uint64_t c0 = base + 16ull * q;
        if (c0 + 16 <= end_all) {
            dst[q] = __ldcs(reinterpret_cast<const uint4 *>(bytes + c0));
        } else {
            uint8_t *d8 = stage + 16 * q;
            for (int t = 0; t < 16; t++) d8[t] = c0 + t < hi ? __ldg(bytes + c0 + t) : 0;
        }
    }
    if (lane == 0) dst[nvec] = make_uint4(0, 0, 0, 0);   // word a+1 may be read
    __syncwarp();
    // The stage holds every byte of the string plus at least 16 readable
    // bytes after it, so the words past its end may be read unguarded.
    const uint32_t start = (uint32_t)(a - base);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(stage) + (start >> 2);
    return hash_string_words([&](uint32_t k) { return w[k]; }, 8 * (start & 3u), (uint32_t)(e - a), seed);
}

}  // namespace ptrhash
