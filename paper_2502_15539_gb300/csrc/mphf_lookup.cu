// Fused lookup: out[i] = table[value(keys[i])] in one kernel.
//
// The MPHF's use is as the index of a static key set whose per-key data sits
// in an array addressed by the hash value (Sec. 1, Motivation: the k-mer
// index of SSHash).  Fusing the lookup into the kernel that consumes the
// value is the streaming-inside-an-application direction of Sec. 5: the
// value never leaves registers, so the separate query pass's 4-byte write and
// the gather pass's 4-byte re-read per key disappear, and so does a launch.
//
// The single-pass kernel is written against the public device API
// (mphf_device.cuh), exactly as an application kernel would use it:
// eval_u64_n puts K pilot gathers in flight per thread, then the K table
// reads go out together.  Large batches against a pilot array above L2 take
// the windowed query instead (mphf_window.cu), whose last pass does the
// table read.
// Table reads are evict-first (ld.global.cs): each touches a line of a table
// far larger than L2 once, and with the default policy those lines displace
// pilot lines (at 1e9 keys and a 4 GB table, 36.6 ms instead of 33.8 ms).
#include "mphf_internal.cuh"

namespace ptrhash {
namespace {

constexpr int kLookupThreads = 256;
constexpr int kLookupKeys = 8;

template <typename T, bool WIDE>
__global__ void __launch_bounds__(kLookupThreads, 3)
lookup_u64_kernel(const mphf_view_t v, const uint64_t *__restrict__ keys, const uint64_t count,
                  const T *__restrict__ table, T *__restrict__ out) {
    constexpr int K = kLookupKeys;
    const uint64_t tile = (uint64_t)blockIdx.x * (kLookupThreads * K);
    uint64_t k[K];
#pragma unroll
    for (int q = 0; q < K; q++) {
        const uint64_t i = tile + (uint64_t)q * kLookupThreads + threadIdx.x;
        k[q] = i < count ? __ldcs(keys + i) : 0ull;   // past the end: any key, its value is < n
    }
    T val[K];
    if constexpr (WIDE) {
        uint64_t idx[K];
        mphf_dev::eval_u64_wide_n<K>(v, k, idx);
#pragma unroll
        for (int q = 0; q < K; q++) {
            const uint64_t i = tile + (uint64_t)q * kLookupThreads + threadIdx.x;
            val[q] = i < count ? __ldcs(table + idx[q]) : T(0);
        }
    } else {
        uint32_t idx[K];
        mphf_dev::eval_u64_n<K>(v, k, idx);
#pragma unroll
        for (int q = 0; q < K; q++) {
            const uint64_t i = tile + (uint64_t)q * kLookupThreads + threadIdx.x;
            val[q] = i < count ? __ldcs(table + idx[q]) : T(0);
        }
    }
#pragma unroll
    for (int q = 0; q < K; q++) {
        const uint64_t i = tile + (uint64_t)q * kLookupThreads + threadIdx.x;
        if (i < count) __stcs(out + i, val[q]);
    }
}

template <typename T>
int launch_lookup(const mphf_view_t &v, const uint64_t *keys, uint64_t count, const void *table, void *out,
                  cudaStream_t s) {
    const uint64_t per_block = (uint64_t)kLookupThreads * kLookupKeys;
    const uint64_t blocks = (count + per_block - 1) / per_block;
    if (blocks > 0x7FFFFFFFull) { set_error("too many keys for one launch"); return MPHF_ERR_ARG; }
    if (v.n > (1ull << 32))
        lookup_u64_kernel<T, true><<<(unsigned)blocks, kLookupThreads, 0, s>>>(
            v, keys, count, static_cast<const T *>(table), static_cast<T *>(out));
    else
        lookup_u64_kernel<T, false><<<(unsigned)blocks, kLookupThreads, 0, s>>>(
            v, keys, count, static_cast<const T *>(table), static_cast<T *>(out));
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPHF_OK : cuda_fail(e, "lookup launch");
}

}  // namespace
}  // namespace ptrhash

using namespace ptrhash;

extern "C" int mphf_lookup_u64(const mphf_t *m, const uint64_t *keys_dev, uint64_t count, const void *table_dev,
                               uint32_t elem_bytes, void *out_dev, void *stream) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    if (elem_bytes != 4 && elem_bytes != 8) { set_error("table elements must be 4 or 8 bytes"); return MPHF_ERR_ARG; }
    if (count == 0) return MPHF_OK;
    if (!keys_dev || !table_dev || !out_dev || ((uintptr_t)keys_dev & 7) ||
        ((uintptr_t)table_dev % elem_bytes) || ((uintptr_t)out_dev % elem_bytes)) {
        set_error("keys must be 8-byte aligned, table and out aligned to their element size");
        return MPHF_ERR_ARG;
    }
    mphf_view_t v;
    int rc = mphf_device_view(m, &v);
    if (rc) return rc;
    if (v.key_kind != MPHF_KEY_U64) { set_error("structure was built for byte keys"); return MPHF_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    // Large batches against a pilot array above L2 take the windowed query,
    // whose last pass reads the table entry in place of writing the value.
    if (try_windowed(m, keys_dev, count, out_dev, elem_bytes == 4 ? kWinTable4 : kWinTable8, table_dev, s, &rc))
        return rc;
    return elem_bytes == 4 ? launch_lookup<unsigned int>(v, keys_dev, count, table_dev, out_dev, s)
                           : launch_lookup<unsigned long long>(v, keys_dev, count, table_dev, out_dev, s);
}
