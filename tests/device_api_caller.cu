// A caller's own kernels that evaluate PtrHash structures through the public
// device header (include/mphf_device.cuh), built apart from libmphf the way
// an application would build them.  Used by the device-API tests.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mphf_device.cuh"

namespace {

constexpr int kThreads = 256;

unsigned grid_for(uint64_t n) {
    const uint64_t blocks = (n + kThreads - 1) / kThreads;
    return (unsigned)(blocks < 152 * 16 ? blocks : 152 * 16);
}

__global__ void eval_u64_kernel(mphf_view_t v, const uint64_t *keys, uint64_t n, uint32_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = mphf_dev::eval_u64(v, keys[i]);
}

__global__ void eval_bytes_kernel(mphf_view_t v, const uint8_t *bytes, const uint64_t *off, uint64_t n,
                                  uint32_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = mphf_dev::eval_bytes(v, bytes + off[i], off[i + 1] - off[i]);
}

// The lookup fused into a consumer: each key's value indexes a counter,
// and nothing but the counters is written.
__global__ void count_u64_kernel(mphf_view_t v, const uint64_t *keys, uint64_t n, uint32_t *counts) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + mphf_dev::eval_u64(v, keys[i]), 1u);
}

__global__ void eval_u64_wide_kernel(mphf_view_t v, const uint64_t *keys, uint64_t n, uint64_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = mphf_dev::eval_u64_wide(v, keys[i]);
}

// K keys per thread through eval_u64_n, with a ragged last group.
template <int K>
__global__ void eval_u64_n_kernel(mphf_view_t v, const uint64_t *keys, uint64_t n, uint32_t *out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * K;
    for (uint64_t base = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * K; base < n; base += stride) {
        uint64_t k[K];
        uint32_t val[K];
#pragma unroll
        for (int q = 0; q < K; q++) k[q] = base + q < n ? keys[base + q] : keys[0];
        mphf_dev::eval_u64_n<K>(v, k, val);
#pragma unroll
        for (int q = 0; q < K; q++)
            if (base + q < n) out[base + q] = val[q];
    }
}

__global__ void slot_u64_kernel(mphf_view_t v, const uint64_t *keys, uint64_t n, uint64_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = mphf_dev::slot_hash(v, v.C * keys[i]);
}

}  // namespace

extern "C" {

int caller_eval_u64(const mphf_view_t *v, const uint64_t *keys, uint64_t n, uint32_t *out, void *stream) {
    if (n) eval_u64_kernel<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(*v, keys, n, out);
    return (int)cudaGetLastError();
}

int caller_eval_bytes(const mphf_view_t *v, const uint8_t *bytes, const uint64_t *off, uint64_t n, uint32_t *out,
                      void *stream) {
    if (n) eval_bytes_kernel<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(*v, bytes, off, n, out);
    return (int)cudaGetLastError();
}

int caller_count_u64(const mphf_view_t *v, const uint64_t *keys, uint64_t n, uint32_t *counts, void *stream) {
    if (n) count_u64_kernel<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(*v, keys, n, counts);
    return (int)cudaGetLastError();
}

int caller_eval_u64_wide(const mphf_view_t *v, const uint64_t *keys, uint64_t n, uint64_t *out, void *stream) {
    if (n) eval_u64_wide_kernel<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(*v, keys, n, out);
    return (int)cudaGetLastError();
}

int caller_eval_u64_n4(const mphf_view_t *v, const uint64_t *keys, uint64_t n, uint32_t *out, void *stream) {
    if (n) eval_u64_n_kernel<4><<<grid_for((n + 3) / 4), kThreads, 0, (cudaStream_t)stream>>>(*v, keys, n, out);
    return (int)cudaGetLastError();
}

int caller_slot_u64(const mphf_view_t *v, const uint64_t *keys, uint64_t n, uint64_t *out, void *stream) {
    if (n) slot_u64_kernel<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(*v, keys, n, out);
    return (int)cudaGetLastError();
}

}  // extern "C"
