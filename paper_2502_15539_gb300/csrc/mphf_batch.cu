// Multi-MPHF batched queries: one persistent launch over many structures.
//
// A batch is a list of requests (structure, keys, count, out).  The host
// turns it into one descriptor per request (the structure's view plus the
// request's first tile) and the kernel's warps pull tiles of 32 K keys (K
// keys per lane) from a global counter until every tile is done, so
// structures of very different sizes and batches of 1 to 1e6 keys share one
// launch.  The upload of the descriptors, the counter reset and the kernel
// are captured once into a CUDA graph and replayed for every batch.  Launch
// shape (keys per lane, threads, CTAs per SM) comes from an autotuner that
// times the candidates on a real batch and keeps the winner in a small JSON
// cache.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "mphf_internal.cuh"

struct mphf;   // opaque handle of mphf_api.cu
namespace ptrhash {
const Header &handle_header(const mphf *m);
View handle_view(const mphf *m);
}  // namespace ptrhash

namespace ptrhash {

// One request as the kernel sees it.
struct BatchDesc {
    View v;                    // 96 bytes
    const void *keys;          // u64 keys, or packed bytes
    const uint64_t *offsets;   // byte keys: count + 1 offsets, else NULL
    uint32_t *out;
    uint32_t count;
    uint8_t gamma, reduce, remap, key_kind;
};

struct BatchHeader {
    uint32_t nreq;
    uint32_t total_tiles;
    uint32_t counter;          // next tile (reset to 0 before each launch)
    uint32_t pad;
};

// Eq. partbucket with P, B < 2^32 (true of every structure): 32 x 64-bit products.
__device__ __forceinline__ uint64_t bucket_any(const View &v, uint64_t h, uint64_t &part, bool cubic) {
    uint64_t x, unused;
    part = mul_hi_lo_32x64((uint32_t)v.P, h, x);
    return part * v.B + mul_hi_lo_32x64((uint32_t)v.B, cubic ? bucket_fn<MPHF_GAMMA_CUBIC>(x) : x, unused);
}

__device__ __forceinline__ uint32_t slot_any(const View &v, uint64_t h, uint64_t part, uint32_t pilot, bool pow2,
                                             int remap) {
    const uint64_t x = h ^ (v.C * ((uint64_t)pilot ^ v.seed));
    const uint64_t r = pow2 ? (mul_hi(v.C, x) & v.s_mask) : mod_barrett(x, v.fm, v.S);
    const uint64_t s = part * v.S + r;
    if (s < v.n) return (uint32_t)s;
    const uint32_t j = (uint32_t)(s - v.n);
    if (remap == kRemapClef) return clef_get(static_cast<const uint8_t *>(v.remap), j);
    return __ldg(static_cast<const uint32_t *>(v.remap) + j);
}

constexpr int kMaxReqSmem = 4096;   // request tile starts cached in shared memory

// Persistent CTAs whose warps take tiles on their own: tile t of request r
// covers keys [(t - first_tile[r]) * 32 K, ...), lane l handling keys
// l, l + 32, ... of it.  A warp asks for its next tile while it works on the
// current one, so the atomic's latency is hidden, and no barrier ties the
// warps of a block together after the request table is loaded.
// Up to 4 keys per lane the registers allow 1536 resident threads per SM
// (more warps to hide the latency of each tile); 8 and 16 keys need more.
template <int K>
__global__ void __launch_bounds__(512, K <= 4 ? 3 : (K == 8 ? 2 : 1))
batch_query_kernel(const BatchDesc *__restrict__ desc, const uint32_t *__restrict__ first_tile,
                   BatchHeader *__restrict__ hdr) {
    __shared__ uint32_t s_first[kMaxReqSmem + 1];
    extern __shared__ __align__(16) uint8_t s_stage[];   // kStrStage bytes per warp
    const uint32_t nreq = hdr->nreq, total = hdr->total_tiles;
    for (uint32_t i = threadIdx.x; i <= nreq && i <= kMaxReqSmem; i += blockDim.x) s_first[i] = first_tile[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *stage = s_stage + (size_t)warp * kStrStage;
    constexpr uint32_t TK = 32 * K;
    uint32_t t = lane == 0 ? atomicAdd(&hdr->counter, 1u) : 0u;
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    uint32_t lo = 0;   // the request of the warp's previous tile
    while (t < total) {
        const uint32_t tn = lane == 0 ? atomicAdd(&hdr->counter, 1u) : 0u;   // the next tile, in flight
        // The request owning tile t: the last r with first_tile[r] <= t.  A
        // warp's consecutive tiles mostly fall in one large request, so the
        // previous request is checked before searching.
        if (!(s_first[lo] <= t && t < s_first[lo + 1])) {
            uint32_t a = 0, b = nreq;   // invariant: first[a] <= t < first[b]
            while (b - a > 1) {
                const uint32_t mid = (a + b) >> 1;
                if (s_first[mid] <= t) a = mid; else b = mid;
            }
            lo = a;
        }
        const BatchDesc &d = desc[lo];
        const View v = d.v;
        const bool cubic = d.gamma == MPHF_GAMMA_CUBIC, pow2 = d.reduce == kReducePow2;
        const int remap = d.remap;
        const uint32_t count = d.count;
        const uint64_t base = (uint64_t)(t - s_first[lo]) * TK;
        if (d.key_kind == MPHF_KEY_U64) {
            const uint64_t *keys = static_cast<const uint64_t *>(d.keys);
            uint64_t h[K], part[K], b[K];
            uint32_t p[K];
            // A full tile whose keys are 16-byte and outputs 8-byte aligned:
            // lane l takes the key pairs base + 64 j + 2 l (+1), loaded as one
            // uint4 and stored as one uint2, with no per-key bounds checks.
            const bool paired = base + TK <= count &&
                                ((reinterpret_cast<uintptr_t>(keys + base) | (reinterpret_cast<uintptr_t>(d.out + base) & 7)) & 15) == 0;
            if (paired) {
#pragma unroll
                for (int j = 0; j < K / 2; j++) {
                    const uint4 kk = __ldcs(reinterpret_cast<const uint4 *>(keys + base + 64u * j + 2 * lane));
                    h[2 * j] = v.C * (((uint64_t)kk.y << 32) | kk.x);
                    h[2 * j + 1] = v.C * (((uint64_t)kk.w << 32) | kk.z);
                }
#pragma unroll
                for (int q = 0; q < K; q++) b[q] = bucket_any(v, h[q], part[q], cubic);
#pragma unroll
                for (int q = 0; q < K; q++) p[q] = __ldg(v.pilots + b[q]);
#pragma unroll
                for (int j = 0; j < K / 2; j++)
                    __stcs(reinterpret_cast<uint2 *>(d.out + base + 64u * j + 2 * lane),
                           make_uint2(slot_any(v, h[2 * j], part[2 * j], p[2 * j], pow2, remap),
                                      slot_any(v, h[2 * j + 1], part[2 * j + 1], p[2 * j + 1], pow2, remap)));
            } else {   // a ragged or unaligned tile: lane l takes keys base + 32 q + l
#pragma unroll
                for (int q = 0; q < K; q++) {
                    const uint64_t i = base + 32u * q + lane;
                    h[q] = v.C * (i < count ? __ldcs(keys + i) : 0ull);
                    b[q] = bucket_any(v, h[q], part[q], cubic);
                }
#pragma unroll
                for (int q = 0; q < K; q++) {
                    const uint64_t i = base + 32u * q + lane;
                    p[q] = i < count ? __ldg(v.pilots + b[q]) : 0u;
                }
#pragma unroll
                for (int q = 0; q < K; q++) {
                    const uint64_t i = base + 32u * q + lane;
                    if (i < count) __stcs(d.out + i, slot_any(v, h[q], part[q], p[q], pow2, remap));
                }
            }
        } else {
            // Strings: groups of 32 consecutive strings through the warp's stage.
            const uint8_t *bytes = static_cast<const uint8_t *>(d.keys);
            for (int g = 0; g < K; g++) {
                const uint64_t w0 = base + 32ull * g;
                if (w0 >= count) break;
                const uint64_t hh = warp_hash_strings(bytes, d.offsets, w0, count, stage, v.seed, lane);
                const uint64_t i = w0 + lane;
                if (i < count) {
                    uint64_t pt;
                    const uint64_t bb = bucket_any(v, hh, pt, cubic);
                    d.out[i] = slot_any(v, hh, pt, __ldg(v.pilots + bb), pow2, remap);
                }
            }
        }
        t = __shfl_sync(0xFFFFFFFFu, tn, 0);
    }
}

// ----------------------------------------------------------------- host
struct BatchConfig {
    int keys_per_thread = 8, threads = 512, blocks_per_sm = 2;
};

static bool valid_config(const BatchConfig &c) {
    return (c.keys_per_thread == 2 || c.keys_per_thread == 4 || c.keys_per_thread == 8 || c.keys_per_thread == 16) &&
           (c.threads == 128 || c.threads == 256 || c.threads == 512) && c.blocks_per_sm >= 1 && c.blocks_per_sm <= 16;
}

template <int K>
static void launch_k(unsigned grid, int threads, size_t smem, const BatchDesc *desc, const uint32_t *first,
                     BatchHeader *hdr, cudaStream_t s) {
    // Static + dynamic shared memory can exceed 48 KB: opt in once per device.
    static std::atomic<uint64_t> opted{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (!(opted.load(std::memory_order_relaxed) & bit)) {
        cudaFuncSetAttribute(batch_query_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16 * kStrStage);
        opted.fetch_or(bit, std::memory_order_relaxed);
    }
    batch_query_kernel<K><<<grid, threads, smem, s>>>(desc, first, hdr);
}

static cudaError_t launch_batch_kernel(const BatchConfig &c, int sms, const BatchDesc *desc, const uint32_t *first,
                                       BatchHeader *hdr, cudaStream_t s) {
    const unsigned grid = (unsigned)(sms * c.blocks_per_sm);
    const size_t smem = (size_t)(c.threads / 32) * kStrStage;
    switch (c.keys_per_thread) {
        case 2: launch_k<2>(grid, c.threads, smem, desc, first, hdr, s); break;
        case 4: launch_k<4>(grid, c.threads, smem, desc, first, hdr, s); break;
        case 16: launch_k<16>(grid, c.threads, smem, desc, first, hdr, s); break;
        default: launch_k<8>(grid, c.threads, smem, desc, first, hdr, s); break;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace ptrhash

using namespace ptrhash;

constexpr int kStages = 2;   // staging sets: batch i+1 is staged while batch i runs

struct mphf_batch {
    uint32_t cap = 0;
    int sms = 0, device = 0;
    BatchConfig cfg;
    // Per staging set: page-locked host buffer, device buffer (header, first
    // tiles, descriptors), the captured graph and the event of its last run.
    uint8_t *h_buf[kStages] = {}, *d_buf[kStages] = {};
    cudaGraph_t graph[kStages] = {};
    cudaGraphExec_t exec[kStages] = {};
    cudaEvent_t done[kStages] = {};
    size_t buf_bytes = 0;
    cudaStream_t cap_stream = nullptr;
    bool use_graph = true;
    uint64_t runs = 0;
    std::mutex mu;
};

static size_t off_first(uint32_t) { return sizeof(BatchHeader); }
static size_t off_desc(uint32_t cap) { return (sizeof(BatchHeader) + (cap + 1) * 4 + 255) & ~(size_t)255; }

static void free_graphs(mphf_batch *b) {
    for (int i = 0; i < kStages; i++) {
        if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
        if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
        b->exec[i] = nullptr;
        b->graph[i] = nullptr;
    }
}

// Captures staging set i: copy of its staging buffer, then the kernel.
static int capture_graph(mphf_batch *b, int i) {
    cudaStream_t s = b->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "batch: begin capture");
    cudaMemcpyAsync(b->d_buf[i], b->h_buf[i], b->buf_bytes, cudaMemcpyHostToDevice, s);
    launch_batch_kernel(b->cfg, b->sms, reinterpret_cast<const BatchDesc *>(b->d_buf[i] + off_desc(b->cap)),
                        reinterpret_cast<const uint32_t *>(b->d_buf[i] + off_first(b->cap)),
                        reinterpret_cast<BatchHeader *>(b->d_buf[i]), s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) return cuda_fail(e, "batch: end capture");
    b->graph[i] = g;
    e = cudaGraphInstantiate(&b->exec[i], g, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch: instantiate");
    return MPHF_OK;
}

// Fills staging buffer `hb` from the requests.
static int stage_requests(mphf_batch *b, uint8_t *hb, const mphf_request *reqs, uint32_t nreq, uint32_t *total_tiles_out) {
    if (nreq > b->cap) { set_error("%u requests, batch capacity %u", nreq, b->cap); return MPHF_ERR_CAPACITY; }
    BatchHeader *hdr = reinterpret_cast<BatchHeader *>(hb);
    uint32_t *first = reinterpret_cast<uint32_t *>(hb + off_first(b->cap));
    BatchDesc *desc = reinterpret_cast<BatchDesc *>(hb + off_desc(b->cap));
    const uint64_t TK = 32ull * b->cfg.keys_per_thread;   // one warp's tile
    uint64_t tiles = 0;
    for (uint32_t i = 0; i < nreq; i++) {
        const mphf_request &r = reqs[i];
        if (!r.m || (r.count && (!r.keys_dev || !r.out_dev)) || r.count > 0xFFFFFFFFull) {
            set_error("request %u: bad structure, pointers or count", i);
            return MPHF_ERR_ARG;
        }
        const Header &h = handle_header(r.m);
        if (wide_values(h.n) || h.hash128) {
            set_error("request %u: n > 2^32 or a 128-bit string hash (use mphf_query_*_wide)", i);
            return MPHF_ERR_ARG;
        }
        if ((h.key_kind == MPHF_KEY_BYTES) != (r.offsets_dev != nullptr)) {
            set_error("request %u: offsets must be given exactly for byte-key structures", i);
            return MPHF_ERR_ARG;
        }
        if (h.key_kind == MPHF_KEY_U64 && ((uintptr_t)r.keys_dev & 7)) { set_error("request %u: keys not 8-byte aligned", i); return MPHF_ERR_ARG; }
        if (((uintptr_t)r.out_dev & 3)) { set_error("request %u: out not 4-byte aligned", i); return MPHF_ERR_ARG; }
        BatchDesc &d = desc[i];
        d.v = handle_view(r.m);
        d.keys = r.keys_dev;
        d.offsets = r.offsets_dev;
        d.out = r.out_dev;
        d.count = (uint32_t)r.count;
        d.gamma = (uint8_t)h.gamma;
        d.reduce = (uint8_t)h.reduce;
        d.remap = (uint8_t)h.remap;
        d.key_kind = (uint8_t)h.key_kind;
        first[i] = (uint32_t)tiles;
        tiles += (r.count + TK - 1) / TK;
        if (tiles > 0xFFFFFFF0ull) { set_error("too many tiles in one batch"); return MPHF_ERR_CAPACITY; }
    }
    first[nreq] = (uint32_t)tiles;
    hdr->nreq = nreq;
    hdr->total_tiles = (uint32_t)tiles;
    hdr->counter = 0;
    hdr->pad = 0;
    *total_tiles_out = (uint32_t)tiles;
    return MPHF_OK;
}

extern "C" {

int mphf_batch_create(uint32_t max_requests, mphf_batch_t **out) {
    if (!out) { set_error("out is NULL"); return MPHF_ERR_ARG; }
    *out = nullptr;
    if (max_requests == 0 || max_requests > kMaxReqSmem) {
        set_error("max_requests must be in [1, %d]", kMaxReqSmem);
        return MPHF_ERR_ARG;
    }
    mphf_batch *b = new (std::nothrow) mphf_batch();
    if (!b) { set_error("host allocation"); return MPHF_ERR_OOM; }
    b->cap = max_requests;
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    b->buf_bytes = off_desc(max_requests) + (size_t)max_requests * sizeof(BatchDesc);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    for (int i = 0; i < kStages && e == cudaSuccess; i++) {
        e = cudaHostAlloc(&b->h_buf[i], b->buf_bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_buf[i], b->buf_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) memset(b->h_buf[i], 0, b->buf_bytes);
    }
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "batch: allocation");
        mphf_batch_free(b);
        return rc;
    }
    *out = b;
    return MPHF_OK;
}

void mphf_batch_free(mphf_batch_t *b) {
    if (!b) return;
    for (int i = 0; i < kStages; i++)
        if (b->done[i]) cudaEventSynchronize(b->done[i]);
    free_graphs(b);
    for (int i = 0; i < kStages; i++) {
        if (b->done[i]) cudaEventDestroy(b->done[i]);
        cudaFree(b->d_buf[i]);
        cudaFreeHost(b->h_buf[i]);
    }
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

int mphf_batch_set_config(mphf_batch_t *b, const mphf_batch_config *c) {
    if (!b || !c) { set_error("NULL argument"); return MPHF_ERR_ARG; }
    BatchConfig nc{c->keys_per_thread, c->threads, c->blocks_per_sm};
    if (!valid_config(nc)) { set_error("keys_per_thread in {2,4,8,16}, threads in {128,256,512}, blocks_per_sm in [1,16]"); return MPHF_ERR_ARG; }
    std::lock_guard<std::mutex> lock(b->mu);
    for (int i = 0; i < kStages; i++) cudaEventSynchronize(b->done[i]);
    b->cfg = nc;
    b->use_graph = c->use_graph != 0;
    free_graphs(b);
    return MPHF_OK;
}

int mphf_batch_get_config(const mphf_batch_t *b, mphf_batch_config *c) {
    if (!b || !c) { set_error("NULL argument"); return MPHF_ERR_ARG; }
    c->keys_per_thread = b->cfg.keys_per_thread;
    c->threads = b->cfg.threads;
    c->blocks_per_sm = b->cfg.blocks_per_sm;
    c->use_graph = b->use_graph;
    return MPHF_OK;
}

// Stages the requests into the next staging set (after that set's previous
// run finished) and launches its graph on `stream`.  Asynchronous.
int mphf_batch_run(mphf_batch_t *b, const mphf_request *reqs, uint32_t nreq, void *stream) {
    if (!b || (nreq && !reqs)) { set_error("NULL argument"); return MPHF_ERR_ARG; }
    std::lock_guard<std::mutex> lock(b->mu);
    cudaStream_t s = (cudaStream_t)stream;
    const int i = (int)(b->runs % kStages);
    cudaError_t e = cudaEventSynchronize(b->done[i]);
    if (e != cudaSuccess) return cuda_fail(e, "batch: previous run of this staging set");
    uint32_t tiles = 0;
    int rc = stage_requests(b, b->h_buf[i], reqs, nreq, &tiles);
    if (rc) return rc;
    if (tiles == 0) return MPHF_OK;
    if (b->use_graph) {
        if (!b->exec[i]) {
            rc = capture_graph(b, i);
            if (rc) return rc;
        }
        e = cudaGraphLaunch(b->exec[i], s);
        count_launch();
        if (e != cudaSuccess) return cuda_fail(e, "batch: graph launch");
    } else {
        e = cudaMemcpyAsync(b->d_buf[i], b->h_buf[i], b->buf_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch: descriptor upload");
        e = launch_batch_kernel(b->cfg, b->sms, reinterpret_cast<const BatchDesc *>(b->d_buf[i] + off_desc(b->cap)),
                                reinterpret_cast<const uint32_t *>(b->d_buf[i] + off_first(b->cap)),
                                reinterpret_cast<BatchHeader *>(b->d_buf[i]), s);
        if (e != cudaSuccess) return cuda_fail(e, "batch: kernel launch");
    }
    e = cudaEventRecord(b->done[i], s);
    if (e != cudaSuccess) return cuda_fail(e, "batch: event");
    b->runs++;
    return MPHF_OK;
}

// Times every candidate launch shape on this batch (best of 3 after one
// warm-up) and keeps the fastest.  With cache_path, the result is read from
// / appended to a JSON-lines file keyed by (key kind, log10 of total keys,
// SM count), so the search runs once per workload class.
int mphf_batch_autotune(mphf_batch_t *b, const mphf_request *reqs, uint32_t nreq, void *stream,
                        const char *cache_path, mphf_batch_config *best_out) {
    if (!b || !reqs || nreq == 0) { set_error("NULL argument or empty batch"); return MPHF_ERR_ARG; }
    uint64_t total = 0;
    int kind = MPHF_KEY_U64;
    for (uint32_t i = 0; i < nreq; i++) {
        total += reqs[i].count;
        if (reqs[i].offsets_dev) kind = MPHF_KEY_BYTES;
    }
    const int decade = total ? (int)floor(log10((double)total)) : 0;
    // The build stamp keeps a shape measured on another build of the kernel
    // (whose best shape may differ) from being reused.
    char key[192];
    snprintf(key, sizeof(key), "\"kind\": %d, \"log10_keys\": %d, \"sms\": %d, \"build\": \"%s %s\"", kind, decade,
             b->sms, __DATE__, __TIME__);
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[512];
            while (fgets(line, sizeof(line), f)) {
                if (!strstr(line, key)) continue;
                mphf_batch_config c{};
                const char *p = strstr(line, "\"keys_per_thread\": ");
                const char *q = strstr(line, "\"threads\": ");
                const char *r = strstr(line, "\"blocks_per_sm\": ");
                if (p && q && r) {
                    c.keys_per_thread = atoi(p + 19);
                    c.threads = atoi(q + 11);
                    c.blocks_per_sm = atoi(r + 17);
                    c.use_graph = 1;
                    if (valid_config({c.keys_per_thread, c.threads, c.blocks_per_sm})) {
                        fclose(f);
                        if (best_out) *best_out = c;
                        return mphf_batch_set_config(b, &c);
                    }
                }
            }
            fclose(f);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "events");
    const int kpts[] = {2, 4, 8, 16}, thr[] = {128, 256, 512}, bps[] = {1, 2, 4, 8};
    float best = 1e30f;
    mphf_batch_config bestc{8, 256, 4, 1};
    for (int k : kpts)
        for (int t : thr)
            for (int o : bps) {
                if (t * o > 2048) continue;
                mphf_batch_config c{k, t, o, 0};
                int rc = mphf_batch_set_config(b, &c);
                if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
                float ms_best = 1e30f;
                for (int rep = 0; rep < 4; rep++) {
                    cudaEventRecord(e0, s);
                    rc = mphf_batch_run(b, reqs, nreq, stream);
                    cudaEventRecord(e1, s);
                    if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
                    cudaEventSynchronize(e1);
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) ms_best = std::min(ms_best, ms);
                }
                if (ms_best < best) { best = ms_best; bestc = c; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bestc.use_graph = 1;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "{%s, \"keys_per_thread\": %d, \"threads\": %d, \"blocks_per_sm\": %d, \"ms\": %.4f}\n", key,
                    bestc.keys_per_thread, bestc.threads, bestc.blocks_per_sm, best);
            fclose(f);
        }
    }
    if (best_out) *best_out = bestc;
    return mphf_batch_set_config(b, &bestc);
}

}  // extern "C"
