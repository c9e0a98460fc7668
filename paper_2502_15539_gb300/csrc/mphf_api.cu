// C ABI of libmphf: structure handle, parameter rule, serialized format,
// error reporting and the host-buffer query pipeline.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "mphf_internal.cuh"

struct mphf {
    ptrhash::Header hdr;
    uint8_t *d_pilots = nullptr;
    uint8_t *d_remap = nullptr;
    int device = 0;
    uint64_t evictions = 0;
    double build_ms = 0.0;
    double hash_sort_ms = 0.0, search_ms = 0.0, remap_ms = 0.0;
    // Staging for mphf_query_u64_host: two buffer sets, two copy streams.
    std::mutex stage_mu;
    uint64_t stage_chunk = 0;
    uint64_t *d_stage_keys[2] = {nullptr, nullptr};
    uint32_t *d_stage_out[2] = {nullptr, nullptr};
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_h2d[2] = {}, ev_q[2] = {}, ev_d2h[2] = {};
    bool owns_device_memory = true;   // false: pilots / remap live in a caller's arena
    // Scratch of the windowed query (6 bytes per key of a chunk rounded up
    // to 16 keys; win_chunk holds that rounded count), allocated
    // on first use and kept; win_done orders its uses on different streams.
    std::mutex win_mu;
    uint8_t *d_win = nullptr;
    uint64_t win_chunk = 0;
    cudaEvent_t win_done = nullptr;
};

namespace ptrhash {

static thread_local char g_err[512] = "no error";
static std::atomic<uint64_t> g_launches{0};

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    if (e == cudaErrorMemoryAllocation) return MPHF_ERR_OOM;
    return MPHF_ERR_CUDA;
}

void count_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static bool is_pow2(uint64_t v) { return v && !(v & (v - 1)); }

// Sec. 3.1 "Parameter values": alpha S >= 80000 ln(n / 80000) keys per part
// (at least 80000), S the smallest power of two that holds them, P =
// ceil(n / (alpha S)), B = ceil(alpha S / lambda).  When that wastes more
// than 5% of n/alpha slots (few parts), reduce becomes x mod S with P =
// ceil(n / kpp), S = max(ceil(n / (alpha P)), ceil(n/P) + 16), made odd: the
// paper wants S not a power of two so that x mod S depends on every bit of x,
// and an even S would let keys whose hashes share trailing zero bits (h = C k
// keeps those of k) reach only S / gcd(S, 2^t) slots.  A forced S keeps P =
// ceil(n / (alpha S)).
int choose_layout(uint64_t n, double lambda, double alpha, uint64_t slots_override,
                  uint64_t *P_out, uint64_t *S_out, uint64_t *B_out, int *reduce_out) {
    if (n == 0 || n > kMaxKeys || !(lambda > 0.0) || !(alpha > 0.0) || alpha > 1.0) {
        set_error("invalid n=%llu, lambda=%g or alpha=%g", (unsigned long long)n, lambda, alpha);
        return MPHF_ERR_ARG;
    }
    const double nd = (double)n;
    const double keys_per_part = fmax(80000.0, 80000.0 * log(nd / 80000.0));
    uint64_t S, P;
    int reduce;
    if (slots_override) {
        S = slots_override;
        P = (uint64_t)ceil(nd / (alpha * (double)S));
        reduce = is_pow2(S) ? kReducePow2 : kReduceMod;
    } else {
        int k = 0;
        while ((double)(1ull << k) < keys_per_part / alpha) k++;
        S = 1ull << k;
        P = (uint64_t)ceil(nd / (alpha * (double)S));
        reduce = kReducePow2;
        if ((double)(P * S) > 1.05 * nd / alpha) {
            P = (uint64_t)ceil(nd / keys_per_part);
            if (P == 0) P = 1;
            S = (uint64_t)ceil(nd / (alpha * (double)P));
            const uint64_t floor_s = (n + P - 1) / P + 16;
            if (S < floor_s) S = floor_s;
            if (S % 2 == 0) S++;
            reduce = kReduceMod;
        }
    }
    if (P == 0) P = 1;
    uint64_t B = (uint64_t)ceil(alpha * (double)S / lambda);
    if (B == 0) B = 1;
    if (P * S < n || P * S - n >= kMaxKeys || S > 0xFFFFFFFFull || B > 0xFFFFFFFEull) {
        set_error("layout out of range: P=%llu S=%llu B=%llu", (unsigned long long)P,
                  (unsigned long long)S, (unsigned long long)B);
        return MPHF_ERR_ARG;
    }
    *P_out = P;
    *S_out = S;
    *B_out = B;
    *reduce_out = reduce;
    return MPHF_OK;
}

uint64_t barrett_constant(uint64_t S) {
    return (uint64_t)(((unsigned __int128)1 << 64) / S);   // floor(2^64 / S), S >= 2
}

uint64_t clef_lines_for(uint64_t remap_len) { return (remap_len + kClefPerLine - 1) / kClefPerLine; }

View make_view(const Header &h, const uint8_t *pilots, const void *remap) {
    View v;
    v.pilots = pilots;
    v.remap = remap;
    v.n = h.n; v.P = h.P; v.S = h.S; v.B = h.B; v.C = h.C; v.seed = h.seed;
    v.s_mask = h.S - 1;
    v.fm = v.fm_unused = 0;
    if (h.reduce == kReduceMod) v.fm = barrett_constant(h.S);
    return v;
}

const Header &handle_header(const mphf *m) { return m->hdr; }
View handle_view(const mphf *m) { return make_view(m->hdr, m->d_pilots, m->d_remap); }

}  // namespace ptrhash

using namespace ptrhash;

// ------------------------------------------------------------- serialize
// 128-byte little-endian header; see include/mphf.h.
static void wr64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void wr32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static uint64_t rd64(const uint8_t *p) { uint64_t v = 0; for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i); return v; }
static uint32_t rd32(const uint8_t *p) { uint32_t v = 0; for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i); return v; }
static uint64_t round64(uint64_t v) { return (v + 63) & ~63ull; }

static const char kMagic[8] = {'P', 'T', 'R', 'H', 'A', 'S', 'H', '1'};

extern "C" {

int mphf_default_params(mphf_params *p) {
    if (!p) { set_error("params is NULL"); return MPHF_ERR_ARG; }
    memset(p, 0, sizeof(*p));
    p->lambda = 3.5;
    p->alpha = 0.99;
    p->gamma = MPHF_GAMMA_CUBIC;
    p->remap = MPHF_REMAP_CLEF;
    p->seed = 0;
    p->C = 0x9E3779B97F4A7C15ull;   // any odd constant; the paper prints none
    p->slots_override = 0;
    p->max_reseeds = 8;
    p->evict_mult = 10;             // "a total of 10S evictions" (Sec. 4.1.2)
    return MPHF_OK;
}

int mphf_layout(const mphf_params *params, uint64_t n, mphf_info_t *out) {
    if (!params || !out) { set_error("NULL argument"); return MPHF_ERR_ARG; }
    memset(out, 0, sizeof(*out));
    uint64_t P, S, B;
    int reduce;
    int rc = choose_layout(n, params->lambda, params->alpha, params->slots_override, &P, &S, &B, &reduce);
    if (rc) return rc;
    out->n = n; out->P = P; out->S = S; out->B = B; out->reduce = reduce;
    out->C = params->C; out->seed = params->seed; out->gamma = params->gamma; out->remap = params->remap;
    out->remap_len = P * S - n;
    out->pilot_bytes = P * B;
    out->remap_bytes = params->remap == MPHF_REMAP_VEC ? vec_entry_bytes(n) * out->remap_len
                                                       : 64 * clef_lines_for(out->remap_len);
    out->bits_per_key = 8.0 * (double)(out->pilot_bytes + out->remap_bytes) / (double)n;
    return MPHF_OK;
}

int mphf_serialize(const mphf_t *m, void *host_buf, size_t cap, size_t *needed) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    const Header &h = m->hdr;
    const uint64_t pb = h.P * h.B;
    const uint64_t need = 128 + round64(pb) + h.remap_bytes;
    if (needed) *needed = need;
    if (!host_buf) return MPHF_OK;
    if (cap < need) { set_error("buffer of %zu bytes, %llu needed", cap, (unsigned long long)need); return MPHF_ERR_ARG; }
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(m->device);
    uint8_t *b = (uint8_t *)host_buf;
    memset(b, 0, 128 + round64(pb));
    memcpy(b, kMagic, 8);
    wr32(b + 8, 1);
    wr32(b + 12, (uint32_t)h.key_kind);
    wr32(b + 16, (uint32_t)h.gamma);
    wr32(b + 20, (uint32_t)h.remap);
    wr32(b + 24, (uint32_t)h.reduce);
    wr32(b + 28, h.hash128 ? 1u : 0u);   // flags: bit 0 = 128-bit string hash
    wr64(b + 32, h.n); wr64(b + 40, h.P); wr64(b + 48, h.S); wr64(b + 56, h.B);
    wr64(b + 64, h.C); wr64(b + 72, h.seed);
    wr64(b + 80, h.remap_len); wr64(b + 88, h.remap_bytes);
    uint64_t lb, ab;
    memcpy(&lb, &h.lambda, 8); memcpy(&ab, &h.alpha, 8);
    wr64(b + 96, lb); wr64(b + 104, ab);
    wr64(b + 112, pb);
    cudaError_t e = cudaMemcpy(b + 128, m->d_pilots, pb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h.remap_bytes)
        e = cudaMemcpy(b + 128 + round64(pb), m->d_remap, h.remap_bytes, cudaMemcpyDeviceToHost);
    cudaSetDevice(dev_prev);
    if (e != cudaSuccess) return cuda_fail(e, "serialize: device to host copy");
    return MPHF_OK;
}

static void free_handle(mphf_t *m) {
    if (!m) return;
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(m->device);
    if (m->owns_device_memory) {
        cudaFree(m->d_pilots);
        cudaFree(m->d_remap);
    }
    for (int i = 0; i < 2; i++) {
        cudaFree(m->d_stage_keys[i]);
        cudaFree(m->d_stage_out[i]);
        if (m->ev_h2d[i]) cudaEventDestroy(m->ev_h2d[i]);
        if (m->ev_q[i]) cudaEventDestroy(m->ev_q[i]);
        if (m->ev_d2h[i]) cudaEventDestroy(m->ev_d2h[i]);
    }
    if (m->s_h2d) cudaStreamDestroy(m->s_h2d);
    if (m->s_d2h) cudaStreamDestroy(m->s_d2h);
    cudaFree(m->d_win);
    if (m->win_done) cudaEventDestroy(m->win_done);
    cudaSetDevice(dev_prev);
    delete m;
}

}  // extern "C"

// Parses and checks a serialized header; *pb gets the pilot byte count.
static int parse_serialized(const uint8_t *b, size_t len, Header *out, uint64_t *pb_out) {
    if (len < 128 || memcmp(b, kMagic, 8) != 0 || rd32(b + 8) != 1) {
        set_error("not a PtrHash v1 structure");
        return MPHF_ERR_FORMAT;
    }
    Header h;
    h.key_kind = (int32_t)rd32(b + 12);
    h.gamma = (int32_t)rd32(b + 16);
    h.remap = (int32_t)rd32(b + 20);
    h.reduce = (int32_t)rd32(b + 24);
    const uint32_t flags = rd32(b + 28);
    h.hash128 = (int32_t)(flags & 1u);
    h.n = rd64(b + 32); h.P = rd64(b + 40); h.S = rd64(b + 48); h.B = rd64(b + 56);
    h.C = rd64(b + 64); h.seed = rd64(b + 72);
    h.remap_len = rd64(b + 80); h.remap_bytes = rd64(b + 88);
    uint64_t lb = rd64(b + 96), ab = rd64(b + 104);
    memcpy(&h.lambda, &lb, 8); memcpy(&h.alpha, &ab, 8);
    const uint64_t pb = rd64(b + 112);
    bool bad = (h.key_kind != MPHF_KEY_U64 && h.key_kind != MPHF_KEY_BYTES) ||
               (h.gamma != MPHF_GAMMA_LINEAR && h.gamma != MPHF_GAMMA_CUBIC) ||
               (h.remap != MPHF_REMAP_CLEF && h.remap != MPHF_REMAP_VEC) ||
               (h.reduce != kReducePow2 && h.reduce != kReduceMod) ||
               flags > 1u || (h.hash128 && h.key_kind != MPHF_KEY_BYTES) ||
               h.n == 0 || h.n > kMaxKeys || h.P == 0 || h.S == 0 || h.B == 0 ||
               h.S > 0xFFFFFFFFull || h.P > 0xFFFFFFFFull || h.B > 0xFFFFFFFFull ||
               pb != h.P * h.B || h.P * h.S < h.n || h.P * h.S - h.n >= kMaxKeys ||
               h.remap_len != h.P * h.S - h.n || (h.C & 1) == 0 ||
               (h.reduce == kReducePow2 && !is_pow2(h.S)) ||
               (h.reduce == kReduceMod && is_pow2(h.S));
    if (!bad) {
        uint64_t want = h.remap == MPHF_REMAP_CLEF ? 64 * clef_lines_for(h.remap_len)
                                                   : vec_entry_bytes(h.n) * h.remap_len;
        bad = h.remap_bytes != want || len < 128 + round64(pb) + h.remap_bytes;
    }
    if (bad) { set_error("inconsistent header fields"); return MPHF_ERR_FORMAT; }
    *out = h;
    *pb_out = pb;
    return MPHF_OK;
}

namespace ptrhash {

// Device bytes a serialized structure needs in an arena (256-byte aligned parts).
int serialized_device_bytes(const void *blob, size_t len, uint64_t *bytes, uint64_t *n) {
    Header h;
    uint64_t pb = 0;
    int rc = parse_serialized((const uint8_t *)blob, len, &h, &pb);
    if (rc) return rc;
    *bytes = ((pb + 255) & ~255ull) + ((h.remap_bytes + 255) & ~255ull);
    if (n) *n = h.n;
    return MPHF_OK;
}

// A handle whose pilots and remap live at `dev` (caller-owned, at least
// serialized_device_bytes long); the copies are queued on `s`.
int handle_in_arena(const void *blob, size_t len, uint8_t *dev, cudaStream_t s, mphf_t **out) {
    *out = nullptr;
    Header h;
    uint64_t pb = 0;
    const uint8_t *b = (const uint8_t *)blob;
    int rc = parse_serialized(b, len, &h, &pb);
    if (rc) return rc;
    mphf_t *m = new (std::nothrow) mphf_t();
    if (!m) { set_error("host allocation"); return MPHF_ERR_OOM; }
    m->hdr = h;
    m->owns_device_memory = false;
    cudaGetDevice(&m->device);
    m->d_pilots = dev;
    m->d_remap = dev + ((pb + 255) & ~255ull);
    cudaError_t e = cudaMemcpyAsync(m->d_pilots, b + 128, pb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && h.remap_bytes)
        e = cudaMemcpyAsync(m->d_remap, b + 128 + round64(pb), h.remap_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "arena load: copy");
    }
    *out = m;
    return MPHF_OK;
}

}  // namespace ptrhash

extern "C" {

int mphf_deserialize(const void *host_buf, size_t len, mphf_t **out) {
    if (!out) { set_error("out is NULL"); return MPHF_ERR_ARG; }
    *out = nullptr;
    if (!host_buf) { set_error("buffer is NULL"); return MPHF_ERR_ARG; }
    const uint8_t *b = (const uint8_t *)host_buf;
    Header h;
    uint64_t pb = 0;
    int rc = parse_serialized(b, len, &h, &pb);
    if (rc) return rc;
    mphf_t *m = new (std::nothrow) mphf_t();
    if (!m) { set_error("host allocation"); return MPHF_ERR_OOM; }
    m->hdr = h;
    cudaGetDevice(&m->device);
    cudaError_t e = cudaMalloc(&m->d_pilots, round64(pb));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_remap, h.remap_bytes ? round64(h.remap_bytes) : 64);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_pilots, b + 128, pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && h.remap_bytes)
        e = cudaMemcpy(m->d_remap, b + 128 + round64(pb), h.remap_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "deserialize: device allocation or copy");
        free_handle(m);
        return rc;
    }
    *out = m;
    return MPHF_OK;
}

int mphf_build(const mphf_params *params, int key_kind, const void *keys_dev,
               const uint64_t *offsets_dev, uint64_t n, void *stream, mphf_t **out) {
    if (!out) { set_error("out is NULL"); return MPHF_ERR_ARG; }
    *out = nullptr;
    if (!params || !keys_dev) { set_error("NULL params or keys"); return MPHF_ERR_ARG; }
    if (key_kind == MPHF_KEY_U64 && (offsets_dev || ((uintptr_t)keys_dev & 7))) {
        set_error("u64 keys need 8-byte alignment and no offsets");
        return MPHF_ERR_ARG;
    }
    if (key_kind == MPHF_KEY_BYTES && (!offsets_dev || ((uintptr_t)offsets_dev & 7))) {
        set_error("byte keys need n+1 aligned u64 offsets");
        return MPHF_ERR_ARG;
    }
    if (key_kind != MPHF_KEY_U64 && key_kind != MPHF_KEY_BYTES) { set_error("bad key kind"); return MPHF_ERR_ARG; }
    BuildResult r;
    int rc = build_structure(*params, key_kind, keys_dev, offsets_dev, n, (cudaStream_t)stream, &r);
    if (rc) return rc;
    mphf_t *m = new (std::nothrow) mphf_t();
    if (!m) {
        cudaFree(r.d_pilots);
        cudaFree(r.d_remap);
        set_error("host allocation");
        return MPHF_ERR_OOM;
    }
    m->hdr = r.hdr;
    m->d_pilots = r.d_pilots;
    m->d_remap = r.d_remap;
    m->evictions = r.evictions;
    m->build_ms = r.build_ms;
    m->hash_sort_ms = r.hash_sort_ms;
    m->search_ms = r.search_ms;
    m->remap_ms = r.remap_ms;
    cudaGetDevice(&m->device);
    *out = m;
    return MPHF_OK;
}

int mphf_info(const mphf_t *m, mphf_info_t *out) {
    if (!m || !out) { set_error("NULL argument"); return MPHF_ERR_ARG; }
    const Header &h = m->hdr;
    memset(out, 0, sizeof(*out));
    out->n = h.n; out->P = h.P; out->S = h.S; out->B = h.B; out->C = h.C; out->seed = h.seed;
    out->gamma = h.gamma; out->remap = h.remap; out->reduce = h.reduce; out->key_kind = h.key_kind;
    out->remap_len = h.remap_len;
    out->pilot_bytes = h.P * h.B;
    out->remap_bytes = h.remap_bytes;
    out->bits_per_key = 8.0 * (double)(out->pilot_bytes + out->remap_bytes) / (double)h.n;
    out->evictions = m->evictions;
    out->build_ms = m->build_ms;
    out->build_hash_sort_ms = m->hash_sort_ms;
    out->build_search_ms = m->search_ms;
    out->build_remap_ms = m->remap_ms;
    return MPHF_OK;
}

void mphf_free(mphf_t *m) { free_handle(m); }

int mphf_device_view(const mphf_t *m, mphf_view_t *out) {
    if (!m || !out) { set_error("NULL argument"); return MPHF_ERR_ARG; }
    const Header &h = m->hdr;
    memset(out, 0, sizeof(*out));
    out->pilots = m->d_pilots;
    out->remap = m->d_remap;
    out->n = h.n; out->P = h.P; out->S = h.S; out->B = h.B; out->C = h.C; out->seed = h.seed;
    out->barrett = h.reduce == kReduceMod ? barrett_constant(h.S) : 0;
    out->s_mask = h.S - 1;
    out->gamma = h.gamma; out->reduce = h.reduce; out->remap_kind = h.remap; out->key_kind = h.key_kind;
    out->hash128 = h.hash128;
    return MPHF_OK;
}

static int check_query_u64(const mphf_t *m, const uint64_t *keys_dev, const uint32_t *out_dev) {
    if (!keys_dev || !out_dev || ((uintptr_t)keys_dev & 7) || ((uintptr_t)out_dev & 3)) {
        set_error("keys must be 8-byte and out 4-byte aligned device pointers");
        return MPHF_ERR_ARG;
    }
    if (m->hdr.key_kind != MPHF_KEY_U64) { set_error("structure was built for byte keys"); return MPHF_ERR_ARG; }
    if (wide_values(m->hdr.n)) { set_error("n > 2^32: values need the _wide query"); return MPHF_ERR_ARG; }
    return MPHF_OK;
}

}  // extern "C"

namespace ptrhash {

// The windowed query on the handle's scratch.  Returns MPHF_ERR_OOM (and
// leaves no CUDA error pending) if the scratch cannot be allocated.
int handle_windowed_query(const mphf_t *mc, const uint64_t *keys, uint64_t count, void *out, int mode,
                          const void *table, uint64_t W, uint64_t chunk_keys, cudaStream_t s) {
    mphf_t *m = const_cast<mphf_t *>(mc);   // the scratch is mutable state of a const structure
    const uint64_t chunk = window_chunk_for(count, chunk_keys);
    const uint64_t cp = window_stream_keys(chunk);   // the scratch holds 6 bytes per padded key
    std::lock_guard<std::mutex> lock(m->win_mu);
    if (m->win_chunk < cp) {
        if (m->d_win) {   // grow: cudaFree waits for every earlier use
            cudaFree(m->d_win);
            m->d_win = nullptr;
            m->win_chunk = 0;
        }
        cudaError_t e = cudaMalloc(&m->d_win, 6 * cp);
        if (e != cudaSuccess) {
            m->d_win = nullptr;
            cudaGetLastError();
            return cuda_fail(e, "windowed query scratch");
        }
        m->win_chunk = cp;
    }
    if (!m->win_done) {
        cudaError_t e = cudaEventCreateWithFlags(&m->win_done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "windowed query event");
    }
    // A use on another stream may still run: wait for it on the GPU.
    cudaError_t e = cudaStreamWaitEvent(s, m->win_done, 0);
    if (e != cudaSuccess) return cuda_fail(e, "windowed query: order after the previous use");
    View v = make_view(m->hdr, m->d_pilots, m->d_remap);
    const int rc = launch_query_u64_windowed(m->hdr, v, keys, count, out, mode, table, W, chunk, m->d_win, s);
    e = cudaEventRecord(m->win_done, s);
    if (rc == MPHF_OK && e != cudaSuccess) return cuda_fail(e, "windowed query: record");
    return rc;
}

// The automatic choice of the query entry points: the windowed path for a
// large batch against a pilot array above the window size, with buffers
// aligned for it.  Returns 1 if it ran (rc holds its result), 0 if the
// single pass should run (not applicable, or no room for the scratch).
int try_windowed(const mphf_t *m, const uint64_t *keys, uint64_t count, void *out, int mode, const void *table,
                 cudaStream_t s, int *rc) {
    const uint64_t W = window_plan(m->hdr, count);
    if (W < 2 || !window_supported(m->hdr, keys, out, window_out_bytes(mode))) return 0;
    *rc = handle_windowed_query(m, keys, count, out, mode, table, W, 0, s);
    return *rc != MPHF_ERR_OOM;
}

}  // namespace ptrhash

extern "C" {

int mphf_query_u64(const mphf_t *m, const uint64_t *keys_dev, uint64_t count, uint32_t *out_dev,
                   void *stream) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    if (count == 0) return MPHF_OK;
    int rc = check_query_u64(m, keys_dev, out_dev);
    if (rc) return rc;
    // No room for the windowed path's scratch: the single pass needs none.
    if (try_windowed(m, keys_dev, count, out_dev, kWinMphf32, nullptr, (cudaStream_t)stream, &rc)) return rc;
    View v = make_view(m->hdr, m->d_pilots, m->d_remap);
    return launch_query_u64(m->hdr, v, keys_dev, count, out_dev, false, (cudaStream_t)stream);
}

int mphf_query_u64_windowed(const mphf_t *m, const uint64_t *keys_dev, uint64_t count, uint32_t *out_dev,
                            uint64_t window_bytes, uint64_t chunk_keys, void *stream) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    if (count == 0) return MPHF_OK;
    int rc = check_query_u64(m, keys_dev, out_dev);
    if (rc) return rc;
    if (chunk_keys % 2 || chunk_keys > (1ull << 31)) {
        set_error("chunk_keys must be even and at most 2^31 (0: the default)");
        return MPHF_ERR_ARG;
    }
    const uint64_t W = window_count_for(m->hdr.P * m->hdr.B, window_bytes);
    if (W < 2) {
        View v = make_view(m->hdr, m->d_pilots, m->d_remap);
        return launch_query_u64(m->hdr, v, keys_dev, count, out_dev, false, (cudaStream_t)stream);
    }
    if (!window_supported(m->hdr, keys_dev, out_dev, 4)) {
        set_error("windowed query: keys 16-byte and out 8-byte aligned, P B < 2^32");
        return MPHF_ERR_ARG;
    }
    return handle_windowed_query(m, keys_dev, count, out_dev, kWinMphf32, nullptr, W, chunk_keys, (cudaStream_t)stream);
}

int mphf_bucket_u64(const mphf_t *m, const uint64_t *keys_dev, uint64_t count, uint64_t *out_dev, void *stream) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    if (count == 0) return MPHF_OK;
    if (!keys_dev || !out_dev || ((uintptr_t)keys_dev & 7) || ((uintptr_t)out_dev & 7)) {
        set_error("keys and out must be 8-byte aligned device pointers");
        return MPHF_ERR_ARG;
    }
    if (m->hdr.key_kind != MPHF_KEY_U64) { set_error("structure was built for byte keys"); return MPHF_ERR_ARG; }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attributes");
    View v = make_view(m->hdr, m->d_pilots, m->d_remap);
    return launch_bucket_u64(m->hdr, v, keys_dev, count, out_dev, sms, (cudaStream_t)stream);
}

int mphf_query_u64_wide(const mphf_t *m, const uint64_t *keys_dev, uint64_t count, uint64_t *out_dev,
                        void *stream) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    if (count == 0) return MPHF_OK;
    if (!keys_dev || !out_dev || ((uintptr_t)keys_dev & 7) || ((uintptr_t)out_dev & 7)) {
        set_error("keys and out must be 8-byte aligned device pointers");
        return MPHF_ERR_ARG;
    }
    if (m->hdr.key_kind != MPHF_KEY_U64) { set_error("structure was built for byte keys"); return MPHF_ERR_ARG; }
    int rc = MPHF_OK;
    if (try_windowed(m, keys_dev, count, out_dev, kWinWide64, nullptr, (cudaStream_t)stream, &rc)) return rc;
    View v = make_view(m->hdr, m->d_pilots, m->d_remap);
    return launch_query_u64_wide(m->hdr, v, keys_dev, count, out_dev, (cudaStream_t)stream);
}

int mphf_query_u64_phf(const mphf_t *m, const uint64_t *keys_dev, uint64_t count, uint32_t *out_dev,
                       void *stream) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    if (count == 0) return MPHF_OK;
    if (!keys_dev || !out_dev || ((uintptr_t)keys_dev & 7) || ((uintptr_t)out_dev & 3)) {
        set_error("keys must be 8-byte and out 4-byte aligned device pointers");
        return MPHF_ERR_ARG;
    }
    if (m->hdr.key_kind != MPHF_KEY_U64) { set_error("structure was built for byte keys"); return MPHF_ERR_ARG; }
    if (m->hdr.P * m->hdr.S > (1ull << 32)) { set_error("P S > 2^32: slots do not fit 32 bits"); return MPHF_ERR_ARG; }
    int rc = MPHF_OK;
    if (try_windowed(m, keys_dev, count, out_dev, kWinPhf32, nullptr, (cudaStream_t)stream, &rc)) return rc;
    View v = make_view(m->hdr, m->d_pilots, m->d_remap);
    return launch_query_u64(m->hdr, v, keys_dev, count, out_dev, true, (cudaStream_t)stream);
}

int mphf_query_bytes(const mphf_t *m, const uint8_t *bytes_dev, const uint64_t *offsets_dev,
                     uint64_t count, uint32_t *out_dev, void *stream) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    if (count == 0) return MPHF_OK;
    if (!bytes_dev || !offsets_dev || !out_dev || ((uintptr_t)offsets_dev & 7) || ((uintptr_t)out_dev & 3)) {
        set_error("bad pointers for byte-key query");
        return MPHF_ERR_ARG;
    }
    if (m->hdr.key_kind != MPHF_KEY_BYTES) { set_error("structure was built for u64 keys"); return MPHF_ERR_ARG; }
    if (wide_values(m->hdr.n)) { set_error("n > 2^32: values need the _wide query"); return MPHF_ERR_ARG; }
    View v = make_view(m->hdr, m->d_pilots, m->d_remap);
    return launch_query_bytes(m->hdr, v, bytes_dev, offsets_dev, count, out_dev, (cudaStream_t)stream);
}

int mphf_query_bytes_wide(const mphf_t *m, const uint8_t *bytes_dev, const uint64_t *offsets_dev,
                          uint64_t count, uint64_t *out_dev, void *stream) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    if (count == 0) return MPHF_OK;
    if (!bytes_dev || !offsets_dev || !out_dev || ((uintptr_t)offsets_dev & 7) || ((uintptr_t)out_dev & 7)) {
        set_error("bad pointers for byte-key query");
        return MPHF_ERR_ARG;
    }
    if (m->hdr.key_kind != MPHF_KEY_BYTES) { set_error("structure was built for u64 keys"); return MPHF_ERR_ARG; }
    View v = make_view(m->hdr, m->d_pilots, m->d_remap);
    return launch_query_bytes_wide(m->hdr, v, bytes_dev, offsets_dev, count, out_dev, (cudaStream_t)stream);
}

// Host-buffer query: chunk c uses buffer set c % 2.  The copy in of chunk c
// waits for the kernel of chunk c-2 (same key buffer); the kernel of chunk c
// waits for its copy in and for the copy out of chunk c-2 (same output
// buffer); the copy out of chunk c waits for its kernel.  So copy-in,
// kernel and copy-out of consecutive chunks overlap.
int mphf_query_u64_host(mphf_t *m, const uint64_t *keys_host, uint64_t count, uint32_t *out_host,
                        void *stream) {
    if (!m) { set_error("structure is NULL"); return MPHF_ERR_ARG; }
    if (count == 0) return MPHF_OK;
    if (!keys_host || !out_host) { set_error("NULL host buffer"); return MPHF_ERR_ARG; }
    if (m->hdr.key_kind != MPHF_KEY_U64) { set_error("structure was built for byte keys"); return MPHF_ERR_ARG; }
    if (wide_values(m->hdr.n)) { set_error("n > 2^32: values need the _wide query"); return MPHF_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    // Page-locked host buffers are mapped into the device address space: the
    // kernel then reads the keys and writes the results across the host link
    // itself, with no staging copies.
    cudaPointerAttributes ak, ao;
    if (cudaPointerGetAttributes(&ak, keys_host) == cudaSuccess && ak.type == cudaMemoryTypeHost &&
        ak.devicePointer && cudaPointerGetAttributes(&ao, out_host) == cudaSuccess &&
        ao.type == cudaMemoryTypeHost && ao.devicePointer && ((uintptr_t)ak.devicePointer & 7) == 0 &&
        ((uintptr_t)ao.devicePointer & 3) == 0) {
        View v = make_view(m->hdr, m->d_pilots, m->d_remap);
        int rc = launch_query_u64(m->hdr, v, static_cast<const uint64_t *>(ak.devicePointer), count,
                                  static_cast<uint32_t *>(ao.devicePointer), false, s);
        if (rc) return rc;
        cudaError_t e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? MPHF_OK : cuda_fail(e, "host query: mapped buffers");
    }
    cudaGetLastError();   // a pageable pointer is not an error here
    std::lock_guard<std::mutex> lock(m->stage_mu);
    const uint64_t chunk = 1ull << 24;
    cudaError_t e = cudaSuccess;
    if (m->stage_chunk == 0) {   // resumable: a failed setup keeps what it made for the next call
        for (int i = 0; i < 2 && e == cudaSuccess; i++) {
            if (!m->d_stage_keys[i]) e = cudaMalloc(&m->d_stage_keys[i], chunk * sizeof(uint64_t));
            if (e == cudaSuccess && !m->d_stage_out[i]) e = cudaMalloc(&m->d_stage_out[i], chunk * sizeof(uint32_t));
            if (e == cudaSuccess && !m->ev_h2d[i]) e = cudaEventCreateWithFlags(&m->ev_h2d[i], cudaEventDisableTiming);
            if (e == cudaSuccess && !m->ev_q[i]) e = cudaEventCreateWithFlags(&m->ev_q[i], cudaEventDisableTiming);
            if (e == cudaSuccess && !m->ev_d2h[i]) e = cudaEventCreateWithFlags(&m->ev_d2h[i], cudaEventDisableTiming);
        }
        if (e == cudaSuccess && !m->s_h2d) e = cudaStreamCreateWithFlags(&m->s_h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess && !m->s_d2h) e = cudaStreamCreateWithFlags(&m->s_d2h, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "host query: staging setup");
        m->stage_chunk = chunk;
    }
    View v = make_view(m->hdr, m->d_pilots, m->d_remap);
    // Order the first copies after earlier work on the caller's stream.
    e = cudaEventRecord(m->ev_q[0], s);
    if (e == cudaSuccess) e = cudaEventRecord(m->ev_q[1], s);
    if (e == cudaSuccess) e = cudaEventRecord(m->ev_d2h[0], s);
    if (e == cudaSuccess) e = cudaEventRecord(m->ev_d2h[1], s);
    int rc = MPHF_OK;
    for (uint64_t off = 0, c = 0; off < count && e == cudaSuccess && rc == MPHF_OK; off += chunk, c++) {
        const int b = (int)(c & 1);
        const uint64_t cnt = count - off < chunk ? count - off : chunk;
        e = cudaStreamWaitEvent(m->s_h2d, m->ev_q[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_stage_keys[b], keys_host + off, cnt * 8, cudaMemcpyHostToDevice, m->s_h2d);
        if (e == cudaSuccess) e = cudaEventRecord(m->ev_h2d[b], m->s_h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->ev_h2d[b], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->ev_d2h[b], 0);
        if (e != cudaSuccess) break;
        rc = launch_query_u64(m->hdr, v, m->d_stage_keys[b], cnt, m->d_stage_out[b], false, s);
        if (rc) break;
        e = cudaEventRecord(m->ev_q[b], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->s_d2h, m->ev_q[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_host + off, m->d_stage_out[b], cnt * 4, cudaMemcpyDeviceToHost, m->s_d2h);
        if (e == cudaSuccess) e = cudaEventRecord(m->ev_d2h[b], m->s_d2h);
    }
    cudaError_t e2 = cudaStreamSynchronize(m->s_d2h);
    cudaError_t e3 = cudaStreamSynchronize(s);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "host query: copy pipeline");
    if (e2 != cudaSuccess) return cuda_fail(e2, "host query: copy-out stream");
    if (e3 != cudaSuccess) return cuda_fail(e3, "host query: compute stream");
    return MPHF_OK;
}

const char *mphf_strerror(int code) {
    switch (code) {
        case MPHF_OK: return "ok";
        case MPHF_ERR_ARG: return "invalid argument";
        case MPHF_ERR_OOM: return "out of memory";
        case MPHF_ERR_DUP_KEYS: return "duplicate keys";
        case MPHF_ERR_BUILD_FAILED: return "construction failed after every reseed";
        case MPHF_ERR_FORMAT: return "invalid serialized structure";
        case MPHF_ERR_CUDA: return "CUDA error";
        case MPHF_ERR_TIMEOUT: return "device wait timed out";
        case MPHF_ERR_OVERFULL: return "a part holds more keys than slots";
        case MPHF_ERR_CAPACITY: return "capacity exceeded";
        default: return "unknown error";
    }
}

const char *mphf_last_error(void) { return g_err; }

int mphf_set_l2_fetch_granularity(int bytes, int *previous) {
    if (bytes < 0 || bytes > 128) {
        set_error("L2 fetch granularity must be 0..128 bytes");
        return MPHF_ERR_ARG;
    }
    size_t old = 0;
    cudaError_t e = cudaDeviceGetLimit(&old, cudaLimitMaxL2FetchGranularity);
    if (e != cudaSuccess) return cuda_fail(e, "get L2 fetch granularity");
    e = cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "set L2 fetch granularity");
    if (previous) *previous = (int)old;
    return MPHF_OK;
}

uint64_t mphf_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
