// Context, scratch pool, errors, per-kernel timing, the tuning table and
// graph cache, and 2-bit packing.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "nw_internal.cuh"

namespace nw {

int fail(nw_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->msg = buf;
    }
    return code;
}

int cuda_fail(nw_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, NW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int scratch(nw_ctx *ctx, const char *name, size_t bytes, void **out) {
    Buf &b = ctx->bufs[name];
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) {
        *out = b.p;
        return NW_OK;
    }
    size_t want = bytes + bytes / 8;  // headroom to avoid regrowing by a few bytes
    want = (want + 255) & ~size_t(255);
    if (ctx->used - b.cap + want > ctx->budget) {
        want = (bytes + 255) & ~size_t(255);
        if (ctx->used - b.cap + want > ctx->budget)
            return fail(ctx, NW_ERR_OOM, "scratch '%s' needs %zu bytes; budget %llu, in use %llu", name, bytes,
                        (unsigned long long)ctx->budget, (unsigned long long)ctx->used);
    }
    if (b.p) {
        cudaError_t e = cudaFreeAsync(b.p, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFreeAsync");
        ctx->used -= b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    void *p = nullptr;
    cudaError_t e = ctx->mempool ? cudaMallocFromPoolAsync(&p, want, ctx->mempool, ctx->stream)
                                 : cudaMallocAsync(&p, want, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, NW_ERR_OOM, "cudaMallocAsync(%zu) for '%s': %s", want, name, cudaGetErrorString(e));
    }
    b.p = p;
    b.cap = want;
    ctx->used += want;
    *out = p;
    return NW_OK;
}

int check_scoring(nw_ctx *ctx, const nw_scoring &sc) {
    auto in = [](int v) { return v >= -40 && v <= 40; };
    if (!in(sc.match) || !in(sc.mismatch) || !in(sc.gap))
        return fail(ctx, NW_ERR_ARG, "scores must lie in [-40, 40]");
    if (sc.gap > 0) return fail(ctx, NW_ERR_ARG, "gap must be <= 0");
    if (sc.mismatch > sc.match) return fail(ctx, NW_ERR_ARG, "mismatch must be <= match");
    return NW_OK;
}

Profile make_profile(const nw_scoring &sc) {
    Profile p;
    for (int c = 0; c < 4; ++c) {
        uint32_t w = 0;
        for (int d = 0; d < 4; ++d) {
            int v = (c == d ? sc.match : sc.mismatch) - 2 * sc.gap;  // s' in the W domain
            w |= (uint32_t)(uint8_t)(int8_t)v << (8 * d);
        }
        p.prof[c] = w;
    }
    p.gap = sc.gap;
    return p;
}

static cudaEvent_t get_event(nw_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

LaunchTimer::LaunchTimer(nw_ctx *c, const char *n, uint32_t kernels) : ctx(c), name(n), count(kernels) {
    if (ctx->profiling && !ctx->capturing) {
        e0 = get_event(ctx);
        e1 = get_event(ctx);
        cudaEventRecord(e0, ctx->stream);
    }
}

LaunchTimer::~LaunchTimer() {
    if (ctx->profiling && e0 && e1) {
        cudaEventRecord(e1, ctx->stream);
        ctx->stats[name].pending.emplace_back(e0, e1);
        ctx->stats[name].pending_count.push_back(count);
    }
}

static double wall_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

HostTimer::HostTimer(nw_ctx *c, const char *n) : ctx(c), name(n), t0(c->profiling ? wall_ms() : 0.0) {}

void HostTimer::stop() {
    if (done) return;
    done = true;
    if (!ctx->profiling) return;
    KernelStat &st = ctx->stats[std::string("host:") + name];
    st.ms += wall_ms() - t0;
    st.launches += 1;
}

// ------------------------------------------------------- tuning and graphs
bool tuned(nw_ctx *ctx, const std::string &key, uint32_t *choice) {
    const auto it = ctx->tuning.find(key);
    if (it == ctx->tuning.end()) return false;
    *choice = it->second;
    return true;
}

void set_tuned(nw_ctx *ctx, const std::string &key, uint32_t choice) { ctx->tuning[key] = choice; }

std::string size_bucket(uint64_t v) {
    int k = 0;
    while ((1ull << (k + 1)) <= v && k < 62) ++k;
    return std::to_string(k);
}

uint64_t hash_bytes(const void *p, size_t n, uint64_t h) {
    // FNV-1a, 64-bit
    const uint8_t *b = (const uint8_t *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

void free_prefix(nw_ctx *ctx, const std::string &prefix) {
    for (auto it = ctx->bufs.begin(); it != ctx->bufs.end();) {
        if (it->first.compare(0, prefix.size(), prefix) == 0) {
            if (it->second.p) cudaFreeAsync(it->second.p, ctx->stream);
            ctx->used -= it->second.cap;
            it = ctx->bufs.erase(it);
        } else {
            ++it;
        }
    }
}

int graph_launch(nw_ctx *ctx, const std::string &key, const char *label, uint32_t kernels, bool *replayed) {
    *replayed = false;
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) return NW_OK;
    cudaError_t e;
    {
        // timed under the dominant kernel's name (one launch of it), as
        // recorded when the graph was captured; the graph's other kernels
        // are counted, untimed, under their own entry
        LaunchTimer t(ctx, it->second.label, 1);
        e = cudaGraphLaunch(it->second.exec, ctx->stream);
    }
    (void)label;
    (void)kernels;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
    if (ctx->profiling && it->second.kernels > 1)
        ctx->stats["graph_other_kernels"].launches += it->second.kernels - 1;
    it->second.last_use = ++ctx->graph_seq;
    ++ctx->graph_replays;
    *replayed = true;
    return NW_OK;
}

int graph_store(nw_ctx *ctx, const std::string &key, const std::string &prefix, const char *label,
                uint32_t kernels, cudaGraph_t g) {
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    while (ctx->graphs.size() >= kMaxGraphs) {  // evict the least recently used
        auto old = ctx->graphs.begin();
        for (auto it = ctx->graphs.begin(); it != ctx->graphs.end(); ++it)
            if (it->second.last_use < old->second.last_use) old = it;
        cudaStreamSynchronize(ctx->stream);  // a replay of it may still run
        cudaGraphExecDestroy(old->second.exec);
        free_prefix(ctx, old->second.prefix);
        ctx->graphs.erase(old);
    }
    GraphEntry &ge = ctx->graphs[key];
    ge.exec = exec;
    ge.prefix = prefix;
    ge.label = label;
    ge.kernels = kernels;
    ge.last_use = ++ctx->graph_seq;
    ++ctx->graph_captures;
    return NW_OK;
}

int pinned_host(nw_ctx *ctx, size_t bytes, void **out) {
    if (bytes > ctx->pinned_cap) {
        if (ctx->pinned) cudaFreeHost(ctx->pinned);
        ctx->pinned = nullptr;
        ctx->pinned_cap = 0;
        const size_t cap = std::max<size_t>(bytes + bytes / 4, 1u << 20);
        const cudaError_t e = cudaHostAlloc(&ctx->pinned, cap, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            ctx->pinned = nullptr;
            return cuda_fail(ctx, e, "pinned staging");
        }
        ctx->pinned_cap = cap;
    }
    *out = ctx->pinned;
    return NW_OK;
}

int to_device(nw_ctx *ctx, const void *host, size_t bytes, const char *slot, void **dev) {
    int rc = scratch(ctx, slot, bytes, dev);
    if (rc) return rc;
    if (bytes) {
        cudaError_t e = cudaMemcpyAsync(*dev, host, bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync H2D");
    }
    return NW_OK;
}

// ------------------------------------------------------------------ packing
// a1: ASCII -> 2-bit.  One thread packs 4 bases into one byte; the 4-byte
// group is read as one aligned word when possible.
__global__ void k_pack(const char *__restrict__ ascii, uint64_t len, uint8_t *__restrict__ out, uint32_t *err) {
    uint64_t nbytes = (len + 3) >> 2;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nbytes;
         q += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t byte = 0;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint64_t pos = q * 4 + k;
            if (pos < len) {
                uint32_t ch = (uint8_t)ascii[pos] & 0xDFu;  // upper-case letters
                uint32_t code = ch == 'A' ? 0u : ch == 'C' ? 1u : ch == 'G' ? 2u : ch == 'T' ? 3u : 4u;
                bad |= code > 3u;
                byte |= (code & 3u) << (2 * k);
            }
        }
        if (bad) raise_error(err, NW_ERR_BAD_BASE, (uint32_t)q);
        out[q] = (uint8_t)byte;
    }
}

// the certificate of the banded rounds (defined with them)
bool band_exit_bound(int64_t m, int64_t n, int64_t w, int32_t match, int32_t gap, int64_t *bound);
bool band_certifies(int64_t m, int64_t n, int64_t w, int32_t sb, const nw_scoring &sc, bool want);
uint32_t band_next_width(uint32_t m, uint32_t n, uint32_t w, int32_t sb, const nw_scoring &sc, bool want);

}  // namespace nw

using namespace nw;

extern "C" {

const char *nw_strerror(int status) {
    switch (status) {
        case NW_OK: return "ok";
        case NW_ERR_ARG: return "invalid argument";
        case NW_ERR_BAD_BASE: return "character outside ACGT";
        case NW_ERR_OOM: return "scratch memory budget exceeded";
        case NW_ERR_CIGAR_TRUNC: return "CIGAR buffer too small";
        case NW_ERR_TIMEOUT: return "device-side wait timed out";
        case NW_ERR_CUDA: return "CUDA runtime error";
        case NW_ERR_UNSUPPORTED: return "unsupported request";
        case NW_ERR_BOUNDS: return "index out of range (checked build)";
        default: return "unknown status";
    }
}

nw_ctx *nw_ctx_create(int device, void *stream, uint64_t mem_budget) {
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    nw_ctx *ctx = new nw_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return nullptr;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->cc_major = prop.major;
    ctx->cc_minor = prop.minor;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    ctx->budget = mem_budget ? mem_budget : (uint64_t)(free_b * 0.9);
    if (cudaMalloc(&ctx->d_err, 2 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, 2 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return nullptr;
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&ctx->mempool, &props) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(ctx->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
        cudaGetLastError();
        ctx->mempool = nullptr;  // the device's default pool then
    }
    return ctx;
}

void nw_ctx_destroy(nw_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->bufs)
        if (kv.second.p) cudaFreeAsync(kv.second.p, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->stats)
        for (auto &pr : kv.second.pending) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    free_band_model(ctx);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->mempool) cudaMemPoolDestroy(ctx->mempool);
    delete ctx;
}

int nw_ctx_set_stream(nw_ctx *ctx, void *stream) {
    if (!ctx) return NW_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return NW_OK;
}

int nw_ctx_sync(nw_ctx *ctx) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    uint32_t h[2] = {0, 0};
    e = cudaMemcpy(h, ctx->d_err, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the device error word");
    if (h[0] != 0) {
        cudaMemset(ctx->d_err, 0, sizeof h);
        return fail(ctx, (int)h[0], "device reported %s (detail %u)", nw_strerror((int)h[0]), h[1]);
    }
    return NW_OK;
}

const char *nw_ctx_last_message(const nw_ctx *ctx) { return ctx ? ctx->msg.c_str() : ""; }

int nw_ctx_set_profiling(nw_ctx *ctx, int on) {
    if (!ctx) return NW_ERR_ARG;
    ctx->profiling = on != 0;
    return NW_OK;
}

int nw_ctx_kernel_stats(nw_ctx *ctx, const char **names, uint64_t *launches, double *total_ms, int cap) {
    if (!ctx) return -NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    int k = 0;
    for (auto &kv : ctx->stats) {
        KernelStat &st = kv.second;
        for (size_t q = 0; q < st.pending.size(); ++q) {
            const auto &pr = st.pending[q];
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) st.ms += ms;
            st.launches += q < st.pending_count.size() ? st.pending_count[q] : 1;
            ctx->event_pool.push_back(pr.first);
            ctx->event_pool.push_back(pr.second);
        }
        st.pending.clear();
        st.pending_count.clear();
        if (k < cap) {
            if (names) names[k] = kv.first.c_str();
            if (launches) launches[k] = st.launches;
            if (total_ms) total_ms[k] = st.ms;
        }
        ++k;
    }
    cudaGetLastError();
    return k;
}

int nw_ctx_reset_stats(nw_ctx *ctx) {
    if (!ctx) return NW_ERR_ARG;
    nw_ctx_kernel_stats(ctx, nullptr, nullptr, nullptr, 0);
    for (auto &kv : ctx->stats) {
        kv.second.launches = 0;
        kv.second.ms = 0.0;
    }
    return NW_OK;
}

int nw_ctx_set_test_hook(nw_ctx *ctx, uint32_t hook) {
    if (!ctx || (hook & ~NW_TEST_DROP_PROGRESS)) return NW_ERR_ARG;
    ctx->test_hook = hook;
    return NW_OK;
}

int nw_ctx_set_autotune(nw_ctx *ctx, int on) {
    if (!ctx) return NW_ERR_ARG;
    ctx->autotune = on != 0;
    return NW_OK;
}

int64_t nw_ctx_tuning(nw_ctx *ctx, char *buf, uint64_t cap) {
    if (!ctx) return -NW_ERR_ARG;
    std::string text;
    for (const auto &kv : ctx->tuning) text += kv.first + " " + std::to_string(kv.second) + "\n";
    if (buf && cap) {
        const uint64_t k = std::min<uint64_t>(cap - 1, text.size());
        std::memcpy(buf, text.data(), k);
        buf[k] = 0;
    }
    return (int64_t)text.size();
}

int nw_ctx_set_tuning(nw_ctx *ctx, const char *text) {
    if (!ctx || !text) return NW_ERR_ARG;
    std::map<std::string, uint32_t> add;
    const char *p = text;
    while (*p) {
        const char *e = std::strchr(p, '\n');
        const std::string line(p, e ? (size_t)(e - p) : std::strlen(p));
        p = e ? e + 1 : p + line.size();
        if (line.empty()) continue;
        const size_t sp = line.rfind(' ');
        if (sp == std::string::npos || sp == 0 || sp + 1 >= line.size())
            return fail(ctx, NW_ERR_ARG, "tuning line without 'key value': %s", line.c_str());
        char *end = nullptr;
        const unsigned long v = std::strtoul(line.c_str() + sp + 1, &end, 10);
        if (!end || *end) return fail(ctx, NW_ERR_ARG, "tuning value is not a number: %s", line.c_str());
        add[line.substr(0, sp)] = (uint32_t)v;
    }
    for (const auto &kv : add) ctx->tuning[kv.first] = kv.second;
    return NW_OK;
}

int nw_ctx_graph_stats(nw_ctx *ctx, uint64_t *out, int cap) {
    if (!ctx) return -NW_ERR_ARG;
    const uint64_t v[3] = {(uint64_t)ctx->graphs.size(), ctx->graph_captures, ctx->graph_replays};
    for (int k = 0; k < cap && k < 3; ++k) out[k] = v[k];
    return 3;
}

int nw_pack(const char *ascii, uint64_t len, uint8_t *out2b) {
    if (len && (!ascii || !out2b)) return NW_ERR_ARG;
    uint64_t nbytes = (len + 3) / 4;
    for (uint64_t q = 0; q < nbytes; ++q) {
        uint32_t byte = 0;
        for (int k = 0; k < 4; ++k) {
            uint64_t pos = q * 4 + k;
            if (pos >= len) break;
            uint32_t ch = (uint8_t)ascii[pos] & 0xDFu;
            uint32_t code;
            switch (ch) {
                case 'A': code = 0; break;
                case 'C': code = 1; break;
                case 'G': code = 2; break;
                case 'T': code = 3; break;
                default: return NW_ERR_BAD_BASE;
            }
            byte |= code << (2 * k);
        }
        out2b[q] = (uint8_t)byte;
    }
    return NW_OK;
}

int nw_pack_codes(const uint8_t *codes, uint64_t len, uint8_t *out2b) {
    if (len && (!codes || !out2b)) return NW_ERR_ARG;
    const uint64_t nbytes = (len + 3) / 4;
    for (uint64_t q = 0; q < nbytes; ++q) {
        uint32_t byte = 0;
        for (int k = 0; k < 4 && q * 4 + k < len; ++k) {
            const uint32_t code = codes[q * 4 + k];
            if (code > 3u) return NW_ERR_BAD_BASE;
            byte |= code << (2 * k);
        }
        out2b[q] = (uint8_t)byte;
    }
    return NW_OK;
}

int nw_pack_pool(const uint8_t *codes, const uint64_t *code_off, const uint32_t *len, uint32_t count, uint8_t *pool,
                 const uint64_t *pool_off) {
    if (count && (!codes || !code_off || !len || !pool || !pool_off)) return NW_ERR_ARG;
    for (uint32_t k = 0; k < count; ++k) {
        const int rc = nw_pack_codes(codes + code_off[k], len[k], pool + pool_off[k]);
        if (rc) return rc;
    }
    return NW_OK;
}

int nw_pack_device(nw_ctx *ctx, const char *ascii, uint64_t len, uint8_t *out2b) {
    if (!ctx) return NW_ERR_ARG;
    if (len == 0) return NW_OK;
    if (!ascii || !out2b) return fail(ctx, NW_ERR_ARG, "null pointer");
    cudaSetDevice(ctx->device);
    uint64_t nbytes = (len + 3) / 4;
    int threads = 256;
    uint64_t blocks = (nbytes + threads - 1) / threads;
    uint64_t cap = (uint64_t)ctx->sm_count * 8;
    if (blocks > cap) blocks = cap;
    {
        LaunchTimer t(ctx, "pack");
        k_pack<<<(unsigned)blocks, threads, 0, ctx->stream>>>(ascii, len, out2b, ctx->d_err);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "k_pack launch");
}

uint64_t nw_cigar_bound(uint64_t m, uint64_t n) { return 2 * (m + n) + 1; }

int nw_band_certifies(uint64_t m, uint64_t n, uint64_t w, int32_t banded_score, nw_scoring sc, uint32_t want_cigar) {
    if (m >= (1ull << 31) || n >= (1ull << 31) || w >= (1ull << 31) || sc.gap > 0 || sc.match < 0) return -NW_ERR_ARG;
    return nw::band_certifies((int64_t)m, (int64_t)n, (int64_t)w, banded_score, sc, want_cigar != 0) ? 1 : 0;
}

int64_t nw_band_next_width(uint64_t m, uint64_t n, uint64_t w, int32_t banded_score, nw_scoring sc,
                           uint32_t want_cigar) {
    if (m >= (1ull << 31) || n >= (1ull << 31) || w >= (1ull << 30) || sc.gap > 0 || sc.match < 0) return -NW_ERR_ARG;
    return nw::band_next_width((uint32_t)m, (uint32_t)n, (uint32_t)w, banded_score, sc, want_cigar != 0);
}

int nw_band_exit_bound(uint64_t m, uint64_t n, uint64_t w, nw_scoring sc, int64_t *bound) {
    if (!bound || m >= (1ull << 31) || n >= (1ull << 31) || w >= (1ull << 31) || sc.gap > 0 || sc.match < 0) return -NW_ERR_ARG;
    return nw::band_exit_bound((int64_t)m, (int64_t)n, (int64_t)w, sc.match, sc.gap, bound) ? 1 : 0;
}

int nw_align(nw_ctx *ctx, const uint8_t *a2b, uint64_t m, const uint8_t *b2b, uint64_t n, nw_scoring sc,
             uint32_t flags, int32_t *score, char *cigar, uint64_t cigar_cap, uint64_t *cigar_len) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    int rc = check_scoring(ctx, sc);
    if (rc) return rc;
    if (m >= (1ull << 30) || n >= (1ull << 30)) return fail(ctx, NW_ERR_ARG, "sequence longer than 2^30");
    uint64_t mn = m < n ? m : n;
    const uint64_t sp = sc.match > 2 * sc.gap ? (uint64_t)(sc.match - 2 * sc.gap) : 0;  // W <= sp * min(i, j)
    if (sp * mn >= (1ull << 29))
        return fail(ctx, NW_ERR_ARG, "(match - 2*gap) * min(m,n) must stay below 2^29");
    if (!score) return fail(ctx, NW_ERR_ARG, "score pointer is null");
    if ((m && !a2b) || (n && !b2b)) return fail(ctx, NW_ERR_ARG, "sequence pointer is null");
    const bool want_cigar = flags & NW_CIGAR;
    if (want_cigar && (!cigar || !cigar_len)) return fail(ctx, NW_ERR_ARG, "CIGAR buffers are null");
    const uint64_t bound = nw_cigar_bound(m, n);
    if (!(flags & NW_HOST_IO)) {
        if (want_cigar && cigar_cap < bound)
            return fail(ctx, NW_ERR_ARG, "device CIGAR capacity %llu below the bound %llu",
                        (unsigned long long)cigar_cap, (unsigned long long)bound);
        return align_single(ctx, a2b, m, b2b, n, sc, flags, score, cigar, cigar_cap, cigar_len);
    }
    // Host I/O: stage inputs, run on device buffers, copy results back, wait.
    void *da = nullptr, *db = nullptr, *dout = nullptr;
    if ((rc = to_device(ctx, a2b, (m + 3) / 4, "hio_a", &da))) return rc;
    if ((rc = to_device(ctx, b2b, (n + 3) / 4, "hio_b", &db))) return rc;
    size_t out_bytes = 16 + (want_cigar ? bound : 0);
    if ((rc = scratch(ctx, "hio_out", out_bytes, &dout))) return rc;
    int32_t *d_score = (int32_t *)dout;
    uint64_t *d_len = (uint64_t *)((char *)dout + 8);
    char *d_cigar = (char *)dout + 16;
    rc = align_single(ctx, (const uint8_t *)da, m, (const uint8_t *)db, n, sc, flags & ~NW_HOST_IO, d_score,
                      want_cigar ? d_cigar : nullptr, bound, want_cigar ? d_len : nullptr);
    if (rc) return rc;
    uint64_t head[2];
    cudaError_t e = cudaMemcpyAsync(head, dout, 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "score D2H");
    if ((rc = nw_ctx_sync(ctx))) return rc;
    *score = (int32_t)(head[0] & 0xffffffffu);
    if (want_cigar) {
        uint64_t len = head[1];
        *cigar_len = len;
        if (len + 1 > cigar_cap) return fail(ctx, NW_ERR_CIGAR_TRUNC, "CIGAR needs %llu bytes", (unsigned long long)(len + 1));
        e = cudaMemcpyAsync(cigar, d_cigar, len + 1, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "CIGAR D2H");
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    }
    return NW_OK;
}

}  // extern "C"
