// Batched pairs (a7): many independent alignments in one persistent launch.
//
// One warp owns one pair at a time and runs all of its stripes (32*R rows
// each) back to back: lane k at step t works on global index g = t - k,
// stripe g / P, column g % P (P = max(n, 96)), so a lane moves straight from
// the last column of one stripe to the first column of the next and the
// warp only idles for 31 steps per pair.  Lane 31 writes the bottom row of a
// stripe into the warp's row buffer in global memory (L2-resident); lane 0
// reads it back for the next stripe, 32 columns at a time, double buffered
// (the row was written at least P-63 steps earlier by the same warp).  Warps
// take pairs from an atomic queue sorted by descending cell count (longest
// processing time first), which balances uneven lengths.
//
// The cell update is the one of nw_single.cu (W domain, prmt + DPX add-max
// + max; with pointers: prmt + add + two max, the pointer bits taken from
// differences).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "nw_internal.cuh"

namespace nw {

constexpr int kBatchWarps = 8;   // warps per CTA
constexpr uint32_t kMinPeriod = 96;

struct BatchTask {
    uint64_t a_off, b_off;  // byte offsets in the pool
    uint32_t m, n;          // rows (A) and columns (B)
    uint32_t out0, out1;    // score destinations (out1 == ~0u: none)
    uint64_t ptr_off;       // word offset of the pair's pointer words
    uint32_t ncg;           // pointer words per lane row
    uint32_t pad;
};

struct BatchArgs {
    const uint8_t *pool;
    const BatchTask *tasks;
    uint32_t ntasks;
    uint32_t *counter;
    uint32_t prof[4];
    int32_t gap;
    uint32_t *ring;
    uint32_t ring_stride;
    int32_t *scores;
    uint32_t *ptr;
    uint32_t *err;
};

// Base codes of rows [i0, i0+R) of a packed sequence of length m (R = 4, 8
// or 16, i0 a multiple of 4), two bits per row; rows >= m read as 0.
template <int R>
__device__ __forceinline__ uint32_t load_rows(const uint8_t *s, uint32_t i0, uint32_t m) {
    uint32_t w = 0;
    if (i0 < m) {
        const uint32_t nbytes = (m + 3) / 4;
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const uint32_t byte = i0 / 4 + q;
            if (byte < nbytes) w |= (uint32_t)__ldg(s + byte) << (8 * q);
        }
    }
    return w;
}

template <int R, bool PTR>
__global__ void __launch_bounds__(kBatchWarps * 32) k_batch(BatchArgs p) {
    constexpr uint32_t SH = 32u * R;
    constexpr uint32_t CPW = PTR ? 16u / R : 1u;
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t *ring = p.ring + (size_t)gw * p.ring_stride;
    const uint32_t P0 = p.prof[0], P1 = p.prof[1], P2 = p.prof[2], P3 = p.prof[3];

    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(p.counter, 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= p.ntasks) break;
        const BatchTask tk = p.tasks[idx];
        const uint8_t *A = p.pool + tk.a_off;
        const uint8_t *B = p.pool + tk.b_off;
        const uint32_t m = tk.m, n = tk.n;
        if (m == 0 || n == 0) {
            if (lane == 0) {
                const int32_t sc = p.gap * (int32_t)(m + n);
                p.scores[tk.out0] = sc;
                if (tk.out1 != ~0u) p.scores[tk.out1] = sc;
            }
            continue;
        }
        const uint32_t S = (m + SH - 1) / SH;
        const uint32_t P = max(n, kMinPeriod);
        const uint32_t T = S * P + 31;
        const uint32_t sM = (m - 1) / SH, lM = ((m - 1) % SH) / R, rM = (m - 1) % R;
        uint32_t *pbase = PTR ? p.ptr + tk.ptr_off : nullptr;

        uint32_t prof[R];
        int32_t Wl[R];
        int32_t dtop = 0;
        uint32_t xout = 0, bits = 0;
        auto init_rows = [&](uint32_t codes) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t c = (codes >> (2 * r)) & 3u;
                prof[r] = c == 0 ? P0 : c == 1 ? P1 : c == 2 ? P2 : P3;
                Wl[r] = 0;
            }
            dtop = 0;
        };
        init_rows(load_rows<R>(A, (uint32_t)lane * R, m));
        uint32_t next_rows = S > 1 ? load_rows<R>(A, SH + (uint32_t)lane * R, m) : 0u;
        int32_t c = -lane;   // column of this lane at step t (negative: not started)
        uint32_t s = 0;      // stripe of this lane

        // Lane-0 input for global index g: stripe 0 reads B (W = 0), later
        // stripes read the row buffer.
        auto chunk_word = [&](uint32_t g) -> uint32_t {
            const uint32_t sg = g / P, cg = g - sg * P;
            if (sg >= S || cg >= n) return 0u;
            return sg == 0 ? base_at(B, cg) : __ldcg(ring + cg);
        };
        uint32_t stage = 0, stage_next = chunk_word((uint32_t)lane);

        for (uint32_t t = 0; t < T; ++t) {
            if ((t & 31u) == 0) {
                stage = stage_next;
                __threadfence_block();
                __syncwarp();
                stage_next = chunk_word(t + 32u + (uint32_t)lane);
            }
            uint32_t x = __shfl_up_sync(kFull, xout, 1);
            const uint32_t x0 = __shfl_sync(kFull, stage, t & 31u);
            if (lane == 0) x = x0;
            if (c >= 0 && c < (int32_t)n && s < S) {
                const int32_t up = (int32_t)(x >> 2);
                const uint32_t sel = sext_selector(x & 3u);
                int32_t d = dtop, u = up;
                uint32_t code = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int32_t sv = (int32_t)prmt(prof[r], 0u, sel);
                    int32_t w;
                    if constexpr (PTR) {
                        // bit0: diagonal is the maximum; bit1: W == up (the
                        // vertical candidate wins over the horizontal one
                        // whenever the diagonal loses) -- from differences,
                        // off the dependency chain
                        const int32_t t1 = d + sv;
                        w = max(t1, max(u, Wl[r]));
                        const uint32_t bits = 3u - (uint32_t)min(w - t1, 1) - (uint32_t)min(2 * (w - u), 2);
                        code |= bits << (2 * r);
                    } else {
                        w = max(__viaddmax_s32(d, sv, Wl[r]), u);
                    }
                    d = Wl[r];
                    Wl[r] = w;
                    u = w;
                }
                dtop = up;
                xout = ((uint32_t)u << 2) | (x & 3u);
                if constexpr (PTR) {
                    const uint32_t cc = (uint32_t)c % CPW;
                    bits |= code << (2u * R * cc);
                    if (cc == CPW - 1 || c == (int32_t)n - 1) {
                        pbase[(size_t)(s * 32u + lane) * tk.ncg + (uint32_t)c / CPW] = bits;
                        bits = 0;
                    }
                }
                if (lane == 31 && s + 1 < S) ring[c] = xout;
                if (s == sM && (uint32_t)lane == lM && c == (int32_t)n - 1) {
                    int32_t wmn = 0;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if ((uint32_t)r == rM) wmn = Wl[r];
                    const int32_t sc = wmn + p.gap * (int32_t)(m + n);
                    p.scores[tk.out0] = sc;
                    if (tk.out1 != ~0u) p.scores[tk.out1] = sc;
                }
            }
            if (++c == (int32_t)P) {
                c = 0;
                ++s;
                if (s < S) {
                    init_rows(next_rows);
                    next_rows = s + 1 < S ? load_rows<R>(A, (s + 1) * SH + (uint32_t)lane * R, m) : 0u;
                }
            }
        }
        __syncwarp();
    }
}

// Diagonal of the all-vs-all matrix: score(a, a) = len * match.
__global__ void k_diag(const uint32_t *len, uint32_t nseq, int32_t match, int32_t *out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nseq; i += gridDim.x * blockDim.x)
        out[(size_t)i * nseq + i] = (int32_t)len[i] * match;
}

// ------------------------------------------------------------------- host
template <int R, bool PTR>
static int launch_batch_R(nw_ctx *ctx, BatchArgs &ba, uint32_t max_n) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<R, PTR>, kBatchWarps * 32, 0);
    if (occ < 1) occ = 1;
    uint32_t blocks = (uint32_t)occ * (uint32_t)ctx->sm_count;
    const uint32_t need = (ba.ntasks + kBatchWarps - 1) / kBatchWarps;
    if (blocks > need) blocks = need ? need : 1;
    const uint32_t warps = blocks * kBatchWarps;
    ba.ring_stride = ((max_n + 31) / 32) * 32 + 32;
    void *v = nullptr;
    int rc = scratch(ctx, "batch_ring", (size_t)warps * ba.ring_stride * 4, &v);
    if (rc) return rc;
    ba.ring = (uint32_t *)v;
    if ((rc = scratch(ctx, "batch_counter", 16, &v))) return rc;
    ba.counter = (uint32_t *)v;
    cudaMemsetAsync(ba.counter, 0, 4, ctx->stream);
    LaunchTimer t(ctx, PTR ? "batch_fill_ptr" : "batch_score");
    k_batch<R, PTR><<<blocks, kBatchWarps * 32, 0, ctx->stream>>>(ba);
    return NW_OK;
}

static int launch_batch(nw_ctx *ctx, int R, bool ptr, BatchArgs &ba, uint32_t max_n) {
    if (ptr) {
        switch (R) {
            case 4: return launch_batch_R<4, true>(ctx, ba, max_n);
            case 8: return launch_batch_R<8, true>(ctx, ba, max_n);
            default: return launch_batch_R<16, true>(ctx, ba, max_n);
        }
    }
    switch (R) {
        case 4: return launch_batch_R<4, false>(ctx, ba, max_n);
        case 8: return launch_batch_R<8, false>(ctx, ba, max_n);
        default: return launch_batch_R<16, false>(ctx, ba, max_n);
    }
}

// Rows per lane for a set of pairs: the one that wastes the fewest padded
// rows per useful row, counting a per-column overhead of ~10 instructions
// against 3 per cell.
static int pick_rows(const std::vector<BatchTask> &tasks) {
    double best = 1e300;
    int bestR = 8;
    for (int R : {4, 8, 16}) {
        double cost = 0;
        const uint32_t SH = 32u * R;
        for (const auto &t : tasks) {
            const double rows = (double)((t.m + SH - 1) / SH) * SH;
            const double P = std::max<uint32_t>(t.n, kMinPeriod);
            cost += rows * P * (3.0 + 10.0 / R);
        }
        if (cost < best) {
            best = cost;
            bestR = R;
        }
    }
    return bestR;
}

template <typename T>
static int upload(nw_ctx *ctx, const char *slot, const std::vector<T> &v, T **dev) {
    void *d = nullptr;
    int rc = scratch(ctx, slot, v.size() * sizeof(T) + 16, &d);
    if (rc) return rc;
    if (!v.empty()) {
        cudaError_t e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "task upload");
        // the host vector may be freed right after: wait for the copy
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "task upload sync");
    }
    *dev = (T *)d;
    return NW_OK;
}

static void sort_lpt(std::vector<BatchTask> &tasks) {
    std::stable_sort(tasks.begin(), tasks.end(), [](const BatchTask &x, const BatchTask &y) {
        return (uint64_t)x.m * std::max(x.n, kMinPeriod) > (uint64_t)y.m * std::max(y.n, kMinPeriod);
    });
}

static int check_common(nw_ctx *ctx, const nw_scoring &sc) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    return check_scoring(ctx, sc);
}

static int check_len(nw_ctx *ctx, const nw_scoring &sc, uint64_t m, uint64_t n) {
    if (m >= (1ull << 30) || n >= (1ull << 30)) return fail(ctx, NW_ERR_ARG, "sequence longer than 2^30");
    const uint64_t mn = m < n ? m : n;
    if ((uint64_t)(sc.match - 2 * sc.gap) * mn >= (1ull << 29))
        return fail(ctx, NW_ERR_ARG, "(match - 2*gap) * min(m,n) must stay below 2^29");
    return NW_OK;
}

}  // namespace nw

using namespace nw;

// Score-only or CIGAR batch on device buffers (the C entry point stages
// host buffers around this).
static int batch_device(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                        const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, const nw_scoring &sc,
                        uint32_t flags, int32_t *scores, char *cigar_pool, const uint64_t *cigar_off,
                        uint64_t *cigar_len) {
    const Profile pf = make_profile(sc);
    const bool want = flags & NW_CIGAR;
    int rc;
    std::vector<BatchTask> tasks(npairs);
    uint32_t max_n = 1;
    for (uint32_t k = 0; k < npairs; ++k) {
        if ((rc = check_len(ctx, sc, a_len[k], b_len[k]))) return rc;
        if (want && cigar_off[k + 1] - cigar_off[k] < nw_cigar_bound(a_len[k], b_len[k]))
            return fail(ctx, NW_ERR_ARG, "CIGAR capacity of pair %u below its bound", k);
        BatchTask t{};
        t.a_off = a_off[k];
        t.b_off = b_off[k];
        t.m = a_len[k];
        t.n = b_len[k];
        // score-only: the optimum is symmetric, so put the sequence whose
        // stripes waste fewer padded rows on the rows
        if (!want && t.m > 0 && t.n > 0) {
            const uint32_t SH = 256;
            const uint32_t wm = (t.m + SH - 1) / SH * SH - t.m, wn = (t.n + SH - 1) / SH * SH - t.n;
            if (wn * (uint64_t)t.m < wm * (uint64_t)t.n && t.m >= kMinPeriod) {
                std::swap(t.a_off, t.b_off);
                std::swap(t.m, t.n);
            }
        }
        t.out0 = k;
        t.out1 = ~0u;
        max_n = std::max(max_n, t.n);
        tasks[k] = t;
    }
    const int R = pick_rows(tasks);
    BatchArgs ba{};
    ba.pool = pool;
    for (int c = 0; c < 4; ++c) ba.prof[c] = pf.prof[c];
    ba.gap = pf.gap;
    ba.scores = scores;
    ba.err = ctx->d_err;
    if (!want) {
        sort_lpt(tasks);
        BatchTask *dt = nullptr;
        if ((rc = upload(ctx, "batch_tasks", tasks, &dt))) return rc;
        ba.tasks = dt;
        ba.ntasks = npairs;
        return launch_batch(ctx, R, false, ba, max_n);
    }
    // CIGAR: waves whose pointer words fit half of the remaining budget.
    // (a wave always takes at least one pair; scratch() reports NW_ERR_OOM if
    // even that does not fit)
    const uint64_t wave_budget = (ctx->budget - std::min(ctx->budget, ctx->used)) / 2;
    std::vector<uint32_t> order(npairs);
    std::iota(order.begin(), order.end(), 0u);
    size_t k0 = 0;
    while (k0 < npairs) {
        std::vector<BatchTask> wave;
        std::vector<uint32_t> ids;
        uint64_t words = 0, mvbytes = 0;
        size_t k = k0;
        for (; k < npairs; ++k) {
            BatchTask t = tasks[order[k]];
            const uint32_t SH = 32u * R;
            t.ncg = ptr_words_per_lane_row(std::max(t.n, 1u), R);
            const uint64_t w = (uint64_t)((t.m + SH - 1) / SH) * 32u * t.ncg;
            if (!wave.empty() && (words + w) * 4 > wave_budget) break;
            t.ptr_off = words;
            words += w;
            mvbytes += (uint64_t)t.m + t.n + 16;
            wave.push_back(t);
            ids.push_back(order[k]);
        }
        void *pv = nullptr, *mv = nullptr, *nm = nullptr;
        if ((rc = scratch(ctx, "batch_ptr", words * 4 + 16, &pv))) return rc;
        if ((rc = scratch(ctx, "batch_moves", mvbytes + 16, &mv))) return rc;
        if ((rc = scratch(ctx, "batch_nmoves", wave.size() * 8 + 16, &nm))) return rc;
        std::vector<TraceTask> tt(wave.size());
        uint64_t mpos = 0;
        for (size_t q = 0; q < wave.size(); ++q) {
            const BatchTask &t = wave[q];
            const uint32_t id = ids[q];
            tt[q] = TraceTask{(const uint32_t *)pv + t.ptr_off, t.ncg, t.m, t.n, (uint8_t *)mv + mpos,
                              (uint64_t *)nm + q, pool + t.a_off, pool + t.b_off, cigar_pool + cigar_off[id],
                              cigar_len + id};
            mpos += (uint64_t)t.m + t.n + 16;
        }
        // order the fill by cell count; ptr_off stays attached to each task
        std::vector<BatchTask> fill = wave;
        sort_lpt(fill);
        BatchTask *dt = nullptr;
        TraceTask *dtt = nullptr;
        if ((rc = upload(ctx, "batch_tasks", fill, &dt))) return rc;
        if ((rc = upload(ctx, "batch_trace_tasks", tt, &dtt))) return rc;
        ba.tasks = dt;
        ba.ntasks = (uint32_t)fill.size();
        ba.ptr = (uint32_t *)pv;
        uint32_t wave_max_n = 1;
        for (const auto &t : wave) wave_max_n = std::max(wave_max_n, t.n);
        if ((rc = launch_batch(ctx, R, true, ba, wave_max_n))) return rc;
        if ((rc = launch_trace(ctx, R, tt[0], dtt, (uint32_t)tt.size(), (flags & NW_CIGAR_M) ? 1u : 0u))) return rc;
        k0 = k;
    }
    return NW_OK;
}

extern "C" int nw_align_batch(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                              const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, nw_scoring sc,
                              uint32_t flags, int32_t *scores, char *cigar_pool, const uint64_t *cigar_off,
                              uint64_t *cigar_len) {
    int rc = check_common(ctx, sc);
    if (rc) return rc;
    if (npairs == 0) return NW_OK;
    if (!a_off || !a_len || !b_off || !b_len || !scores || !pool2b) return fail(ctx, NW_ERR_ARG, "null argument");
    const bool want = flags & NW_CIGAR;
    if (want && (!cigar_pool || !cigar_off || !cigar_len)) return fail(ctx, NW_ERR_ARG, "CIGAR buffers are null");
    if (flags & NW_LEARNED_BAND) return fail(ctx, NW_ERR_UNSUPPORTED, "learned band is not built yet");
    if (!(flags & NW_HOST_IO))
        return batch_device(ctx, pool2b, a_off, a_len, b_off, b_len, npairs, sc, flags, scores, cigar_pool,
                            cigar_off, cigar_len);
    // host buffers: the pool spans up to the furthest sequence end
    uint64_t pool_bytes = 16;
    for (uint32_t k = 0; k < npairs; ++k) {
        pool_bytes = std::max<uint64_t>(pool_bytes, a_off[k] + (a_len[k] + 3) / 4);
        pool_bytes = std::max<uint64_t>(pool_bytes, b_off[k] + (b_len[k] + 3) / 4);
    }
    void *dpool = nullptr, *dsc = nullptr, *dcig = nullptr, *dlen = nullptr;
    if ((rc = to_device(ctx, pool2b, pool_bytes, "hio_pool", &dpool))) return rc;
    if ((rc = scratch(ctx, "hio_scores", (size_t)npairs * 4, &dsc))) return rc;
    if (want) {
        if ((rc = scratch(ctx, "hio_cigar", cigar_off[npairs] + 16, &dcig))) return rc;
        if ((rc = scratch(ctx, "hio_cigar_len", (size_t)npairs * 8, &dlen))) return rc;
    }
    rc = batch_device(ctx, (const uint8_t *)dpool, a_off, a_len, b_off, b_len, npairs, sc, flags & ~NW_HOST_IO,
                      (int32_t *)dsc, (char *)dcig, cigar_off, (uint64_t *)dlen);
    if (rc) return rc;
    cudaMemcpyAsync(scores, dsc, (size_t)npairs * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (want) {
        cudaMemcpyAsync(cigar_len, dlen, (size_t)npairs * 8, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(cigar_pool, dcig, cigar_off[npairs], cudaMemcpyDeviceToHost, ctx->stream);
    }
    return nw_ctx_sync(ctx);
}

extern "C" int nw_score_all_pairs(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *off, const uint32_t *len,
                                  uint32_t nseq, nw_scoring sc, uint32_t flags, int32_t *out) {
    int rc = check_common(ctx, sc);
    if (rc) return rc;
    if (nseq == 0) return NW_OK;
    if (!off || !len || !out || !pool2b) return fail(ctx, NW_ERR_ARG, "null argument");
    if (nseq > 65535) return fail(ctx, NW_ERR_ARG, "at most 65535 sequences");
    for (uint32_t i = 0; i < nseq; ++i)
        if ((rc = check_len(ctx, sc, len[i], len[i]))) return rc;
    const uint8_t *pool = pool2b;
    int32_t *dout = out;
    if (flags & NW_HOST_IO) {
        uint64_t pool_bytes = 16;
        for (uint32_t i = 0; i < nseq; ++i) pool_bytes = std::max<uint64_t>(pool_bytes, off[i] + (len[i] + 3) / 4);
        void *dp = nullptr, *dq = nullptr;
        if ((rc = to_device(ctx, pool2b, pool_bytes, "hio_pool", &dp))) return rc;
        if ((rc = scratch(ctx, "hio_matrix", (size_t)nseq * nseq * 4, &dq))) return rc;
        pool = (const uint8_t *)dp;
        dout = (int32_t *)dq;
    }
    // n(n-1)/2 pairs (Eq. 2), each written to both triangle entries
    std::vector<BatchTask> tasks;
    tasks.reserve((size_t)nseq * (nseq - 1) / 2);
    uint32_t max_n = 1;
    for (uint32_t i = 0; i < nseq; ++i)
        for (uint32_t j = i + 1; j < nseq; ++j) {
            BatchTask t{};
            // rows: the sequence whose 256-row stripes waste fewer padded rows
            const uint32_t SH = 256;
            const uint32_t wi = (len[i] + SH - 1) / SH * SH - len[i], wj = (len[j] + SH - 1) / SH * SH - len[j];
            const bool rows_i = (uint64_t)wi * len[j] <= (uint64_t)wj * len[i] || len[j] < kMinPeriod;
            const uint32_t r = rows_i ? i : j, c = rows_i ? j : i;
            t.a_off = off[r];
            t.m = len[r];
            t.b_off = off[c];
            t.n = len[c];
            t.out0 = i * nseq + j;
            t.out1 = j * nseq + i;
            max_n = std::max(max_n, t.n);
            tasks.push_back(t);
        }
    sort_lpt(tasks);
    const Profile pf = make_profile(sc);
    BatchArgs ba{};
    ba.pool = pool;
    for (int c = 0; c < 4; ++c) ba.prof[c] = pf.prof[c];
    ba.gap = pf.gap;
    ba.scores = dout;
    ba.err = ctx->d_err;
    BatchTask *dt = nullptr;
    if ((rc = upload(ctx, "batch_tasks", tasks, &dt))) return rc;
    ba.tasks = dt;
    ba.ntasks = (uint32_t)tasks.size();
    void *dl = nullptr;
    std::vector<uint32_t> lens(len, len + nseq);
    uint32_t *dlen = nullptr;
    if ((rc = upload(ctx, "allpairs_len", lens, &dlen))) return rc;
    (void)dl;
    if ((rc = launch_batch(ctx, pick_rows(tasks), false, ba, max_n))) return rc;
    {
        LaunchTimer t(ctx, "diag");
        k_diag<<<(nseq + 255) / 256, 256, 0, ctx->stream>>>(dlen, nseq, sc.match, dout);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "all-pairs launch");
    if (flags & NW_HOST_IO) {
        e = cudaMemcpyAsync(out, dout, (size_t)nseq * nseq * 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "matrix D2H");
        return nw_ctx_sync(ctx);
    }
    return NW_OK;
}
