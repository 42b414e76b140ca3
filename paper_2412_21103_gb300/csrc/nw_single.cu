// One pair: score-matrix fill (a3/a4), traceback (a5) and CIGAR assembly.
//
// Fill layout.  The query rows are cut into stripes of 32*R rows; one warp
// owns a stripe and lane k of it owns R consecutive rows, kept in registers.
// The warp is a systolic array over the anti-diagonal wavefront: at step t
// lane k works on column t-k+1, receives the bottom W value of lane k-1 (and
// the column's base code) by one warp shuffle, and updates its R cells with
// the Sec. 2.3 recurrence in the W domain (one prmt + one DPX add-max + one
// max per cell).  Lane 0 of stripe s reads stripe s-1's bottom row from a
// global boundary buffer, 32 columns at a time, double buffered, after an
// acquire on the producer's progress counter; lane 31 writes its bottom row
// there and releases the counter every 32 columns.  Every wait is bounded.
//
// Pointer layout (with the alignment requested).  For every cell the fill
// stores two bits: bit0 = the diagonal candidate is the maximum, bit1 = the
// vertical candidate is not below the horizontal one.  The Sec. 2.4 backtrack
// with priority diagonal > vertical > horizontal reads: bit0 -> diagonal,
// else bit1 -> vertical, else horizontal (the 1/2/3 codes of Sec. 3.1 are
// recovered as 1, 2, 3).  A 32-bit word holds R rows x (16/R) columns of one
// lane; words are stored [stripe][lane][column group], so one lane's words
// are contiguous along the row.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <string>

#include "nw_bits.cuh"

namespace nw {

constexpr int kFillWarps = 4;  // warps per CTA of the fill kernel

struct FillArgs {
    const uint8_t *a;
    const uint8_t *b;
    uint32_t m, n;
    uint32_t prof[4];
    int32_t gap;
    uint32_t S;          // stripes
    uint32_t bstride;    // words per boundary row
    uint32_t *bnd;       // boundary rows: row s holds stripe s's bottom, packed (W << 2) | b_j at [j]
    uint32_t *progress;  // progress[s] = columns of row s published
    uint32_t *ptr;       // pointer words (may be null)
    uint32_t ncg;        // words per lane row of the pointer layout
    int32_t *score;      // H(m,n) out
    uint32_t *err;
};

// Warp-uniform bounded wait on a progress counter.
__device__ __forceinline__ bool warp_wait(const uint32_t *flag, uint32_t target, uint32_t *err, uint32_t where) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = wait_geq(flag, target, err, where) ? 1 : 0;
    ok = __shfl_sync(kFull, ok, 0);
    if (ok) (void)ld_acquire(flag);  // acquire for every lane's following loads
    return ok != 0;
}

// Score-only fill with a global boundary row between consecutive stripes
// (the allocation-free entry point's kernel).
template <int R>
__global__ void __launch_bounds__(kFillWarps * 32) k_fill(FillArgs p) {
    constexpr uint32_t SH = 32u * R;
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t m = p.m, n = p.n;
    const uint32_t sM = (m - 1) / SH, lM = ((m - 1) % SH) / R, rM = (m - 1) % R;

    for (uint32_t s = gw; s < p.S; s += nwarps) {
        const uint32_t row0 = s * SH + lane * R;
        uint32_t prof[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t i = row0 + r;
            const uint32_t c = i < m ? base_at(p.a, i) : 0u;
            prof[r] = c == 0 ? p.prof[0] : c == 1 ? p.prof[1] : c == 2 ? p.prof[2] : p.prof[3];
        }
        int32_t Wl[R];
#pragma unroll
        for (int r = 0; r < R; ++r) Wl[r] = 0;  // column 0: W(i,0) = 0
        int32_t dtop = 0;                        // W(top-1, j-1)
        uint32_t xout = 0;
        const uint32_t *in = s ? p.bnd + (size_t)(s - 1) * p.bstride : nullptr;
        uint32_t *outb = (s + 1 < p.S) ? p.bnd + (size_t)s * p.bstride : nullptr;

        // Lane-0 input chunks: lane l of `stage` holds the word of column c0 + l
        // (row 0 of the grid: W = 0, only the base code).
#define NW_LOAD_CHUNK(C0, DST)                                                              \
    do {                                                                                    \
        const uint32_t c0_ = (C0);                                                          \
        if (c0_ <= n) {                                                                     \
            if (s && !warp_wait(&p.progress[s - 1], min(c0_ + 31u, n), p.err, s)) return;  \
            const uint32_t cl_ = c0_ + lane;                                                \
            if (cl_ <= n) (DST) = s ? __ldcg(in + cl_) : base_at(p.b, cl_ - 1);             \
        }                                                                                   \
    } while (0)
        uint32_t stage = 0, stage_next = 0;
        NW_LOAD_CHUNK(1u, stage_next);

        const uint32_t T = n + 31;
        for (uint32_t t = 0; t < T; ++t) {
            if ((t & 31u) == 0) {
                stage = stage_next;
                NW_LOAD_CHUNK(t + 33u, stage_next);
            }
            uint32_t x = __shfl_up_sync(kFull, xout, 1);
            uint32_t x0 = __shfl_sync(kFull, stage, t & 31u);
            if (lane == 0) x = x0;
            const int32_t c = (int32_t)t - lane;  // 0-based column of this lane
            if (c >= 0 && c < (int32_t)n) {
                const int32_t up = (int32_t)(x >> 2);
                const uint32_t sel = sext_selector(x & 3u);
                int32_t d = dtop, u = up;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int32_t sv = (int32_t)prmt(prof[r], 0u, sel);
                    const int32_t w = max(__viaddmax_s32(d, sv, Wl[r]), u);
                    d = Wl[r];
                    Wl[r] = w;
                    u = w;
                }
                dtop = up;
                xout = ((uint32_t)u << 2) | (x & 3u);
                if (lane == 31 && outb) {
                    outb[c + 1] = xout;
                    if (((c + 1) & 31) == 0 || c + 1 == (int32_t)n) st_release(&p.progress[s], (uint32_t)c + 1);
                }
                if (s == sM && (uint32_t)lane == lM && c == (int32_t)n - 1) {
                    int32_t wmn = 0;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if ((uint32_t)r == rM) wmn = Wl[r];
                    *p.score = wmn + p.gap * (int32_t)(m + n);
                }
            }
        }
#undef NW_LOAD_CHUNK
    }
}

// Zero-length side: score gap*(m+n); CIGAR "<m>I" or "<n>D" or "".
__global__ void k_trivial(uint32_t m, uint32_t n, int32_t gap, int32_t *score, char *cigar, uint64_t *cigar_len) {
    *score = gap * (int32_t)(m + n);
    if (!cigar) return;
    uint32_t L = m + n;
    if (L == 0) {
        cigar[0] = 0;
        *cigar_len = 0;
        return;
    }
    char tmp[12];
    int k = 0;
    while (L) {
        tmp[k++] = '0' + L % 10;
        L /= 10;
    }
    for (int q = 0; q < k; ++q) cigar[q] = tmp[k - 1 - q];
    cigar[k] = m ? 'I' : 'D';
    cigar[k + 1] = 0;
    *cigar_len = k + 1;
}

// ----------------------------------------------------------------- dispatch
// Rows per lane and warps per CTA for the single-pair fill (tunable at run
// time through NW_PAIR_R / NW_PAIR_WARPS for sweeps).
static void pair_shape(nw_ctx *ctx, uint64_t m, int &R, int &C, int &nw) {
    (void)ctx;
    // measured on GB300 (32k x 32k): 8 x 2 blocks lead for long pairs,
    // 4 x 2 for short ones (fewer idle lanes in the last stripe)
    R = m >= 2048 ? 8 : 4;
    C = 2;
    nw = 4;
    // a short pair fits one CTA: no row group boundary at all
    const uint64_t S = (m + 32u * R - 1) / (32u * R);
    if (S <= 8) nw = (int)S;
    if (const char *e = getenv("NW_PAIR_R")) R = atoi(e);
    if (const char *e = getenv("NW_PAIR_C")) C = atoi(e);
    if (const char *e = getenv("NW_PAIR_WARPS")) nw = atoi(e);
}

__global__ void k_walk_init(uint32_t *state, uint32_t m, uint32_t n) {
    state[0] = m;
    state[1] = n;
    state[2] = 0;
    state[3] = 0;
    state[4] = 0;
}

static uint64_t headroom(nw_ctx *ctx, const char *slot) { return scratch_headroom(ctx, slot); }

// Stripe-checkpoint recompute (a6), for pairs whose pointer matrix exceeds
// the memory budget.  A score-only fill keeps the bottom W row of every
// group of nw stripes (one CTA's rows); then, from the bottom up, waves of
// groups are filled again with pointers -- each group starts from its own
// kept row, so the groups of a wave run side by side -- and the traceback
// walks through the wave and pauses at its top.  Each wave computes only the
// columns left of the walk's current cell (read on the device: no host round
// trip).  Memory: (groups-1) rows of 4(n+128) bytes plus one wave of
// pointers; work: at most twice the fill.  Decisions depend only on the
// pointers, which the second pass reproduces exactly, so the alignment is
// the one the full pointer matrix gives.
static int run_pair_recompute(nw_ctx *ctx, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n,
                              const Profile &pf, uint32_t flags, int R, int C, int nw, int32_t *score, char *cigar,
                              uint64_t *cigar_len, uint8_t *moves, uint64_t *nmoves) {
    const uint32_t SH = 32u * R;
    const uint32_t S = (m + SH - 1) / SH;
    const uint32_t CS = (S + nw - 1) / nw;
    const uint32_t ncg = ptr_words_per_lane_row(n, R);
    int rc;
    void *v = nullptr;
    uint32_t *bnd = nullptr;
    if (CS > 1) {
        if ((rc = scratch(ctx, "ckpt_rows", (size_t)(CS - 1) * pair_bstride(n) * 4, &v))) return rc;
        bnd = (uint32_t *)v;
    }
    if ((rc = scratch(ctx, "ckpt_progress", (size_t)CS * 4 + 16, &v))) return rc;
    uint32_t *progress = (uint32_t *)v;
    if ((rc = scratch(ctx, "ckpt_walk", 64, &v))) return rc;
    uint32_t *state = (uint32_t *)v;
    PairFill f;
    f.R = R;
    f.C = C;
    f.nw = nw;
    f.score = score;
    f.bnd = bnd;
    f.progress = progress;
    f.keep_rows = true;
    if ((rc = launch_pair_fill(ctx, a2b, m, b2b, n, pf, f))) return rc;  // checkpoints + score
    f.keep_rows = false;
    {
        LaunchTimer t(ctx, "walk_init");
        k_walk_init<<<1, 1, 0, ctx->stream>>>(state, m, n);
    }
    const uint64_t group_bytes = (uint64_t)nw * 32u * ncg * 4u;
    const uint64_t room = headroom(ctx, "ckpt_wave");
    uint64_t G = room / (group_bytes + group_bytes / 8 + 256);
    if (G == 0) return fail(ctx, NW_ERR_OOM, "one group of pointers (%llu bytes) exceeds the budget",
                            (unsigned long long)group_bytes);
    if (G > CS) G = CS;
    if ((rc = scratch(ctx, "ckpt_wave", G * group_bytes, &v))) return rc;
    uint32_t *wave = (uint32_t *)v;
    TraceTask tt{wave, ncg, m, n, moves, nmoves, a2b, b2b, cigar, cigar_len, kNoBand, 0, state};
    for (int64_t g1 = CS; g1 > 0; g1 -= (int64_t)G) {
        const uint32_t g0 = (uint32_t)std::max<int64_t>(0, g1 - (int64_t)G);
        PairFill r = f;
        r.ptr = true;
        r.ptr_words = wave;
        r.ncg = ncg;
        r.score = nullptr;
        r.cs_lo = g0;
        r.cs_hi = (uint32_t)g1;
        r.ncols = state + 1;
        r.recompute = true;
        if ((rc = launch_pair_fill(ctx, a2b, m, b2b, n, pf, r))) return rc;
        tt.s_lo = g0 * (uint32_t)nw;
        if ((rc = launch_traceback(ctx, R, tt, nullptr, 1))) return rc;
    }
    return launch_finish(ctx, tt, nullptr, 1, (flags & NW_CIGAR_M) ? 1u : 0u);
}

// Autotuner for the single-pair block shape: the first pair of a size
// bucket (powers of two of m and n) runs the score-only fill with each
// candidate R x C x warps, timed by CUDA events, and keeps the fastest.  The
// runs compute the real score.  Environment overrides take precedence.
static int tune_pair_shape(nw_ctx *ctx, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n,
                           const Profile &pf, int32_t *score, int &R, int &C, int &nw) {
    if (!ctx->autotune || getenv("NW_PAIR_R") || getenv("NW_PAIR_C") || getenv("NW_PAIR_WARPS")) return NW_OK;
    const std::string key = "pair_shape:m" + size_bucket(m) + ":n" + size_bucket(n);
    uint32_t c = 0;
    if (tuned(ctx, key, &c)) {
        R = (int)(c / 100);
        C = (int)(c / 10 % 10);
        nw = (int)(c % 10);
        const bool shape_ok = (R == 2 && (C == 2 || C == 4 || C == 8)) || (R == 4 && (C == 2 || C == 4)) ||
                              (R == 8 && C == 2);
        if (!shape_ok || nw < 1 || nw > 8) return fail(ctx, NW_ERR_ARG, "tuning %s: shape %u", key.c_str(), c);
        return NW_OK;
    }
    static const int cand[][3] = {{8, 2, 4}, {4, 2, 4}, {4, 4, 4}, {8, 2, 3}, {4, 2, 8}, {2, 2, 4}};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    int rc = NW_OK;
    for (const auto &k : cand) {
        PairFill f;
        f.R = k[0];
        f.C = k[1];
        const uint64_t S = (m + 32u * f.R - 1) / (32u * f.R);
        f.nw = (int)std::min<uint64_t>((uint64_t)k[2], S);
        f.score = score;
        cudaEventRecord(a, ctx->stream);
        if ((rc = launch_pair_fill(ctx, a2b, m, b2b, n, pf, f))) break;
        cudaEventRecord(b, ctx->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
            best = ms;
            R = f.R;
            C = f.C;
            nw = f.nw;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!rc) set_tuned(ctx, key, (uint32_t)(R * 100 + C * 10 + nw));
    return rc;
}

static int run_pair(nw_ctx *ctx, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n, const Profile &pf,
                    uint32_t flags, int32_t *score, char *cigar, uint64_t *cigar_len) {
    const bool want = flags & NW_CIGAR;
    int R, C, nw;
    pair_shape(ctx, m, R, C, nw);
    int rc0 = tune_pair_shape(ctx, a2b, m, b2b, n, pf, score, R, C, nw);
    if (rc0) return rc0;
    PairFill f;
    f.R = R;
    f.C = C;
    f.nw = nw;
    f.score = score;
    if (ctx->test_hook & NW_TEST_DROP_PROGRESS) {
        // failure-path test: every group after the first waits for a kept
        // row whose progress counter nothing releases (zeroed, and recompute
        // passes release none) -- the waits run out and report a timeout
        ctx->test_hook &= ~NW_TEST_DROP_PROGRESS;
        const uint64_t S = (m + 32u * R - 1) / (32u * R), CS = (S + nw - 1) / nw;
        void *v = nullptr, *g = nullptr;
        int rc = scratch(ctx, "hook_rows", (size_t)std::max<uint64_t>(CS, 2) * pair_bstride(n) * 4, &v);
        if (!rc) rc = scratch(ctx, "hook_progress", (size_t)CS * 4 + 16, &g);
        if (rc) return rc;
        cudaMemsetAsync(g, 0, (size_t)CS * 4 + 16, ctx->stream);
        f.bnd = (uint32_t *)v;
        f.progress = (uint32_t *)g;
        f.recompute = true;
        return launch_pair_fill(ctx, a2b, m, b2b, n, pf, f);
    }
    if (!want) return launch_pair_fill(ctx, a2b, m, b2b, n, pf, f);
    int rc;
    void *mv = nullptr, *nm = nullptr;
    if ((rc = scratch(ctx, "moves", (size_t)m + n + 16, &mv))) return rc;
    if ((rc = scratch(ctx, "nmoves", 16, &nm))) return rc;
    const uint32_t SH = 32u * R;
    const uint32_t S = (m + SH - 1) / SH;
    const uint32_t ncg = ptr_words_per_lane_row(n, R);
    const uint64_t ptr_bytes = (uint64_t)S * 32u * ncg * 4u;
    const uint64_t CS = (S + nw - 1) / nw;
    const uint64_t rows_bytes = (CS > 1 ? (CS - 1) * pair_bstride(n) * 4 : 0) + 4 * pair_bstride(n) + CS * 4 + 1024;
    // the full pointer matrix, unless it (with the fill's rows) exceeds the budget
    if ((flags & NW_RECOMPUTE) || ptr_bytes + ptr_bytes / 8 + rows_bytes > headroom(ctx, "ptr"))
        // (groups of at most 4 stripes: the recompute's unit of memory)
        return run_pair_recompute(ctx, a2b, m, b2b, n, pf, flags, R, C, std::min(nw, 4), score, cigar, cigar_len,
                                  (uint8_t *)mv,
                                  (uint64_t *)nm);
    void *v = nullptr;
    if ((rc = scratch(ctx, "ptr", ptr_bytes, &v))) return rc;
    f.ptr = true;
    f.ptr_words = (uint32_t *)v;
    f.ncg = ncg;
    if ((rc = launch_pair_fill(ctx, a2b, m, b2b, n, pf, f))) return rc;
    TraceTask tt{f.ptr_words, ncg, m, n, (uint8_t *)mv, (uint64_t *)nm, a2b, b2b, cigar, cigar_len, kNoBand, 0,
                 nullptr};
    return launch_trace(ctx, R, &tt, nullptr, 1, (flags & NW_CIGAR_M) ? 1u : 0u);
}

// Score-only fill with 16 rows per lane on `stream`, using scratch the
// caller provides (no context, no allocation): `bnd` holds
// (S-1) * bstride words and `progress` S words that must be zero, where
// S = ceil(m / 512) and bstride = 32 * ceil((n + 1) / 32).  m, n >= 1.
cudaError_t fill_score_with_scratch(const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n,
                                    const nw_scoring &sc, int32_t *score, uint32_t *bnd, uint32_t *progress,
                                    uint32_t *err, cudaStream_t stream, int sm_count) {
    constexpr int R = 16;
    const Profile pf = make_profile(sc);
    FillArgs fa{};
    fa.a = a2b;
    fa.b = b2b;
    fa.m = m;
    fa.n = n;
    for (int c = 0; c < 4; ++c) fa.prof[c] = pf.prof[c];
    fa.gap = pf.gap;
    fa.S = (m + 32u * R - 1) / (32u * R);
    fa.bstride = ((n + 1 + 31) / 32) * 32;
    fa.bnd = bnd;
    fa.progress = progress;
    fa.score = score;
    fa.err = err;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fill<R>, kFillWarps * 32, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    uint32_t blocks = (fa.S + kFillWarps - 1) / kFillWarps;
    const uint32_t cap = (uint32_t)occ * (uint32_t)sm_count;  // all CTAs co-resident
    if (blocks > cap) blocks = cap;
    k_fill<R><<<blocks, kFillWarps * 32, 0, stream>>>(fa);
    return cudaGetLastError();
}

int align_single(nw_ctx *ctx, const uint8_t *a2b, uint64_t m, const uint8_t *b2b, uint64_t n, const nw_scoring &sc,
                 uint32_t flags, int32_t *score, char *cigar, uint64_t cigar_cap, uint64_t *cigar_len) {
    (void)cigar_cap;
    const Profile pf = make_profile(sc);
    const bool want = flags & NW_CIGAR;
    if (m == 0 || n == 0) {
        LaunchTimer t(ctx, "trivial");
        k_trivial<<<1, 1, 0, ctx->stream>>>((uint32_t)m, (uint32_t)n, sc.gap, score, want ? cigar : nullptr,
                                            want ? cigar_len : nullptr);
    } else if (!(ctx->test_hook & NW_TEST_DROP_PROGRESS) && !(flags & NW_RECOMPUTE) &&
               bits_pair_takes(ctx, (uint32_t)m, (uint32_t)n, sc, want)) {
        // the paper's scoring (any with 0 <= s'x <= s'm <= 3): bit-sliced stripes
        const int rc = bits_pair(ctx, a2b, (uint32_t)m, b2b, (uint32_t)n, sc, want, (flags & NW_CIGAR_M) ? 1u : 0u,
                                 score, cigar, cigar_len);
        if (rc) return rc;
    } else {
        const int rc = run_pair(ctx, a2b, (uint32_t)m, b2b, (uint32_t)n, pf, flags, score, cigar, cigar_len);
        if (rc) return rc;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "single-pair launch");
}

}  // namespace nw
