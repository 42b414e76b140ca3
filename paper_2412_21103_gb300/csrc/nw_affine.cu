// Affine gaps (Gotoh; not in the paper, whose gap penalty is linear -- the
// center-star method it cites uses affine gaps): a run of k gap moves of one
// kind scores go + k*ge.  Three grids: E (ends in a horizontal move), F
// (ends in a vertical move), H (best):
//     E(i,j) = max(E(i,j-1) + ge, H(i,j-1) + go + ge)
//     F(i,j) = max(F(i-1,j) + ge, H(i-1,j) + go + ge)
//     H(i,j) = max(H(i-1,j-1) + s(A_i,B_j), E(i,j), F(i,j))
// from H(0,0) = 0, H(0,j) = E(0,j) = go + j*ge, H(i,0) = F(i,0) = go + i*ge.
//
// Shifted domain: W = H - ge*(i+j), E' = E - ge*(i+j), F' = F - ge*(i+j).
// Every move adds one to i+j, so the extension cost drops out:
//     E'(i,j) = max(E'(i,j-1), W(i,j-1) + go)
//     F'(i,j) = max(F'(i-1,j), W(i-1,j) + go)
//     W(i,j)  = max(W(i-1,j-1) + s - 2*ge, E'(i,j), F'(i,j))
// with W(0,0) = 0, W(0,j) = W(i,0) = go, F'(0,j) = E'(i,0) = -inf and
// H(m,n) = W(m,n) + ge*(m+n).  A cell is one byte permute (s - 2ge), three
// DPX add-max (E', F', W) and one max.  The walk needs four bits per cell:
// L (the diagonal candidate is below max(E', F')) and H (E' above F') in
// the global kernels' pointer words, and in a second word array at the same
// index the extension bits of the cell's gap states -- F: F'(i-1,j) >
// W(i-1,j) + go, E: E'(i,j-1) > W(i,j-1) + go (a tie closes the gap).
//
// Batched by stripe jobs: every 32R-row stripe of every pair is one job,
// jobs queued pair by pair (longest pairs first) and stripes in order, so a
// long pair's stripes run on many warps at once as a wavefront instead of
// one after another on one warp (which left a batch waiting on its longest
// pair).  A warp takes the next job from an atomic counter; lane k owns R
// rows of the stripe and a step hands the lane below two values (W with the
// base code, and F').  Lane 31 writes the stripe's bottom row (W and F')
// to the job's row buffer and publishes every 32 columns with a release
// store to the job's progress word; the warp of the next stripe waits (a
// bounded spin) on that word before it reads each chunk of 32 columns.
// The job it waits on was taken earlier by a warp of the same persistent,
// fully resident grid, so every wait ends.
#include <algorithm>
#include <vector>

#include "nw_internal.cuh"

namespace nw {
namespace {

constexpr int kAffWarps = 8;
constexpr uint32_t kAffMinPeriod = 96;
constexpr int32_t kAffNeg = -(1 << 27);   // -inf: far below any W, no add wraps

struct AffTask {
    uint64_t a_off, b_off;
    uint32_t m, n;
    uint32_t out;
    uint32_t ncg;        // pointer words per lane row
    uint64_t ptr_off;    // word offset (the extension words follow at + ext_off)
    uint64_t row_off;    // word offset of the pair's stripe rows: stripe s (< S-1) at row_off + 2*s*nr
    uint32_t nr;         // words per row half (n rounded up to 32)
    uint32_t pad;
};

struct AffJob {
    uint32_t task;       // index into the launch's tasks
    uint32_t stripe;
};

struct AffArgs {
    const uint8_t *pool;
    const AffTask *tasks;
    const AffJob *jobs;
    uint32_t njobs;
    uint32_t *counter;
    uint32_t prof[4];    // byte d of prof[c] = s(c, d) - 2*ge as int8
    int32_t go, ge;
    uint32_t *rows;      // stripe rows of every pair (W words, then F' words)
    uint64_t rows_cap;
    uint32_t *progress;  // per job: columns of its bottom row published
    int32_t *scores;
    uint32_t *ptr;
    uint64_t ext_off;    // words from a pointer word to its extension word
    uint32_t *err;
    uint32_t out_cap;    // pairs at scores (checked build; the pointer words
                         // of a launch are 2 * ext_off)
};

template <int R>
__device__ __forceinline__ uint32_t aff_rows(const uint8_t *s, uint32_t i0, uint32_t m) {
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

__device__ __forceinline__ void aff_st_if(bool p, uint32_t *dst, uint32_t v) {
    asm volatile("{.reg .pred q; setp.ne.b32 q, %0, 0; @q st.global.u32 [%1], %2;}" ::"r"((uint32_t)p), "l"(dst), "r"(v)
                 : "memory");
}

// Warp-uniform bounded wait until *flag >= target (lane 0 spins; then every
// lane acquires, so its following loads see what the producer published).
__device__ __forceinline__ bool aff_wait(const uint32_t *flag, uint32_t target, uint32_t *err, uint32_t where) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = wait_geq(flag, target, err, where) ? 1 : 0;
    ok = __shfl_sync(kFull, ok, 0);
    if (ok) (void)ld_acquire(flag);
    return ok != 0;
}

template <int R, bool PTR>
__global__ void __launch_bounds__(kAffWarps * 32) k_affine(AffArgs p) {
    constexpr uint32_t SH = 32u * R;
    constexpr uint32_t CPW = PTR ? 16u / R : 1u;
    const int lane = threadIdx.x & 31;
    const int32_t go = p.go;
    const uint32_t P0 = p.prof[0], P1 = p.prof[1], P2 = p.prof[2], P3 = p.prof[3];

    for (;;) {
        uint32_t jidx = 0;
        if (lane == 0) jidx = atomicAdd(p.counter, 1u);
        jidx = __shfl_sync(kFull, jidx, 0);
        if (jidx >= p.njobs) break;
        const AffJob jb = p.jobs[jidx];
        const AffTask tk = p.tasks[jb.task];
        const uint32_t s = jb.stripe;
        const uint8_t *A = p.pool + tk.a_off;
        const uint8_t *B = p.pool + tk.b_off;
        const uint32_t m = tk.m, n = tk.n;
        if (m == 0 || n == 0) {   // a single job
            if (lane == 0 && in_range(tk.out, p.out_cap, p.err, kSiteAffScore))
                p.scores[tk.out] = m + n ? go + p.ge * (int32_t)(m + n) : 0;
            continue;
        }
        const uint32_t S = (m + SH - 1) / SH;
        const uint32_t T = n + 31;
        const uint32_t lM = ((m - 1) % SH) / R, rM = (m - 1) % R;
        uint32_t *pbase = PTR ? p.ptr + tk.ptr_off : nullptr;
        // the previous stripe's row (s > 0) and this stripe's (s < S - 1)
        const uint32_t *inW = s ? p.rows + tk.row_off + (size_t)(s - 1) * 2 * tk.nr : nullptr;
        const uint32_t *inF = s ? inW + tk.nr : nullptr;
        uint32_t *outW = s + 1 < S ? p.rows + tk.row_off + (size_t)s * 2 * tk.nr : nullptr;
        uint32_t *outF = s + 1 < S ? outW + tk.nr : nullptr;
        const uint32_t *prev = s ? p.progress + (jidx - 1) : nullptr;   // stripe s-1 is the job before
        uint32_t *mine = p.progress + jidx;

        uint32_t prof[R];
        int32_t Wl[R], El[R];
        uint32_t xout = 0, accL = 0, accH = 0, accF = 0, accE = 0;
        int32_t fout = kAffNeg;
        const uint32_t i0 = s * SH + (uint32_t)lane * R;   // rows i0+1 .. i0+R (1-based)
        {
            const uint32_t codes = aff_rows<R>(A, i0, m);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t c = (codes >> (2 * r)) & 3u;
                prof[r] = c == 0 ? P0 : c == 1 ? P1 : c == 2 ? P2 : P3;
                Wl[r] = go;        // W(i, 0)
                El[r] = kAffNeg;   // E'(i, 0)
            }
        }
        int32_t dtop = i0 == 0 ? 0 : go;   // W(i0, 0)
        int32_t c = -lane;
        // lane 0's inputs for column col: row 0 (W = go, F' = -inf) in stripe
        // 0, the previous stripe's bottom row (published, see the waits) after
        auto chunk_w = [&](uint32_t col) -> uint32_t {
            if (col >= n) return 0u;
            if (!s) return ((uint32_t)go << 2) | base_at(B, col);
            return __ldcg(inW + col);
        };
        auto chunk_f = [&](uint32_t col) -> int32_t {
            if (!s || col >= n) return kAffNeg;
            return (int32_t)__ldcg(inF + col);
        };
        bool alive = !s || aff_wait(prev, min(32u, n), p.err, jidx);
        uint32_t stage = 0, stage_next = alive ? chunk_w((uint32_t)lane) : 0u;
        int32_t fstage = kAffNeg, fstage_next = alive ? chunk_f((uint32_t)lane) : kAffNeg;

        // the R cells of one column; u / fu: W and F' of the row above
        auto column = [&](int32_t d, int32_t u, int32_t fu, uint32_t sel) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int32_t sv = (int32_t)prmt(prof[r], 0u, sel);
                const int32_t e = __viaddmax_s32(Wl[r], go, El[r]);
                const int32_t f = __viaddmax_s32(u, go, fu);
                const int32_t mx = max(e, f);
                const int32_t w = __viaddmax_s32(d, sv, mx);
                if constexpr (PTR) {
                    accL = ptr_append(accL, d + sv - mx);
                    accH = ptr_append(accH, f - e);
                    accF = ptr_append(accF, u + go - fu);
                    accE = ptr_append(accE, Wl[r] + go - El[r]);
                }
                d = Wl[r];
                Wl[r] = w;
                El[r] = e;
                u = w;
                fu = f;
            }
            return make_int2(u, fu);
        };
        // lane 31: this stripe's bottom row out, published every 32 columns
        auto row_out = [&](uint32_t col) {
            if (lane == 31 && outW && in_range((size_t)(outW - p.rows) + tk.nr + col, p.rows_cap, p.err, kSiteAffRing)) {
                outW[col] = xout;
                outF[col] = (uint32_t)fout;
                if (((col + 1) & 31u) == 0 || col + 1 == n) st_release(mine, col + 1);
            }
        };

        for (uint32_t t = 0; t < T && alive; ++t) {
            if ((t & 31u) == 0) {
                stage = stage_next;
                fstage = fstage_next;
                if (s && t + 32 < n && !(alive = aff_wait(prev, min(t + 64u, n), p.err, jidx))) break;
                stage_next = chunk_w(t + 32u + (uint32_t)lane);
                fstage_next = chunk_f(t + 32u + (uint32_t)lane);
                if (__all_sync(kFull, c >= 0 && c + 32 <= (int32_t)n - 1)) {
                    uint32_t cc = (uint32_t)c % CPW;
                    uint32_t *prow = PTR ? pbase + (size_t)(s * 32u + lane) * tk.ncg : nullptr;
#pragma unroll 4
                    for (uint32_t uu = 0; uu < 32u; ++uu) {
                        uint32_t x = __shfl_up_sync(kFull, xout, 1);
                        int32_t fx = __shfl_up_sync(kFull, fout, 1);
                        const uint32_t x0 = __shfl_sync(kFull, stage, uu);
                        const int32_t f0 = __shfl_sync(kFull, fstage, uu);
                        if (lane == 0) {
                            x = x0;
                            fx = f0;
                        }
                        const int32_t up = (int32_t)x >> 2;
                        const int2 o = column(dtop, up, fx, sext_selector(x & 3u));
                        dtop = up;
                        xout = ((uint32_t)o.x << 2) | (x & 3u);
                        fout = o.y;
                        const uint32_t col = (uint32_t)c + uu;
                        if constexpr (PTR) {
                            if (cc == CPW - 1 &&
                                in_range((uint64_t)(prow - p.ptr) + col / CPW, p.ext_off, p.err, kSiteAffPtr)) {
                                prow[col / CPW] = ptr_word(accL, accH);
                                prow[p.ext_off + col / CPW] = ptr_word(accF, accE);
                            }
                            cc = (cc + 1) & (CPW - 1);
                        }
                        row_out(col);
                    }
                    c += 32;
                    t += 31;
                    continue;
                }
            }
            uint32_t x = __shfl_up_sync(kFull, xout, 1);
            int32_t fx = __shfl_up_sync(kFull, fout, 1);
            const uint32_t x0 = __shfl_sync(kFull, stage, t & 31u);
            const int32_t f0 = __shfl_sync(kFull, fstage, t & 31u);
            if (lane == 0) {
                x = x0;
                fx = f0;
            }
            if (c >= 0 && c < (int32_t)n) {
                const int32_t up = (int32_t)x >> 2;
                const int2 o = column(dtop, up, fx, sext_selector(x & 3u));
                dtop = up;
                xout = ((uint32_t)o.x << 2) | (x & 3u);
                fout = o.y;
                if constexpr (PTR) {
                    const uint32_t cc = (uint32_t)c % CPW;
                    if (cc == CPW - 1 || c == (int32_t)n - 1) {
                        const uint32_t miss = (CPW - 1 - cc) * R;
                        const size_t wi = (size_t)(s * 32u + lane) * tk.ncg + (uint32_t)c / CPW;
                        if (in_range(tk.ptr_off + wi, p.ext_off, p.err, kSiteAffPtr)) {
                            pbase[wi] = ptr_word(accL << miss, accH << miss);
                            pbase[p.ext_off + wi] = ptr_word(accF << miss, accE << miss);
                        }
                    }
                }
                row_out((uint32_t)c);
                if (s + 1 == S && (uint32_t)lane == lM && c == (int32_t)n - 1) {
                    int32_t wmn = 0;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if ((uint32_t)r == rM) wmn = Wl[r];
                    if (in_range(tk.out, p.out_cap, p.err, kSiteAffScore))
                        p.scores[tk.out] = wmn + p.ge * (int32_t)(m + n);
                }
            }
            ++c;
        }
        __syncwarp();
        if (!alive) return;   // a wait gave up (NW_ERR_TIMEOUT is raised): leave
    }
}

// The state-machine walk from (m, n), one thread per pair: in state H the
// diagonal when L is clear, else the vertical gap (F) when H is clear, else
// the horizontal one (E); in a gap state the move is emitted and the walk
// stays in the gap while the cell's extension bit is set.  Row 0 / column
// 0: only horizontal / vertical moves remain.  Moves in reverse order (0
// diagonal, 1 vertical, 2 horizontal).
template <int R>
__global__ void k_affine_walk(const AffTask *tasks, uint32_t ntasks, const uint32_t *ptr, uint64_t ext_off,
                              uint8_t *moves, const uint64_t *move_off, uint64_t *nmoves, uint32_t *err) {
    constexpr uint32_t SH = 32u * R, CPW = 16u / R;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < ntasks; q += gridDim.x * blockDim.x) {
        const AffTask tk = tasks[q];
        const uint32_t *pw = ptr + tk.ptr_off;
        uint8_t *mv = moves + move_off[q];
        uint32_t i = tk.m, j = tk.n;
        uint64_t k = 0;
        int state = 0;   // 0 H, 1 F (vertical gap), 2 E (horizontal gap)
        while (i > 0 && j > 0) {
            if (!in_range(k, (uint64_t)tk.m + tk.n, err, kSiteAffMoves)) break;
            const uint32_t i1 = i - 1, j1 = j - 1;
            const size_t wi = (size_t)((i1 / SH) * 32u + (i1 % SH) / R) * tk.ncg + j1 / CPW;
            const uint32_t o = (j1 % CPW) * R + (i1 % R);
            if (state == 0) {
                const uint32_t word = __ldg(pw + wi);
                if (!((word >> (31u - o)) & 1u)) {
                    mv[k++] = 0;
                    --i;
                    --j;
                    continue;
                }
                state = ((word >> (15u - o)) & 1u) ? 2 : 1;
            }
            const uint32_t ext = __ldg(pw + ext_off + wi);
            if (state == 1) {
                mv[k++] = 1;
                state = ((ext >> (31u - o)) & 1u) ? 1 : 0;
                --i;
            } else {
                mv[k++] = 2;
                state = ((ext >> (15u - o)) & 1u) ? 2 : 0;
                --j;
            }
        }
        for (; j > 0; --j) mv[k++] = 2;
        for (; i > 0; --i) mv[k++] = 1;
        nmoves[q] = k;
    }
}

template <int R, bool PTR>
int launch_affine_R(nw_ctx *ctx, AffArgs &aa) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_affine<R, PTR>, kAffWarps * 32, 0);
    if (occ < 1) occ = 1;
    // every CTA resident: a job's warp may wait on an earlier job's warp
    uint32_t blocks = (uint32_t)occ * (uint32_t)ctx->sm_count;
    const uint32_t need = (aa.njobs + kAffWarps - 1) / kAffWarps;
    if (blocks > need) blocks = need ? need : 1;
    void *v = nullptr;
    int rc = scratch(ctx, "affine_counter", 16, &v);
    if (rc) return rc;
    aa.counter = (uint32_t *)v;
    cudaMemsetAsync(aa.counter, 0, 4, ctx->stream);
    LaunchTimer t(ctx, PTR ? "affine_fill_ptr" : "affine_score");
    k_affine<R, PTR><<<blocks, kAffWarps * 32, 0, ctx->stream>>>(aa);
    return NW_OK;
}

int launch_affine(nw_ctx *ctx, int R, bool ptr, AffArgs &aa) {
    if (ptr) {
        if (R == 4) return launch_affine_R<4, true>(ctx, aa);
        if (R == 16) return launch_affine_R<16, true>(ctx, aa);
        return launch_affine_R<8, true>(ctx, aa);
    }
    if (R == 4) return launch_affine_R<4, false>(ctx, aa);
    if (R == 16) return launch_affine_R<16, false>(ctx, aa);
    return launch_affine_R<8, false>(ctx, aa);
}

template <typename T>
int aff_upload(nw_ctx *ctx, const char *slot, const std::vector<T> &v, T **dev) {
    void *d = nullptr;
    int rc = to_device(ctx, v.data(), v.size() * sizeof(T), slot, &d);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);  // the host vector may be freed right after
    if (e != cudaSuccess) return cuda_fail(ctx, e, "task upload sync");
    *dev = (T *)d;
    return NW_OK;
}

// Stripe jobs of a launch's tasks (in order, stripes in order), the tasks'
// row-buffer offsets, and the row buffers and progress words in scratch.
int affine_jobs(nw_ctx *ctx, std::vector<AffTask> &tasks, int R, AffArgs &aa) {
    const uint32_t SH = 32u * R;
    std::vector<AffJob> jobs;
    uint64_t rows = 0;
    for (uint32_t q = 0; q < tasks.size(); ++q) {
        AffTask &t = tasks[q];
        const uint32_t S = (t.m && t.n) ? (t.m + SH - 1) / SH : 1;
        t.nr = (t.n + 31) / 32 * 32;
        t.row_off = rows;
        rows += (uint64_t)(S - 1) * 2 * t.nr;
        for (uint32_t s = 0; s < S; ++s) jobs.push_back(AffJob{q, s});
    }
    int rc;
    void *rv = nullptr, *pv = nullptr;
    if ((rc = scratch(ctx, "affine_rows", rows * 4 + 16, &rv))) return rc;
    if ((rc = scratch(ctx, "affine_progress", jobs.size() * 4 + 16, &pv))) return rc;
    cudaError_t e = cudaMemsetAsync(pv, 0, jobs.size() * 4, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "affine progress reset");
    AffTask *dt = nullptr;
    AffJob *dj = nullptr;
    if ((rc = aff_upload(ctx, "affine_tasks", tasks, &dt))) return rc;
    if ((rc = aff_upload(ctx, "affine_jobs", jobs, &dj))) return rc;
    aa.tasks = dt;
    aa.jobs = dj;
    aa.njobs = (uint32_t)jobs.size();
    aa.rows = (uint32_t *)rv;
    aa.rows_cap = rows;
    aa.progress = (uint32_t *)pv;
    return NW_OK;
}

int affine_device(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                  const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, const nw_affine_scoring &sc,
                  uint32_t flags, int32_t *scores, char *cigar_pool, const uint64_t *cigar_off, uint64_t *cigar_len) {
    const bool want = flags & NW_CIGAR;
    int R = 8;
    if (const char *e = getenv("NW_AFFINE_R")) R = atoi(e) == 4 ? 4 : atoi(e) == 16 ? 16 : 8;
    const uint32_t SH = 32u * R;
    AffArgs aa{};
    aa.pool = pool;
    for (int c = 0; c < 4; ++c) {
        uint32_t w = 0;
        for (int d = 0; d < 4; ++d)
            w |= (uint32_t)(uint8_t)(int8_t)((c == d ? sc.match : sc.mismatch) - 2 * sc.gap_extend) << (8 * d);
        aa.prof[c] = w;
    }
    aa.go = sc.gap_open;
    aa.ge = sc.gap_extend;
    aa.scores = scores;
    aa.err = ctx->d_err;
    aa.out_cap = npairs;
    std::vector<AffTask> all(npairs);
    for (uint32_t k = 0; k < npairs; ++k) {
        AffTask &t = all[k];
        t = AffTask{a_off[k], b_off[k], a_len[k], b_len[k], k, 0, 0, 0, 0, 0};
        if (want) t.ncg = ptr_words_per_lane_row(std::max(t.n, 1u), R);
    }
    // longest pairs first: their stripe jobs start first
    std::stable_sort(all.begin(), all.end(), [](const AffTask &x, const AffTask &y) {
        return (uint64_t)x.m * x.n > (uint64_t)y.m * y.n;
    });
    int rc;
    if (!want) {
        if ((rc = affine_jobs(ctx, all, R, aa))) return rc;
        return launch_affine(ctx, R, false, aa);
    }
    // waves whose pointer words (two arrays) fit half the free budget
    const uint64_t wave_budget = (ctx->budget - std::min(ctx->budget, ctx->used)) / 2;
    size_t k0 = 0;
    while (k0 < all.size()) {
        std::vector<AffTask> wave;
        std::vector<uint64_t> moff;
        uint64_t words = 0, mbytes = 0;
        size_t k = k0;
        for (; k < all.size(); ++k) {
            AffTask t = all[k];
            const uint64_t wds = (uint64_t)((t.m + SH - 1) / SH) * 32u * t.ncg;
            if (!wave.empty() && (words + wds) * 8 > wave_budget) break;
            t.ptr_off = words;
            words += wds;
            moff.push_back(mbytes);
            mbytes += (uint64_t)t.m + t.n + 16;
            wave.push_back(t);
        }
        void *pv = nullptr, *mv = nullptr, *nm = nullptr;
        if ((rc = scratch(ctx, "affine_ptr", words * 8 + 16, &pv))) return rc;
        if ((rc = scratch(ctx, "affine_moves", mbytes + 16, &mv))) return rc;
        if ((rc = scratch(ctx, "affine_nmoves", wave.size() * 8 + 16, &nm))) return rc;
        if ((rc = affine_jobs(ctx, wave, R, aa))) return rc;
        uint64_t *dmoff = nullptr;
        if ((rc = aff_upload(ctx, "affine_move_off", moff, &dmoff))) return rc;
        aa.ptr = (uint32_t *)pv;
        aa.ext_off = words;
        if ((rc = launch_affine(ctx, R, true, aa))) return rc;
        {
            LaunchTimer t(ctx, "affine_walk");
            const AffTask *dt = aa.tasks;
            const uint32_t blocks = std::max<uint32_t>(1, ((uint32_t)wave.size() + 127) / 128);
            if (R == 4)
                k_affine_walk<4><<<blocks, 128, 0, ctx->stream>>>(dt, (uint32_t)wave.size(), (const uint32_t *)pv,
                                                                  words, (uint8_t *)mv, dmoff, (uint64_t *)nm, ctx->d_err);
            else if (R == 16)
                k_affine_walk<16><<<blocks, 128, 0, ctx->stream>>>(dt, (uint32_t)wave.size(), (const uint32_t *)pv,
                                                                   words, (uint8_t *)mv, dmoff, (uint64_t *)nm, ctx->d_err);
            else
                k_affine_walk<8><<<blocks, 128, 0, ctx->stream>>>(dt, (uint32_t)wave.size(), (const uint32_t *)pv,
                                                                  words, (uint8_t *)mv, dmoff, (uint64_t *)nm, ctx->d_err);
        }
        std::vector<TraceTask> tt(wave.size());
        for (size_t q = 0; q < wave.size(); ++q) {
            const AffTask &t = wave[q];
            TraceTask x{};
            x.m = t.m;
            x.n = t.n;
            x.moves = (uint8_t *)mv + moff[q];
            x.nmoves = (uint64_t *)nm + q;
            x.a = pool + t.a_off;
            x.b = pool + t.b_off;
            x.cigar = cigar_pool + cigar_off[t.out];
            x.cigar_len = cigar_len + t.out;
            x.band_lo = kNoBand;
            tt[q] = x;
        }
        TraceTask *dtt = nullptr;
        if ((rc = aff_upload(ctx, "affine_trace_tasks", tt, &dtt))) return rc;
        if ((rc = launch_finish(ctx, tt[0], dtt, (uint32_t)tt.size(), (flags & NW_CIGAR_M) ? 1u : 0u))) return rc;
        k0 = k;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "affine launch");
}

uint64_t aff_pool_extent(const uint64_t *a_off, const uint32_t *a_len, const uint64_t *b_off, const uint32_t *b_len,
                         uint32_t npairs) {
    uint64_t b = 16;
    for (uint32_t k = 0; k < npairs; ++k) {
        b = std::max<uint64_t>(b, a_off[k] + (a_len[k] + 3) / 4);
        b = std::max<uint64_t>(b, b_off[k] + (b_len[k] + 3) / 4);
    }
    return b;
}

}  // namespace
}  // namespace nw

using namespace nw;

extern "C" int nw_affine_align_batch(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off,
                                     const uint32_t *a_len, const uint64_t *b_off, const uint32_t *b_len,
                                     uint32_t npairs, nw_affine_scoring sc, uint32_t flags, int32_t *scores,
                                     char *cigar_pool, const uint64_t *cigar_off, uint64_t *cigar_len) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    auto in = [](int v) { return v >= -40 && v <= 40; };
    if (!in(sc.match) || !in(sc.mismatch) || !in(sc.gap_open) || !in(sc.gap_extend))
        return fail(ctx, NW_ERR_ARG, "scores must lie in [-40, 40]");
    if (sc.gap_open > 0 || sc.gap_extend > 0) return fail(ctx, NW_ERR_ARG, "gap open and extend must be <= 0");
    if (sc.mismatch > sc.match) return fail(ctx, NW_ERR_ARG, "mismatch must be <= match");
    if (npairs == 0) return NW_OK;
    const bool want = flags & NW_CIGAR;
    if (!pool2b || !a_off || !a_len || !b_off || !b_len || !scores) return fail(ctx, NW_ERR_ARG, "null argument");
    if (want && (!cigar_pool || !cigar_off || !cigar_len)) return fail(ctx, NW_ERR_ARG, "CIGAR buffers are null");
    const uint64_t sp = sc.match > 2 * sc.gap_extend ? (uint64_t)(sc.match - 2 * sc.gap_extend) : 0;
    for (uint32_t k = 0; k < npairs; ++k) {
        if (a_len[k] >= (1u << 30) || b_len[k] >= (1u << 30)) return fail(ctx, NW_ERR_ARG, "sequence longer than 2^30");
        if (sp * std::min(a_len[k], b_len[k]) >= (1ull << 29))
            return fail(ctx, NW_ERR_ARG, "(match - 2*gap_extend) * min(m,n) must stay below 2^29");
        if (want && cigar_off[k + 1] - cigar_off[k] < nw_cigar_bound(a_len[k], b_len[k]))
            return fail(ctx, NW_ERR_ARG, "CIGAR capacity of pair %u below nw_cigar_bound", k);
    }
    if (!(flags & NW_HOST_IO))
        return affine_device(ctx, pool2b, a_off, a_len, b_off, b_len, npairs, sc, flags, scores, cigar_pool,
                             cigar_off, cigar_len);
    int rc;
    void *dp = nullptr, *ds = nullptr, *dc = nullptr, *dl = nullptr;
    if ((rc = to_device(ctx, pool2b, aff_pool_extent(a_off, a_len, b_off, b_len, npairs), "hio_pool", &dp))) return rc;
    if ((rc = scratch(ctx, "hio_scores", (size_t)npairs * 4, &ds))) return rc;
    if (want) {
        if ((rc = scratch(ctx, "hio_cigar", cigar_off[npairs] + 16, &dc))) return rc;
        if ((rc = scratch(ctx, "hio_cigar_len", (size_t)npairs * 8, &dl))) return rc;
    }
    if ((rc = affine_device(ctx, (const uint8_t *)dp, a_off, a_len, b_off, b_len, npairs, sc, flags, (int32_t *)ds,
                            (char *)dc, cigar_off, (uint64_t *)dl)))
        return rc;
    cudaError_t e = cudaMemcpyAsync(scores, ds, (size_t)npairs * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && want) e = cudaMemcpyAsync(cigar_len, dl, (size_t)npairs * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && want)
        e = cudaMemcpyAsync(cigar_pool, dc, cigar_off[npairs], cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "affine D2H");
    return nw_ctx_sync(ctx);
}
