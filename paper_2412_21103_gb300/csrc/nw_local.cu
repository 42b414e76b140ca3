// Local alignment (Smith-Waterman; not in the paper): the Sec. 2.3 grid with
// a floor of 0, so an alignment may start and end anywhere:
//     H(i,0) = H(0,j) = 0,
//     H(i,j) = max(0, H(i-1,j-1) + s(A_i,B_j), H(i-1,j) + gap, H(i,j-1) + gap).
// The score is the largest H; the alignment ends at the first cell in
// row-major order holding it and is walked back with the priority diagonal >
// vertical > horizontal until a cell whose H is 0 (its start).
//
// Batched like the global kernel: one warp per pair, taken from an atomic
// queue in descending cell order; lane k owns R rows of a 32R-row stripe
// and walks the stripes back to back (lane 31 hands the stripe's bottom row
// to lane 0 through a per-warp row buffer).  The floor rules out the W
// domain of the global kernels (it would turn into a floor that grows along
// every anti-diagonal), so the cell works on H itself: with m = max(H_up,
// H_left), one cell is a byte permute (s), one max, one add (m + gap) and
// one DPX add-max with ReLU, max(H_diag + s, m + gap, 0) -- the four
// integer operations of the textbook cell.  Tracking the largest H costs
// one more max per cell; when the end cell is wanted, each lane keeps per
// row the largest H and the first column holding it (a DPX max that also
// reports the comparison, and a select), folded into the lane's best when
// the lane leaves the stripe.  Pointer bits are the global kernels' (L: the
// diagonal candidate is below max(up, left) + gap; H: left above up), so
// the walk reads them as usual and tracks H along the path to find the
// start.
#include <algorithm>
#include <vector>

#include "nw_internal.cuh"

namespace nw {
namespace {

constexpr int kLocalWarps = 8;
constexpr uint32_t kLocalMinPeriod = 96;   // ring reuse distance (see the stripe hand-off)
constexpr uint32_t kPadProfile = 0x80808080u;  // rows past the end: s = -128, never above a real row

struct LocalTask {
    uint64_t a_off, b_off;
    uint32_t m, n;
    uint32_t out;        // pair index
    uint32_t ncg;        // pointer words per lane row
    uint64_t ptr_off;    // word offset of the pair's pointer words
};

struct LocalArgs {
    const uint8_t *pool;
    const LocalTask *tasks;
    uint32_t ntasks;
    uint32_t *counter;
    uint32_t prof[4];    // byte d of prof[c] = s(c, d) as int8
    int32_t gap;
    uint32_t *ring;
    uint32_t ring_stride;
    int32_t *scores;     // [out]
    uint32_t *ends;      // [4*out]: i_start, j_start, i_end, j_end (POS)
    uint32_t *ptr;
    uint32_t *err;
    uint64_t ptr_cap;    // words at ptr, pairs at scores / ends (checked build)
    uint32_t out_cap;
};

template <int R>
__device__ __forceinline__ uint32_t rows_codes(const uint8_t *s, uint32_t i0, uint32_t m) {
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

__device__ __forceinline__ void st_if(bool p, uint32_t *dst, uint32_t v) {
    asm volatile("{.reg .pred q; setp.ne.b32 q, %0, 0; @q st.global.u32 [%1], %2;}" ::"r"((uint32_t)p), "l"(dst), "r"(v)
                 : "memory");
}

// (v, i, j) beats (v2, i2, j2): larger value, then smaller row, then column.
__device__ __forceinline__ bool first_max(int32_t v, uint32_t i, uint32_t j, int32_t v2, uint32_t i2, uint32_t j2) {
    return v > v2 || (v == v2 && (i < i2 || (i == i2 && j < j2)));
}

template <int R, bool PTR, bool POS>
__global__ void __launch_bounds__(kLocalWarps * 32) k_local(LocalArgs p) {
    constexpr uint32_t SH = 32u * R;
    constexpr uint32_t CPW = PTR ? 16u / R : 1u;
    constexpr int RT = POS ? R : 1;
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t *ring = p.ring + (size_t)gw * p.ring_stride;
    const int32_t g = p.gap;
    const uint32_t P0 = p.prof[0], P1 = p.prof[1], P2 = p.prof[2], P3 = p.prof[3];

    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(p.counter, 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= p.ntasks) break;
        const LocalTask tk = p.tasks[idx];
        const uint8_t *A = p.pool + tk.a_off;
        const uint8_t *B = p.pool + tk.b_off;
        const uint32_t m = tk.m, n = tk.n;
        if (m == 0 || n == 0) {
            if (lane == 0 && in_range(tk.out, p.out_cap, p.err, kSiteLocalOut)) {
                p.scores[tk.out] = 0;
                if (POS)
                    for (int q = 0; q < 4; ++q) p.ends[4 * (size_t)tk.out + q] = (PTR || q >= 2) ? 0u : ~0u;
            }
            continue;
        }
        const uint32_t S = (m + SH - 1) / SH;
        const uint32_t P = max(n, kLocalMinPeriod);
        const uint32_t T = S * P + 31;
        uint32_t *pbase = PTR ? p.ptr + tk.ptr_off : nullptr;

        uint32_t prof[R];
        int32_t Hl[R];
        int32_t rbest[RT];
        uint32_t rcol[RT];
        int32_t best = 0;            // the lane's largest H so far
        uint32_t bi = 0, bj = 0;     // POS: its cell (row-major first)
        int32_t dtop = 0;
        uint32_t xout = 0, accL = 0, accH = 0;
        auto init_rows = [&](uint32_t codes, uint32_t st) {
            const uint32_t i0 = st * SH + (uint32_t)lane * R;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t c = (codes >> (2 * r)) & 3u;
                prof[r] = i0 + r >= m ? kPadProfile : c == 0 ? P0 : c == 1 ? P1 : c == 2 ? P2 : P3;
                Hl[r] = 0;                          // column 0
            }
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                rbest[r] = 0;
                rcol[r] = 0;
            }
            dtop = 0;
        };
        // POS: the rows of stripe st (rows past m excluded) into the lane's
        // best; rows in order, so an earlier row keeps a tie
        auto fold = [&](uint32_t st) {
            if constexpr (POS) {
                const uint32_t i0 = st * SH + (uint32_t)lane * R;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (i0 + r < m && rbest[r] > best) {
                        best = rbest[r];
                        bi = i0 + r + 1;
                        bj = rcol[r] + 1;
                    }
            }
        };
        init_rows(rows_codes<R>(A, (uint32_t)lane * R, m), 0);
        uint32_t next_rows = S > 1 ? rows_codes<R>(A, SH + (uint32_t)lane * R, m) : 0u;
        int32_t c = -lane;
        uint32_t s = 0;
        // lane 0's input for global index gi: row 0 (H = 0) in stripe 0, the
        // previous stripe's bottom row (written by lane 31 at least P - 94
        // steps earlier, past the fences below) in later stripes
        auto chunk_word = [&](uint32_t gi) -> uint32_t {
            const uint32_t sg = gi / P, tg = gi - sg * P;
            if (sg >= S || tg >= n) return 0u;
            if (sg == 0) return base_at(B, tg);
            return __ldcg(ring + tg);
        };
        uint32_t stage = 0, stage_next = chunk_word((uint32_t)lane);

        // one cell: returns H, appends pointer bits, tracks the maxima
        auto cell = [&](int r, int32_t d, int32_t u, uint32_t sel, int32_t col) -> int32_t {
            const int32_t sv = (int32_t)prmt(prof[r], 0u, sel);
            const int32_t l = Hl[r];
            const int32_t mg = max(u, l) + g;
            const int32_t w = __viaddmax_s32_relu(d, sv, mg);
            if constexpr (PTR) {
                accL = ptr_append(accL, d + sv - mg);
                accH = ptr_append(accH, u - l);
            }
            if constexpr (POS) {
                bool keep;
                rbest[r] = __vibmax_s32(rbest[r], w, &keep);
                rcol[r] = keep ? rcol[r] : (uint32_t)col;
            } else {
                best = max(best, w);
            }
            return w;
        };

        for (uint32_t t = 0; t < T; ++t) {
            if ((t & 31u) == 0) {
                stage = stage_next;
                __threadfence_block();
                __syncwarp();
                stage_next = chunk_word(t + 32u + (uint32_t)lane);
                // 32 steps with every lane inside its stripe, short of its
                // last column: no activity test, stripe change or flush
                if (__all_sync(kFull, c >= 0 && s < S && c + 32 <= (int32_t)n - 1)) {
                    const bool ring_out = lane == 31 && s + 1 < S;
                    uint32_t cc = (uint32_t)c % CPW;
                    uint32_t *prow = PTR ? pbase + (size_t)(s * 32u + lane) * tk.ncg : nullptr;
#pragma unroll 4
                    for (uint32_t u = 0; u < 32u; ++u) {
                        uint32_t x = __shfl_up_sync(kFull, xout, 1);
                        const uint32_t x0 = __shfl_sync(kFull, stage, u);
                        if (lane == 0) x = x0;
                        const int32_t up = (int32_t)x >> 2;
                        const uint32_t sel = sext_selector(x & 3u);
                        const int32_t col = c + (int32_t)u;
                        int32_t d = dtop, uv = up;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const int32_t w = cell(r, d, uv, sel, col);
                            d = Hl[r];
                            Hl[r] = w;
                            uv = w;
                        }
                        dtop = up;
                        xout = ((uint32_t)uv << 2) | (x & 3u);
                        if constexpr (PTR) {
                            if (cc == CPW - 1 && in_range((uint64_t)(prow - p.ptr) + (uint32_t)col / CPW, p.ptr_cap,
                                                          p.err, kSiteLocalPtr))
                                prow[(uint32_t)col / CPW] = ptr_word(accL, accH);
                            cc = (cc + 1) & (CPW - 1);
                        }
                        st_if(ring_out && in_range((uint64_t)col, p.ring_stride, p.err, kSiteLocalRing), ring + col,
                              xout);
                    }
                    c += 32;
                    t += 31;
                    continue;
                }
            }
            uint32_t x = __shfl_up_sync(kFull, xout, 1);
            const uint32_t x0 = __shfl_sync(kFull, stage, t & 31u);
            if (lane == 0) x = x0;
            const bool act = c >= 0 && c < (int32_t)n && s < S;
            if (act) {
                const int32_t up = (int32_t)x >> 2;
                const uint32_t sel = sext_selector(x & 3u);
                int32_t d = dtop, uv = up;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int32_t w = cell(r, d, uv, sel, c);
                    d = Hl[r];
                    Hl[r] = w;
                    uv = w;
                }
                dtop = up;
                xout = ((uint32_t)uv << 2) | (x & 3u);
                if constexpr (PTR) {
                    const uint32_t cc = (uint32_t)c % CPW;
                    if (cc == CPW - 1 || c == (int32_t)n - 1) {
                        const uint32_t miss = (CPW - 1 - cc) * R;  // cells a row's last word lacks
                        const size_t wi = (size_t)(s * 32u + lane) * tk.ncg + (uint32_t)c / CPW;
                        if (in_range(tk.ptr_off + wi, p.ptr_cap, p.err, kSiteLocalPtr))
                            pbase[wi] = ptr_word(accL << miss, accH << miss);
                    }
                }
                if (lane == 31 && s + 1 < S && in_range((uint64_t)c, p.ring_stride, p.err, kSiteLocalRing))
                    ring[c] = xout;
            }
            if (++c == (int32_t)P) {
                fold(s);
                c = 0;
                ++s;
                if (s < S) {
                    init_rows(next_rows, s);
                    next_rows = s + 1 < S ? rows_codes<R>(A, (s + 1) * SH + (uint32_t)lane * R, m) : 0u;
                }
            }
        }
        // the pair's largest H (and its first cell) over the warp
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const int32_t v2 = __shfl_xor_sync(kFull, best, o);
            const uint32_t i2 = __shfl_xor_sync(kFull, bi, o), j2 = __shfl_xor_sync(kFull, bj, o);
            if (POS ? first_max(v2, i2, j2, best, bi, bj) : v2 > best) {
                best = v2;
                bi = i2;
                bj = j2;
            }
        }
        if (lane == 0 && in_range(tk.out, p.out_cap, p.err, kSiteLocalOut)) {
            p.scores[tk.out] = best;
            if (POS) {
                p.ends[4 * (size_t)tk.out + 2] = bi;
                p.ends[4 * (size_t)tk.out + 3] = bj;
                // the start: the walk moves it from the end cell; without
                // pointers it is not computed
                p.ends[4 * (size_t)tk.out + 0] = PTR ? bi : ~0u;
                p.ends[4 * (size_t)tk.out + 1] = PTR ? bj : ~0u;
            }
        }
        __syncwarp();
    }
}

// The walk back from each pair's end cell, one thread per pair: follows the
// pointer words (layout [stripe][lane][column group]) and tracks H along
// the path, stopping where it reaches 0.  Writes the moves in reverse order
// (0 diagonal, 1 vertical, 2 horizontal), their count, and the start cell.
template <int R>
__global__ void k_local_walk(const LocalTask *tasks, uint32_t ntasks, const uint8_t *pool, const uint32_t *ptr,
                             const int32_t *scores, uint32_t *ends, uint8_t *moves, const uint64_t *move_off,
                             uint64_t *nmoves, uint32_t prof0, uint32_t prof1, uint32_t prof2, uint32_t prof3,
                             int32_t gap, uint32_t *err) {
    constexpr uint32_t SH = 32u * R, CPW = 16u / R;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < ntasks; q += gridDim.x * blockDim.x) {
        const LocalTask tk = tasks[q];
        const uint8_t *A = pool + tk.a_off, *B = pool + tk.b_off;
        const uint32_t *pw = ptr + tk.ptr_off;
        uint32_t *e = ends + 4 * (size_t)tk.out;
        uint32_t i = e[2], j = e[3];
        int32_t h = scores[tk.out];
        uint8_t *mv = moves + move_off[q];
        uint64_t k = 0;
        while (h > 0 && i > 0 && j > 0) {
            const uint32_t i1 = i - 1, j1 = j - 1;
            const uint32_t word = __ldg(pw + (size_t)((i1 / SH) * 32u + (i1 % SH) / R) * tk.ncg + j1 / CPW);
            const uint32_t d = ptr_move(word, (j1 % CPW) * R + (i1 % R));
            if (!in_range(k, (uint64_t)tk.m + tk.n, err, kSiteLocalMoves)) break;
            mv[k++] = (uint8_t)d;
            if (d == 0) {
                const uint32_t ca = base_at(A, i1), cb = base_at(B, j1);
                const uint32_t pr = ca == 0 ? prof0 : ca == 1 ? prof1 : ca == 2 ? prof2 : prof3;
                h -= (int32_t)(int8_t)(pr >> (8 * cb));
                --i;
                --j;
            } else {
                h -= gap;
                if (d == 1) --i;
                else --j;
            }
        }
        e[0] = i;
        e[1] = j;
        nmoves[q] = k;
    }
}

template <int R, bool PTR, bool POS>
int launch_local_R(nw_ctx *ctx, LocalArgs &la, uint32_t max_n) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_local<R, PTR, POS>, kLocalWarps * 32, 0);
    if (occ < 1) occ = 1;
    uint32_t blocks = (uint32_t)occ * (uint32_t)ctx->sm_count;
    const uint32_t need = (la.ntasks + kLocalWarps - 1) / kLocalWarps;
    if (blocks > need) blocks = need ? need : 1;
    la.ring_stride = ((max_n + 31) / 32) * 32 + 32;
    void *v = nullptr;
    int rc = scratch(ctx, "local_ring", (size_t)blocks * kLocalWarps * la.ring_stride * 4, &v);
    if (rc) return rc;
    la.ring = (uint32_t *)v;
    if ((rc = scratch(ctx, "local_counter", 16, &v))) return rc;
    la.counter = (uint32_t *)v;
    cudaMemsetAsync(la.counter, 0, 4, ctx->stream);
    LaunchTimer t(ctx, PTR ? "local_fill_ptr" : (POS ? "local_score_pos" : "local_score"));
    k_local<R, PTR, POS><<<blocks, kLocalWarps * 32, 0, ctx->stream>>>(la);
    return NW_OK;
}

int launch_local(nw_ctx *ctx, int R, bool ptr, bool pos, LocalArgs &la, uint32_t max_n) {
#define NW_LOCAL_CASES(PTRV, POSV)                                        \
    switch (R) {                                                          \
        case 4: return launch_local_R<4, PTRV, POSV>(ctx, la, max_n);     \
        case 16: return launch_local_R<16, PTRV, POSV>(ctx, la, max_n);   \
        default: return launch_local_R<8, PTRV, POSV>(ctx, la, max_n);    \
    }
    if (ptr) NW_LOCAL_CASES(true, true)
    if (pos) NW_LOCAL_CASES(false, true)
    NW_LOCAL_CASES(false, false)
#undef NW_LOCAL_CASES
}

template <typename T>
int upload_vec(nw_ctx *ctx, const char *slot, const std::vector<T> &v, T **dev) {
    void *d = nullptr;
    int rc = to_device(ctx, v.data(), v.size() * sizeof(T), slot, &d);
    if (rc) return rc;
    // the host vector may be freed right after: wait for the copy
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "task upload sync");
    *dev = (T *)d;
    return NW_OK;
}

// Row profiles of the plain scores s (the global kernels use s - 2*gap).
void local_profile(const nw_scoring &sc, uint32_t prof[4]) {
    for (int c = 0; c < 4; ++c) {
        uint32_t w = 0;
        for (int d = 0; d < 4; ++d) w |= (uint32_t)(uint8_t)(int8_t)(c == d ? sc.match : sc.mismatch) << (8 * d);
        prof[c] = w;
    }
}

int local_device(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                 const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, const nw_scoring &sc, uint32_t flags,
                 int32_t *scores, uint32_t *ends, char *cigar_pool, const uint64_t *cigar_off, uint64_t *cigar_len) {
    const bool want = flags & NW_CIGAR;
    int R = 8;
    if (const char *e = getenv("NW_LOCAL_R")) R = atoi(e) == 4 ? 4 : atoi(e) == 16 ? 16 : 8;
    const uint32_t SH = 32u * R;
    LocalArgs la{};
    la.pool = pool;
    local_profile(sc, la.prof);
    la.gap = sc.gap;
    la.scores = scores;
    la.ends = ends;
    la.err = ctx->d_err;
    la.out_cap = npairs;
    std::vector<LocalTask> all(npairs);
    for (uint32_t k = 0; k < npairs; ++k) {
        LocalTask &t = all[k];
        t = LocalTask{a_off[k], b_off[k], a_len[k], b_len[k], k, 0, 0};
        // one warp steps through stripes x max(n, 96) columns: a 32-bit count
        if ((uint64_t)((t.m + SH - 1) / SH) * std::max(t.n, kLocalMinPeriod) >= (1ull << 31))
            return fail(ctx, NW_ERR_UNSUPPORTED, "pair %u too large for one warp (m*n/%u >= 2^31)", k, SH);
        if (want) t.ncg = ptr_words_per_lane_row(std::max(t.n, kLocalMinPeriod), R);
    }
    // longest first (the atomic queue then balances the tail)
    std::stable_sort(all.begin(), all.end(), [](const LocalTask &x, const LocalTask &y) {
        return (uint64_t)x.m * x.n > (uint64_t)y.m * y.n;
    });
    int rc;
    if (!want) {
        uint32_t max_n = 1;
        for (const LocalTask &t : all) max_n = std::max(max_n, t.n);
        LocalTask *dt = nullptr;
        if ((rc = upload_vec(ctx, "local_tasks", all, &dt))) return rc;
        la.tasks = dt;
        la.ntasks = npairs;
        return launch_local(ctx, R, false, ends != nullptr, la, max_n);
    }
    // CIGAR: waves whose pointer words fit half the free budget
    const uint64_t wave_budget = (ctx->budget - std::min(ctx->budget, ctx->used)) / 2;
    size_t k0 = 0;
    while (k0 < all.size()) {
        std::vector<LocalTask> wave;
        std::vector<uint64_t> moff;
        uint64_t words = 0, mbytes = 0;
        uint32_t max_n = 1;
        size_t k = k0;
        for (; k < all.size(); ++k) {
            LocalTask t = all[k];
            const uint64_t wds = (uint64_t)((t.m + SH - 1) / SH) * 32u * t.ncg;
            if (!wave.empty() && (words + wds) * 4 > wave_budget) break;
            t.ptr_off = words;
            words += wds;
            moff.push_back(mbytes);
            mbytes += (uint64_t)t.m + t.n + 16;
            max_n = std::max(max_n, t.n);
            wave.push_back(t);
        }
        void *pv = nullptr, *mv = nullptr, *nm = nullptr;
        if ((rc = scratch(ctx, "local_ptr", words * 4 + 16, &pv))) return rc;
        if ((rc = scratch(ctx, "local_moves", mbytes + 16, &mv))) return rc;
        if ((rc = scratch(ctx, "local_nmoves", wave.size() * 8 + 16, &nm))) return rc;
        LocalTask *dt = nullptr;
        uint64_t *dmoff = nullptr;
        if ((rc = upload_vec(ctx, "local_tasks", wave, &dt))) return rc;
        if ((rc = upload_vec(ctx, "local_move_off", moff, &dmoff))) return rc;
        la.tasks = dt;
        la.ntasks = (uint32_t)wave.size();
        la.ptr = (uint32_t *)pv;
        la.ptr_cap = words;
        if ((rc = launch_local(ctx, R, true, true, la, max_n))) return rc;
        {
            LaunchTimer t(ctx, "local_walk");
            const uint32_t blocks = std::max<uint32_t>(1, ((uint32_t)wave.size() + 127) / 128);
#define NW_WALK(RV)                                                                                               \
    k_local_walk<RV><<<blocks, 128, 0, ctx->stream>>>(dt, (uint32_t)wave.size(), pool, (const uint32_t *)pv, scores, \
                                                      ends, (uint8_t *)mv, dmoff, (uint64_t *)nm, la.prof[0],       \
                                                      la.prof[1], la.prof[2], la.prof[3], sc.gap, ctx->d_err)
            if (R == 4) NW_WALK(4);
            else if (R == 16) NW_WALK(16);
            else NW_WALK(8);
#undef NW_WALK
        }
        std::vector<TraceTask> tt(wave.size());
        for (size_t q = 0; q < wave.size(); ++q) {
            const LocalTask &t = wave[q];
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
            x.origin = ends + 4 * (size_t)t.out;
            tt[q] = x;
        }
        TraceTask *dtt = nullptr;
        if ((rc = upload_vec(ctx, "local_trace_tasks", tt, &dtt))) return rc;
        if ((rc = launch_finish(ctx, tt[0], dtt, (uint32_t)tt.size(), (flags & NW_CIGAR_M) ? 1u : 0u))) return rc;
        k0 = k;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "local launch");
}

uint64_t pool_extent(const uint64_t *a_off, const uint32_t *a_len, const uint64_t *b_off, const uint32_t *b_len,
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

extern "C" int nw_local_align_batch(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                                    const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, nw_scoring sc,
                                    uint32_t flags, int32_t *scores, uint32_t *ends, char *cigar_pool,
                                    const uint64_t *cigar_off, uint64_t *cigar_len) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    int rc = check_scoring(ctx, sc);
    if (rc) return rc;
    if (npairs == 0) return NW_OK;
    const bool want = flags & NW_CIGAR;
    if (!pool2b || !a_off || !a_len || !b_off || !b_len || !scores) return fail(ctx, NW_ERR_ARG, "null argument");
    if (want && (!ends || !cigar_pool || !cigar_off || !cigar_len))
        return fail(ctx, NW_ERR_ARG, "NW_CIGAR needs ends and CIGAR buffers");
    for (uint32_t k = 0; k < npairs; ++k) {
        if (a_len[k] >= (1u << 30) || b_len[k] >= (1u << 30)) return fail(ctx, NW_ERR_ARG, "sequence longer than 2^30");
        const uint64_t mn = std::min(a_len[k], b_len[k]);
        if ((uint64_t)std::max(sc.match, 0) * mn >= (1ull << 29))
            return fail(ctx, NW_ERR_ARG, "match * min(m,n) must stay below 2^29");
        if (want && cigar_off[k + 1] - cigar_off[k] < nw_cigar_bound(a_len[k], b_len[k]))
            return fail(ctx, NW_ERR_ARG, "CIGAR capacity of pair %u below nw_cigar_bound", k);
    }
    if (!(flags & NW_HOST_IO))
        return local_device(ctx, pool2b, a_off, a_len, b_off, b_len, npairs, sc, flags, scores, ends, cigar_pool,
                            cigar_off, cigar_len);
    void *dp = nullptr, *ds = nullptr, *de = nullptr, *dc = nullptr, *dl = nullptr;
    if ((rc = to_device(ctx, pool2b, pool_extent(a_off, a_len, b_off, b_len, npairs), "hio_pool", &dp))) return rc;
    if ((rc = scratch(ctx, "hio_scores", (size_t)npairs * 4, &ds))) return rc;
    if (ends && (rc = scratch(ctx, "hio_ends", (size_t)npairs * 16, &de))) return rc;
    if (want) {
        if ((rc = scratch(ctx, "hio_cigar", cigar_off[npairs] + 16, &dc))) return rc;
        if ((rc = scratch(ctx, "hio_cigar_len", (size_t)npairs * 8, &dl))) return rc;
    }
    if ((rc = local_device(ctx, (const uint8_t *)dp, a_off, a_len, b_off, b_len, npairs, sc, flags, (int32_t *)ds,
                           (uint32_t *)de, (char *)dc, cigar_off, (uint64_t *)dl)))
        return rc;
    cudaError_t e = cudaMemcpyAsync(scores, ds, (size_t)npairs * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && ends) e = cudaMemcpyAsync(ends, de, (size_t)npairs * 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && want) e = cudaMemcpyAsync(cigar_len, dl, (size_t)npairs * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && want)
        e = cudaMemcpyAsync(cigar_pool, dc, cigar_off[npairs], cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "local D2H");
    return nw_ctx_sync(ctx);
}
