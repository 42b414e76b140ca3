// Batched pairs (a7) and the banded rounds (a8): the persistent kernel.  The
// pairwise alignments of Sec. 3.2 (all pairs of a sequence family, Eq. 2),
// batched on one GPU instead of split over MPI ranks; each pair's fill is the
// Sec. 2.3 recurrence from the Sec. 2.2 boundary, in the W domain.
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
// The cell update is the one of the single-pair kernels (W domain: prmt +
// DPX add-max + max; with pointers: prmt + max + DPX add-max, and two sign
// bits appended by funnel shifts, see ptr_append).
#pragma once

#include "nw_internal.cuh"

namespace nw {

constexpr int kBatchWarps = 8;   // warps per CTA
// CTAs per SM the register allocation must allow.  1: the R = 16 pointer
// kernel takes 159 registers and an SM holds 8 warps.  Capping it at 128
// registers for 2 CTAs per SM (16 warps, no spills) measured slower on
// GB300 -- 162 ms against 128 ms per banded launch on 20,000 pairs --
// because the fewer registers cost the unrolled step its overlap.
constexpr int kBatchMinBlocks = 1;
constexpr uint32_t kMinPeriod = 96;

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
    uint64_t ptr_cap;    // words at ptr; score slots at scores (checked build)
    uint32_t score_cap;
};

// One predicated 32-bit global store (no branch around it).
__device__ __forceinline__ void st_global_if(bool p, uint32_t *dst, uint32_t v) {
    asm volatile("{.reg .pred q; setp.ne.b32 q, %0, 0; @q st.global.u32 [%1], %2;}" ::"r"((uint32_t)p), "l"(dst), "r"(v)
                 : "memory");
}

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

// Out-of-band cells of the banded variant take this value: far below any
// reachable W (>= 0) and far enough from INT32_MIN that adding scores never
// wraps.
constexpr int32_t kNegW = -(1 << 27);

// BAND (1, 2): only the diagonals d = j - i in [lo, hi] matter.  Stripe s
// runs over its band columns [cbeg(s), cend(s)] (0-based) only, and the
// boundary row/column cells outside the band are kNegW (which stops every
// path through them).  BAND 1 (the strict band) also forces the cells of
// the stripe rectangle outside the band to kNegW; BAND 2 (the region) keeps
// them: the DP then runs over the union of the stripe rectangles, a superset
// of the band, which gives a score between the banded and the full one and
// the same certificate (every path leaving the band is bounded).  The
// stripe period is the task's fixed `period`.
template <int R, bool PTR, int BAND>
__global__ void __launch_bounds__(kBatchWarps * 32, kBatchMinBlocks) k_batch(BatchArgs p) {
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
                if (in_range(tk.out0, p.score_cap, p.err, kSiteBatchScore)) p.scores[tk.out0] = sc;
                if (tk.out1 != ~0u && in_range(tk.out1, p.score_cap, p.err, kSiteBatchScore))
                    p.scores[tk.out1] = sc;
            }
            continue;
        }
        const uint32_t S = (m + SH - 1) / SH;
        const int32_t lo = BAND ? tk.lo : 0, hi = BAND ? tk.hi : 0;
        const uint32_t P = BAND ? tk.period : max(n, kMinPeriod);
        const uint32_t T = S * P + 31;
        const uint32_t sM = (m - 1) / SH, lM = ((m - 1) % SH) / R, rM = (m - 1) % R;
        uint32_t *pbase = PTR ? p.ptr + tk.ptr_off : nullptr;
        // first / last 0-based column of stripe s
        auto cbeg = [&](uint32_t st) -> int32_t { return BAND ? max(0, (int32_t)(st * SH) + lo) : 0; };
        auto cend = [&](uint32_t st) -> int32_t {
            return BAND ? min((int32_t)n - 1, (int32_t)(st * SH + SH - 1) + hi) : (int32_t)n - 1;
        };

        uint32_t prof[R];
        int32_t Wl[R];
        int32_t dtop = 0;
        uint32_t xout = 0, accL = 0, accH = 0;
        int32_t cb = cbeg(0), ce = cend(0);   // this lane's stripe columns
        auto init_rows = [&](uint32_t codes, uint32_t st) {
            const uint32_t i0 = st * SH + (uint32_t)lane * R;  // 1-based row above the lane's first row
            const bool col0 = cbeg(st) == 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t c = (codes >> (2 * r)) & 3u;
                prof[r] = c == 0 ? P0 : c == 1 ? P1 : c == 2 ? P2 : P3;
                // left boundary (column cbeg-1): grid column 0 if the band
                // reaches it (row i in band iff i <= -lo), else out of band
                Wl[r] = (!BAND || (col0 && (int32_t)(i0 + r + 1) <= -lo)) ? 0 : kNegW;
            }
            dtop = (!BAND || (col0 && (int32_t)i0 <= -lo)) ? 0 : kNegW;
            cb = cbeg(st);
            ce = cend(st);
        };
        init_rows(load_rows<R>(A, (uint32_t)lane * R, m), 0);
        uint32_t next_rows = S > 1 ? load_rows<R>(A, SH + (uint32_t)lane * R, m) : 0u;
        int32_t c = -lane;   // step within this lane's stripe (negative: not started)
        uint32_t s = 0;      // stripe of this lane

        // Lane-0 input for global index g: stripe 0 reads B (W = 0 on the
        // grid's row 0, kNegW beyond the band), later stripes read the row
        // buffer (kNegW where the previous stripe computed nothing).
        auto chunk_word = [&](uint32_t g) -> uint32_t {
            const uint32_t sg = g / P, tg = g - sg * P;
            if (sg >= S) return 0u;
            const int32_t col = cbeg(sg) + (int32_t)tg;
            if (col > cend(sg)) return 0u;
            const uint32_t bc = base_at(B, (uint32_t)col);
            if (sg == 0) return BAND && col + 1 > hi ? (((uint32_t)kNegW << 2) | bc) : bc;
            if (BAND && col > cend(sg - 1)) return ((uint32_t)kNegW << 2) | bc;
            return __ldcg(ring + col);
        };
        uint32_t stage = 0, stage_next = chunk_word((uint32_t)lane);

        for (uint32_t t = 0; t < T; ++t) {
            if ((t & 31u) == 0) {
                stage = stage_next;
                __threadfence_block();
                __syncwarp();
                stage_next = chunk_word(t + 32u + (uint32_t)lane);
                // Fast chunk: for the next 32 steps every lane stays inside its
                // stripe and short of the stripe's last column, so no step
                // needs the activity test, the stripe change, the last-column
                // word flush or the score check (not for the strict band,
                // whose edge mask lives in the general step).
                if (BAND != 1 && __all_sync(kFull, c >= 0 && s < S && c + 32 <= ce - cb)) {
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
                        int32_t d = dtop, uv = up;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const int32_t sv = (int32_t)prmt(prof[r], 0u, sel);
                            int32_t w;
                            if constexpr (PTR) {
                                const int32_t l = Wl[r], m2 = max(uv, l);
                                w = __viaddmax_s32(d, sv, m2);
                                accL = ptr_append(accL, d + sv - m2);
                                accH = ptr_append(accH, uv - l);
                            } else {
                                w = max(__viaddmax_s32(d, sv, Wl[r]), uv);
                            }
                            d = Wl[r];
                            Wl[r] = w;
                            uv = w;
                        }
                        dtop = up;
                        xout = ((uint32_t)uv << 2) | (x & 3u);
                        const uint32_t cu = (uint32_t)c + u;
                        if constexpr (PTR) {
                            if (cc == CPW - 1 &&
                                in_range((uint64_t)(prow - p.ptr) + cu / CPW, p.ptr_cap, p.err, kSiteBatchPtr))
                                prow[cu / CPW] = ptr_word(accL, accH);
                            cc = (cc + 1) & (CPW - 1);
                        }
                        st_global_if(ring_out && in_range((uint64_t)cb + cu, p.ring_stride, p.err, kSiteBatchRing),
                                     ring + cb + cu, xout);
                    }
                    c += 32;
                    t += 31;
                    continue;
                }
            }
            uint32_t x = __shfl_up_sync(kFull, xout, 1);
            const uint32_t x0 = __shfl_sync(kFull, stage, t & 31u);
            if (lane == 0) x = x0;
            const int32_t col = cb + c;
            const bool act = c >= 0 && col <= ce && s < S;
            const int32_t D0 = col - (int32_t)(s * SH + (uint32_t)lane * R);  // j - i of row 0 of the lane
            // Banded: mask only when some active lane has rows outside the
            // band this step (warp-uniform; most steps need no masking).
            const bool mask = BAND == 1 && __any_sync(kFull, act && !(D0 - (R - 1) >= lo && D0 <= hi));
            if (act) {
                const int32_t up = (int32_t)x >> 2;
                const uint32_t sel = sext_selector(x & 3u);
                int32_t d = dtop, u = up;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int32_t sv = (int32_t)prmt(prof[r], 0u, sel);
                    int32_t w;
                    if constexpr (PTR) {
                        // pointer bits: signs of d + s' - max(u, l) and u - l,
                        // off the dependency chain
                        const int32_t l = Wl[r], m2 = max(u, l);
                        w = __viaddmax_s32(d, sv, m2);
                        if (mask && (uint32_t)(D0 - r - lo) > (uint32_t)(hi - lo)) w = kNegW;
                        accL = ptr_append(accL, d + sv - m2);
                        accH = ptr_append(accH, u - l);
                    } else {
                        w = max(__viaddmax_s32(d, sv, Wl[r]), u);
                        if (mask && (uint32_t)(D0 - r - lo) > (uint32_t)(hi - lo)) w = kNegW;
                    }
                    d = Wl[r];
                    Wl[r] = w;
                    u = w;
                }
                dtop = up;
                xout = ((uint32_t)u << 2) | (x & 3u);
                if constexpr (PTR) {
                    const uint32_t cc = (uint32_t)c % CPW;
                    if (cc == CPW - 1 || col == ce) {
                        const uint32_t miss = (CPW - 1 - cc) * R;  // cells a row's last word lacks
                        const size_t wi = (size_t)(s * 32u + lane) * tk.ncg + (uint32_t)c / CPW;
                        if (in_range(tk.ptr_off + wi, p.ptr_cap, p.err, kSiteBatchPtr))
                            pbase[wi] = ptr_word(accL << miss, accH << miss);
                    }
                }
                if (lane == 31 && s + 1 < S && in_range((uint64_t)col, p.ring_stride, p.err, kSiteBatchRing))
                    ring[col] = xout;
                if (s == sM && (uint32_t)lane == lM && col == (int32_t)n - 1) {
                    int32_t wmn = 0;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if ((uint32_t)r == rM) wmn = Wl[r];
                    const int32_t sc = wmn + p.gap * (int32_t)(m + n);
                    if (in_range(tk.out0, p.score_cap, p.err, kSiteBatchScore)) p.scores[tk.out0] = sc;
                    if (tk.out1 != ~0u && in_range(tk.out1, p.score_cap, p.err, kSiteBatchScore))
                        p.scores[tk.out1] = sc;
                }
            }
            if (++c == (int32_t)P) {
                c = 0;
                ++s;
                if (s < S) {
                    init_rows(next_rows, s);
                    next_rows = s + 1 < S ? load_rows<R>(A, (s + 1) * SH + (uint32_t)lane * R, m) : 0u;
                    // Banded: lane 0's first cell has its diagonal neighbour on
                    // diagonal lo, inside the band -- the previous stripe's
                    // bottom row at column cb-1 (written by lane 31 at least
                    // P-SH-32 >= 64 steps ago, past two fences).
                    if (BAND && lane == 0 && cb > 0) dtop = (int32_t)__ldcg(ring + cb - 1) >> 2;
                }
            }
        }
        __syncwarp();
    }
}

// scores[tasks[i].out0] for the tasks of a launch, gathered for one copy back.
__global__ void k_gather_scores(const BatchTask *tasks, uint32_t n, const int32_t *scores, int32_t *out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = scores[tasks[i].out0];
}

// Diagonal of the all-vs-all matrix: score(a, a) = len * match.
__global__ void k_diag(const uint32_t *len, uint32_t nseq, int32_t match, int32_t *out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nseq; i += gridDim.x * blockDim.x)
        out[(size_t)i * nseq + i] = (int32_t)len[i] * match;
}

}  // namespace nw
