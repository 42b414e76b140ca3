// Traceback (a5) and CIGAR assembly, shared by the single-pair and the
// batched paths.  The walk of Sec. 2.4 from (m,n) back to (0,0), taking one
// optimal path in the priority order diagonal > vertical > horizontal (the
// 1/2/3 codes of Sec. 3.1).  A task describes one pair: its pointer words (layout
// [stripe][lane][column group], R rows x 16/R columns per word), its
// sequences and where its moves and CIGAR go.  One CTA per task.
#include <algorithm>
#include <vector>

#include <cstdlib>

#include "nw_internal.cuh"

namespace nw {

// ---------------------------------------------------------------- traceback
// One warp.  The walk itself is sequential (lane 0); the warp loads the
// 8-lane x 32-word pointer tile that holds the current cell into shared
// memory whenever the walk leaves the previous tile.  Emits move codes in
// reverse order: 0 diagonal, 1 vertical ('I'), 2 horizontal ('D').


template <int R>
__global__ void __launch_bounds__(32) k_traceback(TraceTask one, const TraceTask *many) {
    const TraceTask &p = many ? many[blockIdx.x] : one;
    constexpr uint32_t SH = 32u * R, CPW = 16u / R;
    __shared__ __align__(16) uint32_t tile[kTileLanes * kTileWords];
    const uint32_t lane = threadIdx.x;
    uint32_t i = p.m, j = p.n;
    uint64_t k = 0;
    if (p.state) {
        // resumed walk: the pointer words of stripes [s_lo, ...) are present
        if (p.state[4]) return;
        i = p.state[0];
        j = p.state[1];
        k = (uint64_t)p.state[2] | ((uint64_t)p.state[3] << 32);
    }
    const uint32_t s_lo = p.s_lo;
    uint32_t cs = 0xffffffffu, ckt = 0, cct = 0;
    // first stored column of stripe s (banded layout) or 0
    auto cbeg = [&](uint32_t s) -> uint32_t {
        if (p.band_lo == kNoBand) return 0u;
        const int64_t v = (int64_t)s * SH + p.band_lo;
        return v > 0 ? (uint32_t)v : 0u;
    };
    while (i > 0 && j > 0 && (i - 1) / SH >= s_lo) {
        const uint32_t i1 = i - 1, j1 = j - 1;
        const uint32_t s = i1 / SH, kt = ((i1 % SH) / R) / kTileLanes, ct = ((j1 - cbeg(s)) / CPW) / kTileWords;
        if (s != cs || kt != ckt || ct != cct) {
            __syncwarp();
            const uint32_t rl = lane >> 2, part = lane & 3u;
            const size_t base =
                (size_t)((s - s_lo) * 32u + kt * kTileLanes + rl) * p.ncg + ct * kTileWords + part * 8u;
            const uint4 v0 = __ldcg(reinterpret_cast<const uint4 *>(p.ptr + base));
            const uint4 v1 = __ldcg(reinterpret_cast<const uint4 *>(p.ptr + base + 4));
            uint4 *dst = reinterpret_cast<uint4 *>(tile + rl * kTileWords + part * 8u);
            dst[0] = v0;
            dst[1] = v1;
            __syncwarp();
            cs = s;
            ckt = kt;
            cct = ct;
        }
        if (lane == 0) {
            const uint32_t cb = cbeg(cs);
            while (i > 0 && j > 0) {
                const uint32_t a1 = i - 1, b1 = j - 1;
                const uint32_t kk = (a1 % SH) / R;
                if (a1 / SH != cs || b1 < cb) break;
                const uint32_t cg = (b1 - cb) / CPW;
                if (kk / kTileLanes != ckt || cg / kTileWords != cct) break;
                const uint32_t word = tile[(kk - ckt * kTileLanes) * kTileWords + (cg - cct * kTileWords)];
                const uint32_t mv = ptr_move(word, ((b1 - cb) % CPW) * R + (a1 % R));
                p.moves[k++] = (uint8_t)mv;
                i -= (mv != 2u);
                j -= (mv != 1u);
            }
        }
        i = __shfl_sync(kFull, i, 0);
        j = __shfl_sync(kFull, j, 0);
        k = __shfl_sync(kFull, k, 0);
    }
    if (i > 0 && j > 0) {
        // paused at the top of the stripes present (resumable walks only)
        __syncwarp();
        if (lane == 0) {
            p.state[0] = i;
            p.state[1] = j;
            p.state[2] = (uint32_t)k;
            p.state[3] = (uint32_t)(k >> 32);
        }
        return;
    }
    // Row 0 / column 0: only horizontal / vertical moves remain.
    const uint32_t rest = i + j;
    const uint8_t mv = i ? 1 : 2;
    for (uint32_t q = lane; q < rest; q += 32) p.moves[k + q] = mv;
    if (lane == 0) {
        *p.nmoves = k + rest;
        if (p.state) {
            p.state[0] = 0;
            p.state[1] = 0;  // no columns left for the passes above
            p.state[4] = 1;
        }
    }
}

// ------------------------------------------------------ stripe-parallel walk
// The walk is sequential, but its pieces need not be found in order.  Every
// stripe of a long pair gets two walks, all stripes at once:
//   spec -- from a guessed cell (on the proportional diagonal) of the
//           bottom row of the stripe below, unrecorded through that stripe,
//           then recorded through this one until it leaves it (the last
//           stripe starts at (m, n) itself).  It records, per row, the
//           columns it visited and its move count on entering the row.
//   link -- from the cell where the stripe below's spec walk left, until it
//           steps onto this stripe's spec path (from there the two are one
//           walk: a move depends only on the cell) or leaves the stripe.
// Then one warp per pair follows the true path stripe by stripe: where the
// true entry is the link walk's start, the stripe's moves are the link
// prefix plus the spec suffix; otherwise (guess too far off, a walk past its
// move cap) it walks the stripe itself, still joining the spec path where it
// can.  Tracebacks from nearby cells merge within a few gap lengths, so for
// similar sequences the sequential pass mostly just links the pieces.  The
// moves are those of the plain walk, one for one.
constexpr uint32_t kWalkDone = 0, kWalkJoined = 1, kWalkFull = 2, kWalkBand = 3, kWalkNone = 4;
constexpr int kWalkWarps = 4;
constexpr uint32_t kParMinStripes = 3;     // shorter pairs walk sequentially,
constexpr uint64_t kParMinMoves = 8192;    // and so do pairs of a batch with m + n below this (the
                                           // other pairs' walks keep the GPU busy, and the
                                           // speculative walks add work)
constexpr uint64_t kParMinMovesOne = 1024; // a lone pair walks in parallel from m + n = 1024 up:
                                           // a 1,000 x 1,000 pair's traceback takes 0.10 ms
                                           // instead of 0.17 ms sequentially (GB300)

struct StripeJob {
    uint64_t moff;  // byte offset of the stripe's spec moves; its link moves follow at moff + lcap
    uint64_t roff;  // offset (uint2 units) of its row records
    uint32_t task, s, lcap, pad;
};

// Job g when the jobs are implicit (one task, stripes 0..S-1, cap lcap).
__device__ __forceinline__ StripeJob job_of(const StripeJob *jobs, uint32_t g, uint32_t lcap, uint32_t SH) {
    if (jobs) return jobs[g];
    StripeJob j;
    j.moff = (uint64_t)g * 2u * lcap;
    j.roff = (uint64_t)g * SH;
    j.task = 0;
    j.s = g;
    j.lcap = lcap;
    j.pad = 0;
    return j;
}

// Pointer layouts the walks read.  A layout splits the rows into stripes of
// at most SH rows (stripe s: rows top(s)+1 .. bot(s)), names the staged tile
// that holds a cell (key), stages it (load, the whole warp) and decodes the
// move of a cell from it.  Cells are (a1, b1) = (i-1, j-1).
//
// Scalar fills: stripes of 32R rows from the top, words of R rows x 16/R
// columns in [stripe][lane][column group] order, optionally banded (stripe s
// keeps the columns from max(0, s*32R + band_lo)); a tile is 8 lane rows x
// 32 words.
template <int R>
struct ScalarLayout {
    static constexpr uint32_t SH = 32u * R, CPW = 16u / R;
    __device__ static uint32_t stripes(const TraceTask &p) { return (p.m + SH - 1) / SH; }
    __device__ static uint32_t top(const TraceTask &, uint32_t s) { return s * SH; }
    __device__ static uint32_t bot(const TraceTask &p, uint32_t s) { return min(p.m, (s + 1) * SH); }
    __device__ static uint32_t stripe_of(const TraceTask &, uint32_t a1) { return a1 / SH; }
    __device__ static uint32_t cbeg(const TraceTask &p, uint32_t s) {
        if (p.band_lo == kNoBand) return 0u;
        const int64_t v = (int64_t)s * SH + p.band_lo;
        return v > 0 ? (uint32_t)v : 0u;
    }
    __device__ static uint32_t cend(const TraceTask &p, uint32_t s) {
        return p.band_lo == kNoBand ? p.n : min(p.n, cbeg(p, s) + p.ncg * CPW);
    }
    __device__ static uint32_t key(const TraceTask &, uint32_t top, uint32_t cb, uint32_t a1, uint32_t b1) {
        return (((b1 - cb) / CPW) / kTileWords) * 4u + ((a1 - top) / R) / kTileLanes;
    }
    __device__ static void load(const TraceTask &p, uint32_t s, uint32_t key, uint32_t *tile, uint32_t lane) {
        const uint32_t kt = key & 3u, ct = key >> 2;
        const uint32_t rl = lane >> 2, part = lane & 3u;
        const size_t base = (size_t)((s - p.s_lo) * 32u + kt * kTileLanes + rl) * p.ncg + ct * kTileWords + part * 8u;
        const uint4 v0 = __ldcg(reinterpret_cast<const uint4 *>(p.ptr + base));
        const uint4 v1 = __ldcg(reinterpret_cast<const uint4 *>(p.ptr + base + 4));
        uint4 *dst = reinterpret_cast<uint4 *>(tile + rl * kTileWords + part * 8u);
        dst[0] = v0;
        dst[1] = v1;
    }
    __device__ static uint32_t move(const TraceTask &, const uint32_t *tile, uint32_t top, uint32_t cb, uint32_t a1,
                                    uint32_t b1) {
        const uint32_t kk = (a1 - top) / R, cg = (b1 - cb) / CPW;
        const uint32_t word = tile[(kk % kTileLanes) * kTileWords + cg % kTileWords];
        return ptr_move(word, ((b1 - cb) % CPW) * R + (a1 % R));
    }
};

// Bit-sliced single-pair fill: bit stripes of 31 rows from the top (bit
// stripe s: rows 31s + 1 .. 31s + 31).  Bit stripe s is lane l = s % 32 of
// warp w = s / 32, and its step t is the warp's step tau = t + 32l; one
// record (L, Hb) per bit stripe and step, laid out [warp][tau / 2][lane] in
// 16-byte pairs of steps (ncg = pairs per warp).  Bit p of the step-t
// record is the cell of row 31s + p + 1 and column t + 1 - p; L = 0 where
// the diagonal predecessor attains the maximum, Hb = 0 where the upper one
// does.  The walk's stripes are G bit stripes each, so that a speculative
// walk has room to meet the true path; a tile is 64 consecutive steps of
// one bit stripe.
template <uint32_t G>
struct BitsLayout {
    static constexpr uint32_t RS = 31u, SH = RS * G;
    __device__ static uint32_t stripes(const TraceTask &p) { return (p.m + SH - 1) / SH; }
    __device__ static uint32_t top(const TraceTask &, uint32_t g) { return g * SH; }
    __device__ static uint32_t bot(const TraceTask &p, uint32_t g) { return min(p.m, (g + 1) * SH); }
    __device__ static uint32_t stripe_of(const TraceTask &, uint32_t a1) { return a1 / SH; }
    __device__ static uint32_t cbeg(const TraceTask &, uint32_t) { return 0u; }
    __device__ static uint32_t cend(const TraceTask &p, uint32_t) { return p.n; }
    __device__ static uint32_t key(const TraceTask &, uint32_t, uint32_t, uint32_t a1, uint32_t b1) {
        const uint32_t s = a1 / RS, bit = a1 - s * RS;
        return ((s % G) << 24) | ((b1 + bit) >> 6);  // bit stripe within the walk stripe, 64-step tile
    }
    __device__ static void load(const TraceTask &p, uint32_t g, uint32_t key, uint32_t *tile, uint32_t lane) {
        const uint32_t s = g * G + (key >> 24);
        const uint32_t w = s >> 5, l = s & 31u;
        const size_t row = (size_t)w * p.ncg + (size_t)(key & 0xffffffu) * 32u + 16u * l;  // tau = 64 tile + 32 l
        reinterpret_cast<uint4 *>(tile)[lane] = __ldcg(reinterpret_cast<const uint4 *>(p.ptr) + (row + lane) * 32u + l);
    }
    __device__ static uint32_t move(const TraceTask &, const uint32_t *tile, uint32_t, uint32_t, uint32_t a1,
                                    uint32_t b1) {
        const uint32_t bit = a1 % RS, t = (b1 + bit) & 63u;
        const uint32_t L = (tile[2 * t] >> bit) & 1u, H = (tile[2 * t + 1] >> bit) & 1u;
        return L ? (H ? 2u : 1u) : 0u;
    }
};
constexpr uint32_t kBitsWalkGroup = 8;  // bit stripes per walk stripe (248 rows)

// Walk from (i, j) inside stripe s until the walk leaves the stripe or
// reaches row / column 0 (kWalkDone), steps on a cell of the spec path in
// `arow` (kWalkJoined; JOIN only; a_from = the spec's move count there), has
// made `cap` moves (kWalkFull) or would read a column left of the stored
// band (kWalkBand).  RECORD writes the row records {entry column,
// (entry - exit column) | moves-before-entry << 16}, indexed by row - top.
// Moves go to out[k..].  Lane 0 walks, the warp stages the layout's tiles;
// i, j, k and the status are valid in every lane on return.
template <class LY, bool RECORD, bool JOIN>
__device__ uint32_t walk_stripe(const TraceTask &p, uint32_t s, uint32_t &i, uint32_t &j, uint32_t &k, uint32_t cap,
                                uint8_t *out, uint2 *rec, const uint2 *arow, uint32_t &a_from, uint32_t *tile) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t top = LY::top(p, s), cb = LY::cbeg(p, s);
    uint32_t ckey = 0xffffffffu;
    uint32_t status = kWalkDone, rjhi = j, ridx = k;
    for (;;) {
        uint32_t need = 0, nkey = 0;
        if (lane == 0) {
            for (;;) {
                if (i == 0 || j == 0 || i <= top) {
                    status = kWalkDone;
                    break;
                }
                if (JOIN) {
                    const uint2 r = arow[i - 1 - top];
                    if (j <= r.x && j + (r.y & 0xffffu) >= r.x) {
                        status = kWalkJoined;
                        a_from = (r.y >> 16) + (r.x - j);
                        break;
                    }
                }
                if (k >= cap) {
                    status = kWalkFull;
                    break;
                }
                const uint32_t a1 = i - 1, b1 = j - 1;
                if (b1 < cb) {
                    status = kWalkBand;
                    break;
                }
                const uint32_t key = LY::key(p, top, cb, a1, b1);
                if (key != ckey) {
                    need = 1;
                    nkey = key;
                    break;
                }
                const uint32_t mv = LY::move(p, tile, top, cb, a1, b1);
                out[k] = (uint8_t)mv;
                ++k;
                if (RECORD && mv != 2u) {  // leaving row i
                    rec[a1 - top] = make_uint2(rjhi, (rjhi - j) | (ridx << 16));
                    rjhi = j - (mv == 0u);
                    ridx = k;
                }
                i -= (mv != 2u);
                j -= (mv != 1u);
            }
        }
        need = __shfl_sync(kFull, need, 0);
        if (!need) break;
        nkey = __shfl_sync(kFull, nkey, 0);
        __syncwarp();
        LY::load(p, s, nkey, tile, lane);
        __syncwarp();
        ckey = nkey;
    }
    if (RECORD && lane == 0 && status == kWalkDone && j == 0 && i > top)
        rec[i - 1 - top] = make_uint2(rjhi, rjhi | (ridx << 16));
    i = __shfl_sync(kFull, i, 0);
    j = __shfl_sync(kFull, j, 0);
    k = __shfl_sync(kFull, k, 0);
    a_from = __shfl_sync(kFull, a_from, 0);
    return __shfl_sync(kFull, status, 0);
}

// Spec (LINK = false) or link (LINK = true) walks, one warp per stripe job.
template <class LY, bool LINK>
__global__ void __launch_bounds__(kWalkWarps * 32, 1) k_tb_stripes(TraceTask one, const TraceTask *many,
                                                                const StripeJob *jobs, uint32_t njobs, uint32_t lcap,
                                                                uint8_t *mbuf, uint2 *rows, uint4 *asum, uint4 *bsum) {
    constexpr uint32_t SH = LY::SH;
    __shared__ __align__(16) uint32_t tiles[kWalkWarps][kTileLanes * kTileWords];
    __shared__ uint2 arows[LINK ? kWalkWarps : 1][LINK ? SH : 1];
    const uint32_t lane = threadIdx.x & 31u, wi = threadIdx.x >> 5;
    const uint32_t g = blockIdx.x * kWalkWarps + wi;
    if (g >= njobs) return;
    const StripeJob jb = job_of(jobs, g, lcap, SH);
    const TraceTask &p = many ? many[jb.task] : one;
    const uint32_t s = jb.s;
    const uint32_t S = LY::stripes(p);
    uint2 *rec = rows + jb.roff;
    uint32_t a_from = 0, k = 0;
    if (!LINK) {
        for (uint32_t r = lane; r < SH; r += 32) rec[r] = make_uint2(0u, 0u);
        __syncwarp();
        // guess for the bottom row of stripe q: the proportional diagonal,
        // kept inside the stored columns
        auto guess = [&](uint32_t q, uint32_t row) -> uint32_t {
            const uint32_t g = (uint32_t)(((uint64_t)row * p.n + p.m / 2) / p.m);
            const uint32_t lo = LY::cbeg(p, q) + 1, hi = LY::cend(p, q);
            return max(lo, min(g, hi));
        };
        uint32_t i = LY::bot(p, s), j = p.n;
        if (s + 1 < S) {
            j = guess(s, i);
            // burn-in: start one stripe lower and walk up to this stripe's
            // bottom row unrecorded; walks from different cells merge, so the
            // entry it reaches is usually the true path's
            uint32_t bi = LY::bot(p, s + 1), bj = s + 2 < S ? guess(s + 1, bi) : p.n;
            uint32_t bk = 0, bf = 0;
            const uint32_t bst = walk_stripe<LY, false, false>(p, s + 1, bi, bj, bk, jb.lcap, mbuf + jb.moff, nullptr,
                                                               nullptr, bf, tiles[wi]);
            if (bst == kWalkDone && bi == i && bj > 0) j = bj;
        }
        const uint32_t st = walk_stripe<LY, true, false>(p, s, i, j, k, jb.lcap, mbuf + jb.moff, rec, nullptr, a_from,
                                                         tiles[wi]);
        if (lane == 0) asum[g] = make_uint4(i, j, k, st);
    } else {
        uint32_t si = p.m, sj = p.n;
        if (s + 1 < S) {
            const uint4 a = asum[g + 1];  // the stripe below (jobs of a task are consecutive)
            if (a.w != kWalkDone || a.x == 0 || a.y == 0) {
                if (lane == 0) {
                    bsum[2 * (size_t)g] = make_uint4(0u, 0u, 0u, 0u);
                    bsum[2 * (size_t)g + 1] = make_uint4(0u, 0u, kWalkNone, 0u);
                }
                return;
            }
            si = a.x;
            sj = a.y;
        }
        const bool av = asum[g].w == kWalkDone;
        for (uint32_t r = lane; r < SH; r += 32) arows[wi][r] = av ? rec[r] : make_uint2(0u, 0u);
        __syncwarp();
        uint32_t i = si, j = sj;
        const uint32_t st = walk_stripe<LY, false, true>(p, s, i, j, k, jb.lcap, mbuf + jb.moff + jb.lcap, nullptr,
                                                         arows[wi], a_from, tiles[wi]);
        if (lane == 0) {
            bsum[2 * (size_t)g] = make_uint4(si, sj, i, j);
            bsum[2 * (size_t)g + 1] = make_uint4(k, a_from, st, 0u);
        }
    }
}

// The true path, one warp per pair: links the stripes' pieces (recording
// the copies in `seg`) and walks the stripes no piece resolves, writing
// those moves in place.  Pairs without stripe jobs (job_base ~0) walk every
// stripe here.  Ends with the row-0 / column-0 moves and the move count.
template <class LY>
__global__ void __launch_bounds__(32) k_tb_stitch(TraceTask one, const TraceTask *many, const uint32_t *job_base,
                                                  const StripeJob *jobs, uint32_t njobs, uint32_t lcap,
                                                  const uint2 *rows, const uint4 *asum, const uint4 *bsum, uint4 *seg,
                                                  uint32_t *err) {
    constexpr uint32_t SH = LY::SH;
    __shared__ __align__(16) uint32_t tile[kTileLanes * kTileWords];
    __shared__ uint2 arow[SH];
    __shared__ uint4 win[32][3];  // summaries of stripes [wlo, wlo + 32)
    const TraceTask &p = many ? many[blockIdx.x] : one;
    const uint32_t lane = threadIdx.x;
    const uint32_t gb = job_base ? job_base[blockIdx.x] : (njobs ? 0u : 0xffffffffu);
    const bool par = gb != 0xffffffffu;
    const uint32_t S = LY::stripes(p);
    if (par)
        for (uint32_t s = lane; s < S; s += 32) seg[gb + s] = make_uint4(0xffffffffu, 0u, 0u, 0u);
    __syncwarp();
    uint32_t i = p.m, j = p.n, k = 0, wlo = 0xffffffffu;
    while (i > 0 && j > 0) {
        const uint32_t s = LY::stripe_of(p, i - 1);
        uint4 A = make_uint4(0u, 0u, 0u, kWalkNone), B0 = make_uint4(0u, 0u, 0u, 0u),
              B1 = make_uint4(0u, 0u, kWalkNone, 0u);
        if (par) {
            if (wlo == 0xffffffffu || s < wlo || s >= wlo + 32) {
                wlo = s >= 31 ? s - 31 : 0;
                __syncwarp();
                const uint32_t q = wlo + lane;
                if (q < S) {
                    win[lane][0] = asum[gb + q];
                    win[lane][1] = bsum[2 * (size_t)(gb + q)];
                    win[lane][2] = bsum[2 * (size_t)(gb + q) + 1];
                }
                __syncwarp();
            }
            A = win[s - wlo][0];
            B0 = win[s - wlo][1];
            B1 = win[s - wlo][2];
        }
        if (B0.x == i && B0.y == j && (B1.z == kWalkDone || B1.z == kWalkJoined)) {
            const bool joined = B1.z == kWalkJoined;
            if (lane == 0) seg[gb + s] = make_uint4(k, B1.x, joined ? B1.y : 0u, joined ? A.z - B1.y : 0u);
            k += B1.x;
            if (joined) {
                k += A.z - B1.y;
                i = A.x;
                j = A.y;
            } else {
                i = B0.z;
                j = B0.w;
            }
            continue;
        }
        const bool av = par && A.w == kWalkDone;
        const uint64_t roff = av ? job_of(jobs, gb + s, lcap, SH).roff : 0;
        __syncwarp();
        for (uint32_t r = lane; r < SH; r += 32) arow[r] = av ? rows[roff + r] : make_uint2(0u, 0u);
        __syncwarp();
        uint32_t a_from = 0;
        const uint32_t st =
            walk_stripe<LY, false, true>(p, s, i, j, k, 0xffffffffu, p.moves, nullptr, arow, a_from, tile);
        if (st == kWalkJoined) {
            if (lane == 0) seg[gb + s] = make_uint4(k, 0u, a_from, A.z - a_from);
            k += A.z - a_from;
            i = A.x;
            j = A.y;
        } else if (st != kWalkDone) {
            // the true path never leaves the stored columns of an accepted band
            if (lane == 0) raise_error(err, NW_ERR_UNSUPPORTED, 0x70000u + s);
            break;
        }
    }
    const uint32_t rest = i + j;
    const uint8_t mv = i ? 1 : 2;
    for (uint32_t q = lane; q < rest; q += 32) p.moves[(uint64_t)k + q] = mv;
    if (lane == 0) *p.nmoves = (uint64_t)k + rest;
}

// Copies of the linked pieces into the move list, one warp per stripe job.
template <class LY>
__global__ void __launch_bounds__(kWalkWarps * 32) k_tb_copy(TraceTask one, const TraceTask *many,
                                                             const StripeJob *jobs, uint32_t njobs, uint32_t lcap,
                                                             const uint8_t *mbuf, const uint4 *seg) {
    constexpr uint32_t SH = LY::SH;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t g = blockIdx.x * kWalkWarps + (threadIdx.x >> 5);
    if (g >= njobs) return;
    const uint4 sg = seg[g];
    if (sg.x == 0xffffffffu) return;
    const StripeJob jb = job_of(jobs, g, lcap, SH);
    const TraceTask &p = many ? many[jb.task] : one;
    uint8_t *dst = p.moves + sg.x;
    const uint8_t *spec = mbuf + jb.moff, *link = spec + jb.lcap;
    for (uint32_t q = lane; q < sg.y; q += 32) dst[q] = link[q];
    for (uint32_t q = lane; q < sg.w; q += 32) dst[sg.y + q] = spec[sg.z + q];
}

// ------------------------------------------------------------------ finish
// Reverses the move list, resolves diagonal moves into '=' / 'X' (or 'M'),
// and run-length encodes.  One CTA of 1024 threads loops over chunks of 4096
// moves; three block scans per chunk give each move its (i,j), each run its
// start and each run string its output offset.
constexpr int kFinThreads = 1024, kFinPer = 4;

template <typename T, typename Op>
__device__ __forceinline__ T block_exscan(T v, Op op, T ident, T *warp_tot, T &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl = op(y, incl);
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T w = warp_tot[lane];
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi = op(y, wi);
        }
        warp_tot[lane] = wi;  // inclusive over warps
    }
    __syncthreads();
    T before = wid ? warp_tot[wid - 1] : ident;
    T ex = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) ex = ident;
    T res = op(before, ex);
    total = warp_tot[31];
    __syncthreads();
    return res;
}


__device__ __forceinline__ uint32_t ndigits(uint64_t v) {
    uint32_t d = 1;
    while (v >= 10) {
        v /= 10;
        ++d;
    }
    return d;
}

__global__ void __launch_bounds__(kFinThreads) k_finish(TraceTask one, const TraceTask *many, uint32_t mflag) {
    const TraceTask &p = many ? many[blockIdx.x] : one;
    __shared__ unsigned long long sc_u64[32];
    __shared__ long long sc_i64[32];
    __shared__ char first_op[kFinThreads + 1];
    const uint64_t L = *p.nmoves;
    const int tid = threadIdx.x;
    // bases of A / B consumed before this chunk (from the start cell)
    uint64_t ci = p.origin ? p.origin[0] : 0u, cj = p.origin ? p.origin[1] : 0u;
    long long last_end = -1;   // forward position of the last run end so far
    uint64_t out = 0;          // chars written so far
    const uint64_t CH = (uint64_t)kFinThreads * kFinPer;
    for (uint64_t base = 0; base < L; base += CH) {
        const uint64_t p0 = base + (uint64_t)tid * kFinPer;
        uint8_t mv[kFinPer];
        uint32_t cnt_i = 0, cnt_j = 0;
#pragma unroll
        for (int e = 0; e < kFinPer; ++e) {
            const uint64_t q = p0 + e;
            mv[e] = q < L ? p.moves[L - 1 - q] : 3;
            cnt_i += (mv[e] == 0 || mv[e] == 1);
            cnt_j += (mv[e] == 0 || mv[e] == 2);
        }
        unsigned long long tot;
        const unsigned long long packed = ((unsigned long long)cnt_i << 32) | cnt_j;
        const unsigned long long ex = block_exscan<unsigned long long>(
            packed, [](unsigned long long x, unsigned long long y) { return x + y; }, 0ull, sc_u64, tot);
        uint64_t pi = ci + (ex >> 32), pj = cj + (ex & 0xffffffffull);
        char op[kFinPer];
#pragma unroll
        for (int e = 0; e < kFinPer; ++e) {
            char o = 0;
            if (mv[e] == 0) {
                o = mflag ? 'M' : (base_at(p.a, pi) == base_at(p.b, pj) ? '=' : 'X');
                ++pi;
                ++pj;
            } else if (mv[e] == 1) {
                o = 'I';
                ++pi;
            } else if (mv[e] == 2) {
                o = 'D';
                ++pj;
            }
            op[e] = o;
        }
        first_op[tid] = op[0];
        if (tid == kFinThreads - 1) {
            // first op of the next chunk (its position is this chunk's end)
            const uint64_t q = base + CH;
            char o = 0;
            if (q < L) {
                const uint8_t m2 = p.moves[L - 1 - q];
                if (m2 == 0)
                    o = mflag ? 'M' : (base_at(p.a, pi) == base_at(p.b, pj) ? '=' : 'X');
                else
                    o = m2 == 1 ? 'I' : 'D';
            }
            first_op[kFinThreads] = o;
        }
        __syncthreads();
        const char next_after = first_op[tid + 1];
        bool is_end[kFinPer];
        long long my_last = -1;
#pragma unroll
        for (int e = 0; e < kFinPer; ++e) {
            const uint64_t q = p0 + e;
            const char nx = e + 1 < kFinPer ? op[e + 1] : next_after;
            is_end[e] = q < L && (q + 1 == L || nx != op[e]);
            if (is_end[e]) my_last = (long long)q;
        }
        long long tot_max;
        const long long prev_excl =
            block_exscan<long long>(my_last, [](long long x, long long y) { return x > y ? x : y; }, -1ll, sc_i64, tot_max);
        long long prev = prev_excl > last_end ? prev_excl : last_end;
        uint32_t chars = 0;
        long long pe = prev;
#pragma unroll
        for (int e = 0; e < kFinPer; ++e)
            if (is_end[e]) {
                chars += ndigits((uint64_t)((long long)(p0 + e) - pe)) + 1;
                pe = (long long)(p0 + e);
            }
        unsigned long long tot_chars;
        const unsigned long long off = block_exscan<unsigned long long>(
            chars, [](unsigned long long x, unsigned long long y) { return x + y; }, 0ull, sc_u64, tot_chars);
        uint64_t w = out + off;
        pe = prev;
#pragma unroll
        for (int e = 0; e < kFinPer; ++e)
            if (is_end[e]) {
                uint64_t len = (uint64_t)((long long)(p0 + e) - pe);
                const uint32_t nd = ndigits(len);
                for (uint32_t d = nd; d-- > 0;) {
                    p.cigar[w + d] = (char)('0' + len % 10);
                    len /= 10;
                }
                p.cigar[w + nd] = op[e];
                w += nd + 1;
                pe = (long long)(p0 + e);
            }
        ci += tot >> 32;
        cj += tot & 0xffffffffull;
        if (tot_max > last_end) last_end = tot_max;
        out += tot_chars;
        __syncthreads();
    }
    if (tid == 0) {
        p.cigar[out] = 0;
        *p.cigar_len = out;
    }
}


template <int R>
static void launch_tb(nw_ctx *ctx, const TraceTask &one, const TraceTask *many, uint32_t ntasks) {
    k_traceback<R><<<ntasks, 32, 0, ctx->stream>>>(one, many);
}

int launch_traceback(nw_ctx *ctx, int R, const TraceTask &one, const TraceTask *many, uint32_t ntasks) {
    if (ntasks == 0) return NW_OK;
    {
        LaunchTimer t(ctx, "traceback");
        switch (R) {
            case 2: launch_tb<2>(ctx, one, many, ntasks); break;
            case 4: launch_tb<4>(ctx, one, many, ntasks); break;
            case 8: launch_tb<8>(ctx, one, many, ntasks); break;
            case 16: launch_tb<16>(ctx, one, many, ntasks); break;
            default: return fail(ctx, NW_ERR_ARG, "unsupported rows per lane %d", R);
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "traceback launch");
}

int launch_finish(nw_ctx *ctx, const TraceTask &one, const TraceTask *many, uint32_t ntasks, uint32_t mflag) {
    if (ntasks == 0) return NW_OK;
    {
        LaunchTimer t(ctx, "finish");
        k_finish<<<ntasks, kFinThreads, 0, ctx->stream>>>(one, many, mflag);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "CIGAR launch");
}

// Stripe jobs of the pairs with at least kParMinStripes stripes, scratch
// for their walks, and the four walk kernels.
template <class LY>
static int launch_walks(nw_ctx *ctx, const TraceTask *host, const TraceTask *dev, uint32_t ntasks) {
    constexpr uint32_t SH = LY::SH;
    HostTimer ht(ctx, "trace_plan");
    static const char *min_env = getenv("NW_TB_MIN_MOVES");  // sweep knob
    const uint64_t min_moves = min_env ? (uint64_t)atoll(min_env) : ntasks == 1 ? kParMinMovesOne : kParMinMoves;
    const TraceTask one = dev ? TraceTask{} : host[0];
    std::vector<StripeJob> jobs;
    std::vector<uint32_t> base(ntasks, 0xffffffffu);
    uint64_t moff = 0, roff = 0;
    for (uint32_t t = 0; t < ntasks; ++t) {
        const uint64_t m = host[t].m, n = host[t].n;
        if (m == 0 || n == 0 || host[t].state) continue;
        const uint32_t S = (uint32_t)((m + SH - 1) / SH);
        if (S < kParMinStripes || m + n < min_moves) continue;
        // moves of a stripe's walks: its rows, twice the proportional columns, slack
        uint64_t cap = SH + 2 * ((SH * n + m - 1) / m) + 512;
        cap = std::min<uint64_t>((cap + 15) / 16 * 16, 65520);
        base[t] = (uint32_t)jobs.size();
        for (uint32_t s = 0; s < S; ++s) {
            jobs.push_back(StripeJob{moff, roff, t, s, (uint32_t)cap, 0u});
            moff += 2 * cap;
            roff += SH;
        }
    }
    uint32_t njobs = (uint32_t)jobs.size();
    const uint64_t need = moff + roff * 8 + (uint64_t)njobs * (16 + 32 + 16 + sizeof(StripeJob)) + 4u * ntasks + 4096;
    const auto it = ctx->bufs.find("tb_moves");
    const uint64_t have = it == ctx->bufs.end() ? 0 : it->second.cap;
    if (njobs && ctx->used - std::min(ctx->used, have) + need > ctx->budget) {
        njobs = 0;  // not enough scratch: every pair walks sequentially
        std::fill(base.begin(), base.end(), 0xffffffffu);
    }
    int rc;
    void *vm = nullptr, *vr = nullptr, *va = nullptr, *vb = nullptr, *vs = nullptr, *vj = nullptr, *vbase = nullptr;
    if (njobs) {
        if ((rc = scratch(ctx, "tb_moves", moff, &vm))) return rc;
        if ((rc = scratch(ctx, "tb_rows", roff * 8, &vr))) return rc;
        if ((rc = scratch(ctx, "tb_asum", (size_t)njobs * 16, &va))) return rc;
        if ((rc = scratch(ctx, "tb_bsum", (size_t)njobs * 32, &vb))) return rc;
        if ((rc = scratch(ctx, "tb_seg", (size_t)njobs * 16, &vs))) return rc;
    }
    // one pair: the jobs are implicit (stripe s = job s); else upload them
    const bool implicit = !dev;
    const uint32_t lcap = njobs ? jobs[0].lcap : 0u;
    if (!implicit) {
        if ((rc = scratch(ctx, "tb_base", (size_t)ntasks * 4, &vbase))) return rc;
        cudaError_t e = cudaMemcpyAsync(vbase, base.data(), (size_t)ntasks * 4, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess && njobs) {
            if ((rc = scratch(ctx, "tb_jobs", (size_t)njobs * sizeof(StripeJob), &vj))) return rc;
            e = cudaMemcpyAsync(vj, jobs.data(), (size_t)njobs * sizeof(StripeJob), cudaMemcpyHostToDevice,
                                ctx->stream);
        }
        // the host vectors die on return: wait for the copies
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "stripe job upload");
    }
    const StripeJob *dj = (const StripeJob *)vj;
    const uint32_t blocks = (njobs + kWalkWarps - 1) / kWalkWarps;
    if (njobs) {
        {
            LaunchTimer t(ctx, "tb_spec");
            k_tb_stripes<LY, false><<<blocks, kWalkWarps * 32, 0, ctx->stream>>>(
                one, dev, dj, njobs, lcap, (uint8_t *)vm, (uint2 *)vr, (uint4 *)va, (uint4 *)vb);
        }
        {
            LaunchTimer t(ctx, "tb_link");
            k_tb_stripes<LY, true><<<blocks, kWalkWarps * 32, 0, ctx->stream>>>(
                one, dev, dj, njobs, lcap, (uint8_t *)vm, (uint2 *)vr, (uint4 *)va, (uint4 *)vb);
        }
    }
    {
        LaunchTimer t(ctx, "tb_stitch");
        k_tb_stitch<LY><<<ntasks, 32, 0, ctx->stream>>>(one, dev, (const uint32_t *)vbase, dj, njobs, lcap,
                                                       (const uint2 *)vr, (const uint4 *)va, (const uint4 *)vb,
                                                       (uint4 *)vs, ctx->d_err);
    }
    if (njobs) {
        LaunchTimer t(ctx, "tb_copy");
        k_tb_copy<LY><<<blocks, kWalkWarps * 32, 0, ctx->stream>>>(one, dev, dj, njobs, lcap, (const uint8_t *)vm,
                                                                  (const uint4 *)vs);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "traceback launch");
}

int launch_trace(nw_ctx *ctx, int R, const TraceTask *host, const TraceTask *dev, uint32_t ntasks, uint32_t mflag) {
    if (ntasks == 0) return NW_OK;
    int rc;
    switch (R) {
        case 2: rc = launch_walks<ScalarLayout<2>>(ctx, host, dev, ntasks); break;
        case 4: rc = launch_walks<ScalarLayout<4>>(ctx, host, dev, ntasks); break;
        case 8: rc = launch_walks<ScalarLayout<8>>(ctx, host, dev, ntasks); break;
        case 16: rc = launch_walks<ScalarLayout<16>>(ctx, host, dev, ntasks); break;
        default: return fail(ctx, NW_ERR_ARG, "unsupported rows per lane %d", R);
    }
    return rc ? rc : launch_finish(ctx, host[0], dev, ntasks, mflag);
}

int launch_trace_bits(nw_ctx *ctx, const TraceTask *host, const TraceTask *dev, uint32_t ntasks, uint32_t mflag) {
    if (ntasks == 0) return NW_OK;
    const int rc = launch_walks<BitsLayout<kBitsWalkGroup>>(ctx, host, dev, ntasks);
    return rc ? rc : launch_finish(ctx, host[0], dev, ntasks, mflag);
}

}  // namespace nw
