// Bit-sliced certified band (a8) with pointers (a4) and its walk (a5).
//
// The fill is the difference form of nw_bits.cu (dH, dV in two bit planes,
// T = max(s', a, b), dV = T - a, dH = T - b) on a window that follows the
// band: on anti-diagonal a the window holds the Hw = 32*g*Q rows
// r0(a) .. r0(a)+Hw-1 with r0(a) = floor((a - hi)/2), so it moves down one
// row every second anti-diagonal and always covers the band's diagonals
// [lo, hi] (2*Hw >= hi - lo + 4).  A pair belongs to a group of g lanes
// (1..32, a power of two) holding Q words each; window bit P = 32*(lane*Q +
// word) + bit is row r0(a) + P, column a - r0(a) - P.
//
// Anti-diagonals come in pairs: a step where r0 stays (the B bases slide one
// bit up, a new column enters at the top; the cell above a bit is the bit
// below it on the previous anti-diagonal, the cell to its left the same bit)
// and a step where r0 grows (the A bases slide one bit down, a new row
// enters at the bottom; the cell above is the same bit, the cell to the left
// the bit above).  Shifts across words go through funnel shifts, across
// lanes of a group through warp shuffles.  Cells just outside the window
// take the values of a gap move from a computed neighbour, which a real
// path reaches: above the top row a horizontal extension (dH = 0), below
// the bottom row a vertical one (dV = 0).  Every computed value is therefore
// reached by some path (never above the full grid's value) and at least the
// value of the DP restricted to the window, which contains the band -- so the
// certificate of the scalar banded kernels holds unchanged: a score above
// the exit bound U0 of the band equals the full score, and the walk below
// gives the full grid's alignment.  Cells of row 0 or column 0 and beyond
// (the grid's boundary) get s' = 0 through a mask in the ramp chunks, which
// keeps their differences at 0.
//
// The score is tracked at the window's top cell (its dH on a step without a
// shift, its dV on a shift) and carried down the last anti-diagonal to
// (m, n).  Pointer bits, per cell: L = T != s' (the diagonal loses), and
// Hb = dV != 0 (the vertical move loses); the walk reads !L -> diagonal,
// else !Hb -> vertical, else horizontal, the diagonal > vertical > horizontal
// order of the scalar kernels.  One 16-byte record per word and pair of
// anti-diagonals: (L, Hb) of the first, (L, Hb) of the second.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "nw_bits.cuh"
#include "nw_order.h"

namespace nw {

// Words per lane: at most 4, so a pair's window holds up to 128 words (4,096
// rows, bands up to ~8,190 diagonals).  Up to 8 words per lane (fewer lanes
// per pair, the lane's fixed work per step shared by more words) measured
// 1.5x slower on the band workload: 27.3 against 18.0 ms per fill.
constexpr int kBandBitsMaxQ = 4;
constexpr int kBandBitsMaxWords = 32 * kBandBitsMaxQ;
constexpr int kWalkWarps = 4;
// Warps per CTA of the fill: at ~150 registers an SM holds 13 warps, so
// CTAs of 4 warps fit 12 of them (CTAs of 8 only 8).
constexpr int kBandWarps = 4;

struct BandBitsTask {
    int64_t a_slot, b_slot; // planar slots of A (rows) and B (columns)
    uint64_t ptr_off;       // first pointer record of the pair (16-byte units)
    uint32_t m, n;
    int32_t hi;             // window anchor: the band's upper diagonal, raised to the parity of m+n
    int32_t a_first;        // first anti-diagonal (a step without a shift), <= 0
    uint32_t nchunks;       // chunks of 64 anti-diagonals; the last ends at m+n
    uint32_t out0;          // the caller's score slot
};

struct BandBitsJob {
    uint32_t t0, cnt;  // tasks [t0, t0 + cnt), one per group of g lanes
    uint32_t g, Q;     // lanes per pair, words per lane
    uint32_t nchunks;  // the job's largest
};

struct BandBitsArgs {
    const uint32_t *pl0, *pl1;
    int64_t max_base;  // largest global base index a window load may start at
    const BandBitsTask *tasks;
    const BandBitsJob *jobs;
    uint32_t njobs;
    uint32_t *counter;
    uint4 *ptr;
    uint64_t ptr_cap;   // records at ptr (checked build)
    int32_t *scores;
    int32_t *gathered;  // per task, in task order
    uint32_t score_cap;
    int32_t gap;
    uint32_t *err;
};

// Bits b of a word with lo <= b <= hi (empty when hi < lo); PTX shifts
// clamp at the register width.
__device__ __forceinline__ uint32_t range_mask(int32_t lo, int32_t hi) {
    uint32_t a, b;
    asm("shl.b32 %0, %1, %2;" : "=r"(a) : "r"(~0u), "r"((uint32_t)max(lo, 0)));
    asm("shl.b32 %0, %1, %2;" : "=r"(b) : "r"(~0u), "r"((uint32_t)max(hi + 1, 0)));
    return a & ~b;
}

// The cells of one word: inputs a (dH above), b (dV to the left), bases A,
// B, mask mk of cells inside the grid (others get s' = 0); outputs the new
// planes and the pointer bits.  The paper's scoring: s' = 3 (match) or 1.
__device__ __forceinline__ void band_cell(uint32_t A0, uint32_t A1, uint32_t B0, uint32_t B1, uint32_t a0,
                                          uint32_t a1, uint32_t b0, uint32_t b1, uint32_t mk, uint32_t &H0,
                                          uint32_t &H1, uint32_t &V0, uint32_t &V1, uint32_t &L, uint32_t &Hb) {
    const uint32_t x = lop3<kLutXorOrNotC>(A1, B1, mk);
    const uint32_t eq = lop3<kLutEq>(A0, B0, x);
    const uint32_t p = lop3<kLutAndOrNot>(a0, a1, b1);
    const uint32_t q = lop3<kLutAndOrNot>(b0, b1, a1);
    const uint32_t v = lop3<kLutCOrNor>(a1, b1, eq);
    const uint32_t T0 = p | lop3<kLutOrAnd>(q, v, mk);
    const uint32_t T1 = lop3<kLutOr3>(a1, b1, eq);
    const uint32_t ca = lop3<kLutAndNot>(a0, T0, 0u), cb = lop3<kLutAndNot>(b0, T0, 0u);
    V0 = T0 ^ a0;
    V1 = lop3<kLutXor3>(T1, a1, ca);
    H0 = T0 ^ b0;
    H1 = lop3<kLutXor3>(T1, b1, cb);
    L = lop3<kLutXorOrNotC>(T1, eq, T0);  // (T1 ^ eq) | ~T0: T differs from s' = (eq, 1)
    Hb = V0 | V1;
}

template <int Q, bool PTR>
__device__ __forceinline__ void band_job(const BandBitsArgs &p, const BandBitsJob &job, uint32_t lane) {
    const uint32_t g = job.g;
    const uint32_t gl = lane & (g - 1), grp = lane / g;
    const bool active = grp < job.cnt;
    const uint32_t tid = job.t0 + (active ? grp : 0u);
    const BandBitsTask t = p.tasks[tid];
    const int32_t gq = (int32_t)g * Q, Hw = 32 * gq;
    const int32_t a0 = t.a_first;
    const int32_t R = (a0 - t.hi - 1) >> 1;  // r0(a_first); a_first - hi is odd
    const int64_t Ag = t.a_slot, Bg = t.b_slot;
    auto ld = [&](const uint32_t *pl, int64_t gidx) {
        return plane_window(pl, min(max(gidx, -kPlanePad), p.max_base));  // outside: bases of no cell that matters
    };
    uint32_t A0[Q], A1[Q], B0[Q], B1[Q], H0[Q], H1[Q], V0[Q], V1[Q], Ln[Q], Hn[Q];
#pragma unroll
    for (int v = 0; v < Q; ++v) {
        const int32_t W = (int32_t)gl * Q + v;
        const int64_t ra = Ag + R + 32 * W - 1;                  // A index of the row of bit 0
        A0[v] = ld(p.pl0, ra);
        A1[v] = ld(p.pl1, ra);
        const int64_t cb = Bg + (a0 - 1 - R - 32 * W - 31) - 1;  // B index of the column of bit 31
        B0[v] = __brev(ld(p.pl0, cb));
        B1[v] = __brev(ld(p.pl1, cb));
        H0[v] = H1[v] = V0[v] = V1[v] = 0;
    }
    int32_t top = 0;  // W of the window's top cell
    const uint32_t nch = t.nchunks;
    const uint32_t gmask = g == 32 ? kFull : (((1u << g) - 1u) << (grp * g));
    for (uint32_t c = 0; c < job.nchunks; ++c) {
        const bool live = active && c < nch;
        const int32_t rc = R + 32 * (int32_t)c, ac = a0 + 64 * (int32_t)c;  // r0 and a of the chunk's first step
        // new columns (top, one per step without a shift) and rows (bottom, one per shift) of the chunk
        const int64_t fb = Bg + (ac - rc) - 1, fa = Ag + rc + Hw - 1;
        uint32_t fB0 = __brev(ld(p.pl0, fb)), fB1 = __brev(ld(p.pl1, fb));
        uint32_t fA0 = ld(p.pl0, fa), fA1 = ld(p.pl1, fa);
        // masks only while some cell of the chunk lies on or beyond row 0 / column 0
        const bool ramp = __any_sync(kFull, live && !(rc >= 1 && ac - rc - Hw >= 0));
        uint32_t cH0 = 0, cH1 = 0, cV0 = 0, cV1 = 0;
        for (int32_t d = 0; d < 32; ++d) {
            // ---- no shift: anti-diagonal ac + 2d, top row rc + d
            {
                uint32_t sB0 = __shfl_up_sync(kFull, B0[Q - 1], 1, g), sB1 = __shfl_up_sync(kFull, B1[Q - 1], 1, g);
                uint32_t sH0 = __shfl_up_sync(kFull, H0[Q - 1], 1, g), sH1 = __shfl_up_sync(kFull, H1[Q - 1], 1, g);
                if (gl == 0) {
                    sB0 = fB0;
                    sB1 = fB1;
                    sH0 = 0u;  // above the window: a horizontal gap, dH = 0
                    sH1 = 0u;
                }
                fB0 <<= 1;
                fB1 <<= 1;
                // (these one-bit shifts as multiply-adds, on the other pipe,
                // measured slower: 20.2 against 18.8 ms per fill)
#pragma unroll
                for (int v = Q - 1; v >= 0; --v) {
                    const int32_t W = (int32_t)gl * Q + v;
                    B0[v] = __funnelshift_l(v ? B0[v - 1] : sB0, B0[v], 1);
                    B1[v] = __funnelshift_l(v ? B1[v - 1] : sB1, B1[v], 1);
                    const uint32_t a0v = __funnelshift_l(v ? H0[v - 1] : sH0, H0[v], 1);
                    const uint32_t a1v = __funnelshift_l(v ? H1[v - 1] : sH1, H1[v], 1);
                    const uint32_t mk = ramp ? range_mask(1 - rc - d - 32 * W, ac - rc + d - 32 * W - 1) : ~0u;
                    band_cell(A0[v], A1[v], B0[v], B1[v], a0v, a1v, V0[v], V1[v], mk, H0[v], H1[v], V0[v], V1[v],
                              Ln[v], Hn[v]);
                }
                cH0 = __funnelshift_r(cH0, H0[0], 1);
                cH1 = __funnelshift_r(cH1, H1[0], 1);
            }
            // ---- shift: anti-diagonal ac + 2d + 1, top row rc + d + 1
            {
                uint32_t sA0 = __shfl_down_sync(kFull, A0[0], 1, g), sA1 = __shfl_down_sync(kFull, A1[0], 1, g);
                uint32_t sV0 = __shfl_down_sync(kFull, V0[0], 1, g), sV1 = __shfl_down_sync(kFull, V1[0], 1, g);
                if (gl == g - 1) {
                    sA0 = fA0;
                    sA1 = fA1;
                    sV0 = 0u;  // below the window: a vertical gap, dV = 0
                    sV1 = 0u;
                }
                fA0 >>= 1;
                fA1 >>= 1;
#pragma unroll
                for (int v = 0; v < Q; ++v) {
                    const int32_t W = (int32_t)gl * Q + v;
                    A0[v] = __funnelshift_r(A0[v], v + 1 < Q ? A0[v + 1] : sA0, 1);
                    A1[v] = __funnelshift_r(A1[v], v + 1 < Q ? A1[v + 1] : sA1, 1);
                    const uint32_t b0v = __funnelshift_r(V0[v], v + 1 < Q ? V0[v + 1] : sV0, 1);
                    const uint32_t b1v = __funnelshift_r(V1[v], v + 1 < Q ? V1[v + 1] : sV1, 1);
                    const uint32_t mk = ramp ? range_mask(-rc - d - 32 * W, ac - rc + d - 32 * W - 1) : ~0u;
                    uint32_t Ls, Hs;
                    band_cell(A0[v], A1[v], B0[v], B1[v], H0[v], H1[v], b0v, b1v, mk, H0[v], H1[v], V0[v], V1[v], Ls,
                              Hs);
                    if (PTR && live) {
                        const uint64_t idx = t.ptr_off + (uint64_t)(32u * c + (uint32_t)d) * (uint32_t)gq + (uint32_t)W;
                        if (in_range(idx, p.ptr_cap, p.err, kSiteBandBitsPtr)) __stcg(p.ptr + idx, make_uint4(Ln[v], Hn[v], Ls, Hs));
                    }
                }
                cV0 = __funnelshift_r(cV0, V0[0], 1);
                cV1 = __funnelshift_r(cV1, V1[0], 1);
            }
        }
        top += __popc(cH0) + 2 * __popc(cH1) + __popc(cV0) + 2 * __popc(cV1);
        if (active && c + 1 == nch) {
            // W(m, n): the top cell, then down the last anti-diagonal: each row
            // adds its cell's dV and takes off the dH of the cell above it
            const int32_t Pm = (int32_t)t.m - (R + 32 * (int32_t)nch);
            int32_t sum = 0;
#pragma unroll
            for (int v = 0; v < Q; ++v) {
                const int32_t W = (int32_t)gl * Q + v;
                const uint32_t vm = range_mask(1 - 32 * W, Pm - 32 * W), hm = range_mask(-32 * W, Pm - 1 - 32 * W);
                sum += __popc(V0[v] & vm) + 2 * __popc(V1[v] & vm) - __popc(H0[v] & hm) - 2 * __popc(H1[v] & hm);
            }
            for (uint32_t o = 1; o < g; o <<= 1) sum += __shfl_xor_sync(gmask, sum, o);
            if (gl == 0) {
                const int32_t sc = top + sum + p.gap * (int32_t)(t.m + t.n);
                if (in_range(t.out0, p.score_cap, p.err, kSiteBatchScore)) p.scores[t.out0] = sc;
                p.gathered[tid] = sc;
            }
        }
    }
}

template <bool PTR>
__global__ void __launch_bounds__(kBandWarps * 32) k_bits_band(BandBitsArgs p) {
    const uint32_t lane = threadIdx.x & 31u;
    for (;;) {
        uint32_t jid = 0;
        if (lane == 0) jid = atomicAdd(p.counter, 1u);
        jid = __shfl_sync(kFull, jid, 0);
        if (jid >= p.njobs) break;
        const BandBitsJob job = p.jobs[jid];
        switch (job.Q) {
            case 1: band_job<1, PTR>(p, job, lane); break;
            case 2: band_job<2, PTR>(p, job, lane); break;
            case 3: band_job<3, PTR>(p, job, lane); break;
            default: band_job<4, PTR>(p, job, lane); break;
        }
    }
}

// ---------------------------------------------------------------- the walk
struct BitsWalkTask {
    uint64_t ptr_off;    // the pair's first record
    uint64_t moves_off;  // its move bytes
    uint32_t m, n, gq;
    int32_t hi, a_first;
    uint32_t slot;       // its move count slot
};

// One warp per pair: it stages 32 records (64 anti-diagonals) of the three
// words around the walk's position into shared memory, then walks from
// (m, n) while the cells stay inside them; moves are written in walk order
// (0 diagonal, 1 vertical, 2 horizontal), as the CIGAR assembly reads.
// While the warp walks one block, the loads of the 32 records before it (the
// same words) are in flight; they fill the second buffer, which the walk
// continues in unless it left those words (then a new block is staged).
//
// RUNS: the whole warp walks, a run of diagonal moves at a time.  A
// diagonal move keeps the cell's row in the window (same word and bit) and
// goes one record row down, so lane t reads the cell t diagonal moves on;
// a ballot of their L bits gives the run's length (its first lane whose
// diagonal loses), the run's zero bytes are one store, and the cell that
// ends it gives the vertical or horizontal move by its Hb bit.  Otherwise
// lane 0 walks one move at a time.
template <bool RUNS>
__global__ void __launch_bounds__(kWalkWarps * 32) k_bits_walk(const uint4 *ptr, const BitsWalkTask *tasks,
                                                               uint32_t ntasks, uint8_t *moves, uint64_t *nmoves,
                                                               uint32_t *err) {
    __shared__ uint4 tile[kWalkWarps][2][32][3];
    const uint32_t lane = threadIdx.x & 31u, wb = threadIdx.x >> 5;
    const uint32_t nw = gridDim.x * kWalkWarps;
    for (uint32_t ti = blockIdx.x * kWalkWarps + wb; ti < ntasks; ti += nw) {
        const BitsWalkTask tk = tasks[ti];
        const uint4 *pp = ptr + tk.ptr_off;
        uint8_t *mv = moves + tk.moves_off;
        int32_t i = (int32_t)tk.m, j = (int32_t)tk.n;
        uint64_t k = 0;
        const int32_t gq = (int32_t)tk.gq;
        bool ok = true, have = false;
        int32_t ds_lo = 0, w_lo = 0, cur = 0;
        while (ok && i > 0 && j > 0) {
            const int32_t a = i + j, ds = (a - tk.a_first) >> 1;
            const int32_t W = (i - ((a - tk.hi) >> 1)) >> 5;
            bool staged = false;
            if (!have || ds < ds_lo || ds > ds_lo + 31 || W < w_lo || W > w_lo + 2) {
                // the 32 records ending at the walk's position, staged now
                ds_lo = max(ds - 31, 0);
                w_lo = max(min(W - 1, gq - 3), 0);
                __syncwarp();
                if (ds_lo + (int32_t)lane <= ds) {
#pragma unroll
                    for (int x = 0; x < 3; ++x)
                        if (w_lo + x < gq)
                            tile[wb][cur][lane][x] = __ldcg(pp + (uint64_t)(ds_lo + (int32_t)lane) * gq + w_lo + x);
                }
                __syncwarp();
                have = staged = true;
            }
            // the 32 records before the block: loads issued now, stored after the walk
            const int32_t nds = ds_lo - 32, rec = nds + (int32_t)lane;
            uint4 r[3];
#pragma unroll
            for (int x = 0; x < 3; ++x)
                r[x] = (rec >= 0 && w_lo + x < gq) ? __ldcg(pp + (uint64_t)rec * gq + w_lo + x) : make_uint4(0, 0, 0, 0);
            if (RUNS) {
                // every pass makes a move or leaves the loop: at most m + n passes
                const uint64_t k0 = k;
                while (i > 0 && j > 0) {
                    const int32_t a2 = i + j, rel = a2 - tk.a_first, x = (rel >> 1) - ds_lo, par = rel & 1;
                    const int32_t P = i - ((a2 - tk.hi) >> 1), W2 = P >> 5, y = W2 - w_lo;
                    if (x < 0 || x > 31 || y < 0 || y > 2 || W2 >= gq || P < 0) break;
                    const uint32_t bit = (uint32_t)P & 31u;
                    // lane t: the cell t diagonal moves on (record row x - t, same word and bit);
                    // rows outside the block count as ending the run
                    const int32_t xr = x - (int32_t)lane;
                    uint32_t Lw = ~0u, Hw = 0u;
                    if (xr >= 0 && ds_lo + xr >= 0) {
                        const uint4 rc = tile[wb][cur][xr][y];
                        Lw = par ? rc.z : rc.x;
                        Hw = par ? rc.w : rc.y;
                    }
                    const uint32_t stop = __ballot_sync(kFull, (Lw >> bit) & 1u);
                    const int32_t f = stop ? __ffs(stop) - 1 : 32;
                    const int32_t run = min(f, min(i, j));
                    if ((int32_t)lane < run) mv[k + lane] = 0;
                    k += (uint64_t)run;
                    i -= run;
                    j -= run;
                    const uint32_t hb = __shfl_sync(kFull, (Hw >> bit) & 1u, f & 31);
                    if (run == f && f < 32 && x - f >= 0 && ds_lo + x - f >= 0 && i > 0 && j > 0) {
                        const uint32_t mvc = hb ? 2u : 1u;
                        if (lane == 0) mv[k] = (uint8_t)mvc;
                        ++k;
                        i -= mvc == 1u;
                        j -= mvc == 2u;
                    } else if (run == 0) {
                        break;
                    }
                }
                // a block staged at the walk's own cell: no progress means the
                // walk left the window, which a certified band excludes
                if (staged && k == k0) {
                    if (lane == 0) raise_error(err, NW_ERR_ARG, 0x50000u + ti);
                    ok = false;
                }
            } else if (lane == 0) {
                uint32_t steps = 0;
                while (i > 0 && j > 0) {
                    const int32_t a2 = i + j, rel = a2 - tk.a_first, d2 = rel >> 1;
                    const int32_t P = i - ((a2 - tk.hi) >> 1), W2 = P >> 5;
                    if (d2 < ds_lo || d2 > ds_lo + 31 || W2 < w_lo || W2 > w_lo + 2 || W2 >= gq || P < 0) break;
                    const uint4 rc = tile[wb][cur][d2 - ds_lo][W2 - w_lo];
                    const uint32_t bit = (uint32_t)P & 31u;
                    const uint32_t L = (rel & 1) ? rc.z : rc.x, Hb = (rel & 1) ? rc.w : rc.y;
                    const uint32_t mvc = !((L >> bit) & 1u) ? 0u : !((Hb >> bit) & 1u) ? 1u : 2u;
                    mv[k++] = (uint8_t)mvc;
                    i -= mvc != 2u;
                    j -= mvc != 1u;
                    ++steps;
                }
                // a block staged at the walk's own cell: no progress means the
                // walk left the window, which a certified band excludes
                if (staged && steps == 0) {
                    raise_error(err, NW_ERR_ARG, 0x50000u + ti);
                    ok = false;
                }
            }
            i = __shfl_sync(kFull, i, 0);
            j = __shfl_sync(kFull, j, 0);
            k = __shfl_sync(kFull, k, 0);
            ok = __shfl_sync(kFull, ok, 0);
            if (nds + 31 >= 0) {
                // the prefetched block becomes the current one
                __syncwarp();
                if (rec >= 0) {
#pragma unroll
                    for (int x = 0; x < 3; ++x) tile[wb][cur ^ 1][lane][x] = r[x];
                }
                __syncwarp();
                cur ^= 1;
                ds_lo = nds;
            } else {
                have = false;
            }
        }
        const uint32_t rest = (uint32_t)(max(i, 0) + max(j, 0));
        const uint8_t mvr = i > 0 ? 1 : 2;
        for (uint32_t q = lane; q < rest; q += 32) mv[k + q] = mvr;
        if (lane == 0) nmoves[tk.slot] = k + rest;
    }
}

// ------------------------------------------------------------------ host
static uint32_t next_pow2(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

int band_bits_max_q() {
    const char *e = getenv("NW_BBAND_MAXQ");
    const int q = e ? atoi(e) : 0;
    return q >= 1 && q <= kBandBitsMaxQ ? q : kBandBitsMaxQ;
}

bool band_bits_shape(uint32_t m, uint32_t n, int32_t lo, int32_t hi, BandBitsShape *s, int max_q) {
    const int32_t hip = hi + (int32_t)(((int64_t)m + n - hi) & 1);
    const int64_t words = ((int64_t)hip - lo + 4 + 63) / 64;
    if (words > kBandBitsMaxWords) return false;
    // throughput shape: the fewest lanes with at most max_q words each (a
    // lane's fixed work per step is shared by more words)
    max_q = std::min(std::max(max_q, 1), kBandBitsMaxQ);
    s->g = std::min<uint32_t>(32, next_pow2((uint32_t)((words + max_q - 1) / max_q)));
    s->Q = (uint32_t)((words + s->g - 1) / s->g);
    s->words = (uint32_t)words;
    s->hi = hip;
    s->nchunks = (uint32_t)(((uint64_t)m + n + 1 + 63) / 64);
    s->a_first = (int32_t)((int64_t)m + n + 1 - 64 * (int64_t)s->nchunks);
    return true;
}

void band_bits_fast(BandBitsShape *s) {
    // latency shape: one word per lane while 32 lanes suffice, else 32 lanes
    s->g = std::min<uint32_t>(32, next_pow2(s->words));
    s->Q = (s->words + s->g - 1) / s->g;
}

uint32_t band_bits_max_width(uint32_t m, uint32_t n) {
    // 2w + |n-m| + 5 <= 64 * kBandBitsMaxWords covers the parity raise of hi
    const int64_t d = (int64_t)n - (int64_t)m, ad = d < 0 ? -d : d;
    const int64_t w = (64 * (int64_t)kBandBitsMaxWords - ad - 5) / 2;
    return w > 0 ? (uint32_t)w : 0u;
}

uint64_t band_bits_records(const BandBitsShape &s) { return (uint64_t)s.nchunks * 32u * s.g * s.Q; }

double band_bits_seconds(const BandBitsShape &s) {
    // 64 anti-diagonals per chunk, ~20 instructions per word and ~14 per
    // lane per step, two cycles each on a scheduler of its own, 2.07 GHz
    return (double)s.nchunks * 64.0 * (20.0 * s.Q + 14.0) * 2.0 / 2.07e9;
}

int band_bits_fill(nw_ctx *ctx, const PlaneSet &planes, const std::vector<BandBitsItem> &items, bool want, int32_t gap, int32_t *scores, uint32_t score_cap,
                   void *ptr, uint64_t ptr_records, std::vector<int32_t> &banded) {
    int rc;
    banded.assign(items.size(), 0);
    if (items.empty()) return NW_OK;
    HostTimer ht(ctx, "bband_fill_host");
    HostTimer htp(ctx, "bband_fill_prep");
    // jobs: pairs of equal shape (g, Q), similar lengths, 32/g per warp
    // (Q, g, chunks), each descending, ties in item order
    std::vector<uint64_t> keys(items.size());
    for (size_t k = 0; k < items.size(); ++k) {
        const BandBitsShape &sh = items[k].shape;
        keys[k] = ((uint64_t)sh.Q << 40) | ((uint64_t)sh.g << 32) | sh.nchunks;
    }
    const std::vector<uint32_t> order = radix_order_desc(std::move(keys));
    std::vector<BandBitsTask> tasks(items.size());
    std::vector<uint32_t> task_item(items.size());
    std::vector<BandBitsJob> jobs;
    for (uint32_t k = 0; k < order.size();) {
        const BandBitsShape &s0 = items[order[k]].shape;
        BandBitsJob j{k, 0, s0.g, s0.Q, s0.nchunks};
        while (k < order.size() && j.cnt < 32 / s0.g && items[order[k]].shape.g == s0.g &&
               items[order[k]].shape.Q == s0.Q) {
            const BandBitsItem &it = items[order[k]];
            BandBitsTask &t = tasks[k];
            t.a_slot = it.a_slot;
            t.b_slot = it.b_slot;
            t.ptr_off = it.ptr_off;
            t.m = it.m;
            t.n = it.n;
            t.hi = it.shape.hi;
            t.a_first = it.shape.a_first;
            t.nchunks = it.shape.nchunks;
            t.out0 = it.out0;
            task_item[k] = order[k];
            ++j.cnt;
            ++k;
        }
        jobs.push_back(j);
    }
    // longest jobs first (ties in job order)
    {
        std::vector<uint64_t> jk(jobs.size());
        for (size_t q = 0; q < jobs.size(); ++q) jk[q] = (uint64_t)jobs[q].nchunks * (20 * jobs[q].Q + 14);
        const std::vector<uint32_t> jo = radix_order_desc(std::move(jk));
        std::vector<BandBitsJob> sorted(jobs.size());
        for (size_t q = 0; q < jobs.size(); ++q) sorted[q] = jobs[jo[q]];
        jobs.swap(sorted);
    }
    void *v = nullptr;
    if ((rc = scratch(ctx, "bband_tasks", tasks.size() * sizeof(BandBitsTask) + 16, &v))) return rc;
    BandBitsTask *dt = (BandBitsTask *)v;
    if ((rc = scratch(ctx, "bband_jobs", jobs.size() * sizeof(BandBitsJob) + 16, &v))) return rc;
    BandBitsJob *dj = (BandBitsJob *)v;
    if ((rc = scratch(ctx, "bband_gather", items.size() * 4 + 16, &v))) return rc;
    int32_t *dg = (int32_t *)v;
    if ((rc = scratch(ctx, "bband_counter", 16, &v))) return rc;
    uint32_t *cnt = (uint32_t *)v;
    cudaError_t e = cudaMemcpyAsync(dt, tasks.data(), tasks.size() * sizeof(BandBitsTask), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dj, jobs.data(), jobs.size() * sizeof(BandBitsJob), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 4, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "banded bit-sliced tasks H2D");
    BandBitsArgs a{};
    a.pl0 = planes.pl0;
    a.pl1 = planes.pl1;
    a.max_base = planes.max_base;
    a.tasks = dt;
    a.jobs = dj;
    a.njobs = (uint32_t)jobs.size();
    a.counter = cnt;
    a.ptr = (uint4 *)ptr;
    a.ptr_cap = ptr_records;
    a.scores = scores;
    a.gathered = dg;
    a.score_cap = score_cap;
    a.gap = gap;
    a.err = ctx->d_err;
    auto kern = want ? k_bits_band<true> : k_bits_band<false>;
    htp.stop();
    // Two CTAs per SM (two warps per scheduler), not the five the registers
    // allow: the jobs are taken longest first, and a long job that shares
    // its scheduler with four others runs at a fifth of its speed and ends
    // the launch alone.  Measured on GB300 (config 4, 20,000 pairs, CTAs per
    // SM 5 / 4 / 3 / 2 / 1): the fills took 54.4 / 48.1 / 41.2 / 37.7 /
    // 45.0 ms.  NW_BBAND_OCC overrides (sweeps).
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBandWarps * 32, 0);
    int cap = 2;
    if (const char *e = getenv("NW_BBAND_OCC")) cap = std::max(1, atoi(e));
    occ = std::min(occ, cap);
    uint32_t blocks = (uint32_t)std::max(occ, 1) * (uint32_t)ctx->sm_count;
    blocks = std::max(1u, std::min(blocks, (a.njobs + kBandWarps - 1) / kBandWarps));
    {
        LaunchTimer t(ctx, want ? "bband_fill_ptr" : "bband_score");
        kern<<<blocks, kBandWarps * 32, 0, ctx->stream>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "banded bit-sliced launch");
    // the banded scores back, in item order
    std::vector<int32_t> g(items.size());
    e = cudaMemcpyAsync(g.data(), dg, items.size() * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "banded scores D2H");
    {
        HostTimer ht(ctx, "band_wait");
        if ((rc = nw_ctx_sync(ctx))) return rc;
    }
    for (size_t k = 0; k < items.size(); ++k) banded[task_item[k]] = g[k];
    return NW_OK;
}

int band_bits_walk(nw_ctx *ctx, const void *ptr, const std::vector<BandBitsItem> &items,
                   const std::vector<uint32_t> &which, const uint8_t *pool, char *cigar_pool,
                   const uint64_t *cigar_off, uint64_t *cigar_len, uint32_t mflag) {
    if (which.empty()) return NW_OK;
    int rc;
    HostTimer ht(ctx, "bband_walk_host");
    // longest walks first: the kernel's warps take pairs in order
    std::vector<uint32_t> order(which.size());
    {
        std::vector<uint64_t> wk(which.size());
        for (size_t q = 0; q < which.size(); ++q) wk[q] = (uint64_t)items[which[q]].m + items[which[q]].n;
        const std::vector<uint32_t> wo = radix_order_desc(std::move(wk));  // ties in `which` order
        for (size_t q = 0; q < which.size(); ++q) order[q] = which[wo[q]];
    }
    uint64_t mbytes = 0;
    for (uint32_t k : order) mbytes += (uint64_t)items[k].m + items[k].n + 16;
    void *mv = nullptr, *nm = nullptr, *v = nullptr;
    if ((rc = scratch(ctx, "bband_moves", mbytes + 16, &mv))) return rc;
    if ((rc = scratch(ctx, "bband_nmoves", which.size() * 8 + 16, &nm))) return rc;
    std::vector<BitsWalkTask> wt(which.size());
    std::vector<TraceTask> tt(which.size());
    uint64_t mpos = 0;
    for (size_t q = 0; q < order.size(); ++q) {
        const BandBitsItem &it = items[order[q]];
        wt[q] = BitsWalkTask{it.ptr_off, mpos, it.m, it.n, it.shape.g * it.shape.Q, it.shape.hi, it.shape.a_first,
                             (uint32_t)q};
        TraceTask x{};
        x.m = it.m;
        x.n = it.n;
        x.moves = (uint8_t *)mv + mpos;
        x.nmoves = (uint64_t *)nm + q;
        x.a = pool + it.a_off;
        x.b = pool + it.b_off;
        x.cigar = cigar_pool + cigar_off[it.out0];
        x.cigar_len = cigar_len + it.out0;
        x.band_lo = kNoBand;
        tt[q] = x;
        mpos += (uint64_t)it.m + it.n + 16;
    }
    if ((rc = scratch(ctx, "bband_walk_tasks", wt.size() * sizeof(BitsWalkTask) + 16, &v))) return rc;
    BitsWalkTask *dw = (BitsWalkTask *)v;
    if ((rc = scratch(ctx, "bband_trace_tasks", tt.size() * sizeof(TraceTask) + 16, &v))) return rc;
    TraceTask *dtt = (TraceTask *)v;
    cudaError_t e = cudaMemcpyAsync(dw, wt.data(), wt.size() * sizeof(BitsWalkTask), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtt, tt.data(), tt.size() * sizeof(TraceTask), cudaMemcpyHostToDevice, ctx->stream);
    // the host task arrays go out of scope: wait for their copies (the fill
    // before them has finished already; its scores were read back), not for
    // the walk, so the caller prepares its next round while the GPU walks
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "walk tasks H2D");
    {
        LaunchTimer t(ctx, "bband_walk");
        // every walk at once: each is a serial chain, so the launch's
        // throughput is the number in flight (capping the CTAs per SM at
        // 16 / 8 / 4 / 2 / 1 measured 8.6 / 9.3 / 10.1 / 14.9 / 24.2 ms per step
        // on config 4, against 8.3 ms uncapped)
        const uint32_t blocks = (uint32_t)std::min<size_t>((which.size() + kWalkWarps - 1) / kWalkWarps, 65535);
        // runs of diagonal moves at a time; NW_BWALK_SERIAL=1 walks one move
        // at a time on lane 0 (for comparisons)
        const char *se = getenv("NW_BWALK_SERIAL");
        auto walk = (se && *se == '1') ? k_bits_walk<false> : k_bits_walk<true>;
        walk<<<blocks, kWalkWarps * 32, 0, ctx->stream>>>((const uint4 *)ptr, dw, (uint32_t)which.size(),
                                                          (uint8_t *)mv, (uint64_t *)nm, ctx->d_err);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "walk launch");
    return launch_finish(ctx, TraceTask{}, dtt, (uint32_t)tt.size(), mflag);
}

}  // namespace nw
