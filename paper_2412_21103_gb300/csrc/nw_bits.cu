// Bit-sliced score-only fill (a3/a7): the Sec. 2.3 recurrence from the
// Sec. 2.2 boundary, 32 cells per machine word.
//
// Difference form.  In the W domain (W = H - gap*(i+j), see nw_internal.cuh)
// gaps cost nothing and a diagonal step gains s' = s - 2*gap, so W never
// decreases along a row or a column and never gains more than s'max over its
// diagonal neighbour.  With
//     dH(i,j) = W(i,j) - W(i,j-1),   dV(i,j) = W(i,j) - W(i-1,j),
// both lie in [0, s'max], and the recurrence becomes, for a = dH(i-1,j) (the
// cell above, against its left neighbour) and b = dV(i,j-1) (the cell to the
// left, against its upper neighbour):
//     T = W(i,j) - W(i-1,j-1) = max(s'(i,j), a, b),
//     dV(i,j) = T - a,   dH(i,j) = T - b.
// When 0 <= s'(mismatch) <= s'(match) <= 3 -- the paper's +1/-1/-1 gives 3
// and 1 -- every value fits in two bits, and a 32-bit word holds one bit of
// 32 cells: a "plane".  A lane keeps the planes of 32 consecutive rows on one
// anti-diagonal (bit p = row top + p); the cell above a bit is the bit below
// it on the previous anti-diagonal and the cell to its left is the same bit,
// so one anti-diagonal step is a fixed sequence of funnel shifts and
// three-input logic operations (LOP3) on whole words: about 20 instructions
// for 32 cells, where the scalar kernels spend 3 per cell.
//
// Work split.  One pair per lane.  Stripes of 32 rows are aligned to the
// bottom of the grid (the last stripe's bit 31 is row m); rows <= 0 of the
// first stripe are padding, forced to the boundary's zero differences by a
// row mask.  A stripe sweeps the anti-diagonals that cross it, in chunks of
// 32 steps: bit 0 meets column t+1 at step t, bit 31 column t-30.  The
// previous stripe's bottom row arrives as 32 input bits per chunk and the
// stripe's own bottom row leaves through the same shift register (one funnel
// shift per plane and step does both); the words go through a per-warp row
// buffer in global memory, [chunk][lane], so a warp's accesses coalesce.
// The lanes of a warp hold pairs of equal stripe count and similar width
// (a "job"), so they run in lockstep; jobs are taken longest first from an
// atomic counter.  The score is W(m,n) = sum over j of dH(m,j), read from the
// last stripe's outgoing words with population counts.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "nw_bits.cuh"

namespace nw {

// One anti-diagonal step of the 32 cells of a lane.  (H, V): the dH, dV
// planes of the previous anti-diagonal; Q: the shift register of the stripe
// boundary (bit 31 = the input bit of this step, the output bit enters at
// bit 0).  bw: the B window (bit p = base of column t+1-p), A: the row bases,
// rmask: rows of the grid (padding rows give s' = 0).  RAMP: the first chunk
// of a stripe, where bits p > u lie in column <= 0 and their dV is forced to
// the boundary's 0.
template <bool GEN, bool RAMP>
__device__ __forceinline__ void bits_step(int u, uint32_t &H0, uint32_t &H1, uint32_t &V0, uint32_t &V1, uint32_t &Q0,
                                          uint32_t &Q1, uint32_t A0, uint32_t A1, uint32_t bw0, uint32_t bw1,
                                          uint32_t rmask, const BitsScoring &g, uint32_t X1r, uint32_t X0r) {
    const uint32_t x = lop3<kLutXorOrNotC>(A1, bw1, rmask);
    const uint32_t eq = lop3<kLutEq>(A0, bw0, x);  // A_i == B_j (0 on padding rows)
    const uint32_t a0 = __funnelshift_l(Q0, H0, 1), a1 = __funnelshift_l(Q1, H1, 1);  // dH of the cell above
    const uint32_t b0 = V0, b1 = V1;                                                  // dV of the cell to the left
    const uint32_t p = lop3<kLutAndOrNot>(a0, a1, b1);  // the low bit of max(a, b), from a
    const uint32_t q = lop3<kLutAndOrNot>(b0, b1, a1);  // ... from b
    uint32_t T0, T1;
    if constexpr (!GEN) {
        // s' = (eq, 1) on grid rows (3 or 1), 0 on padding rows
        const uint32_t v = lop3<kLutCOrNor>(a1, b1, eq);
        T0 = p | lop3<kLutOrAnd>(q, v, rmask);
        T1 = lop3<kLutOr3>(a1, b1, eq);
    } else {
        const uint32_t e1 = lop3<kLutSel>(eq, g.M1, X1r), e0 = lop3<kLutSel>(eq, g.M0, X0r);
        const uint32_t m0 = p | q, m1 = a1 | b1;
        T0 = lop3<kLutAndNotOr>(m0, e1, m1) | lop3<kLutAndNotOr>(e0, m1, e1);
        T1 = m1 | e1;
    }
    const uint32_t ca = lop3<kLutAndNot>(a0, T0, 0u), cb = lop3<kLutAndNot>(b0, T0, 0u);  // borrows
    if constexpr (RAMP) {
        const uint32_t mk = (2u << u) - 1u;  // bits in column >= 1
        V0 = lop3<kLutXorAnd>(T0, a0, mk);
        V1 = lop3<kLutXor3>(T1, a1, ca) & mk;
    } else {
        V0 = T0 ^ a0;
        V1 = lop3<kLutXor3>(T1, a1, ca);
    }
    H0 = T0 ^ b0;
    H1 = lop3<kLutXor3>(T1, b1, cb);
    Q0 = __funnelshift_l(H0, Q0, 1);
    Q1 = __funnelshift_l(H1, Q1, 1);
}

template <bool GEN, bool RAMP>
__device__ __forceinline__ void bits_chunk(uint32_t &H0, uint32_t &H1, uint32_t &V0, uint32_t &V1, uint32_t &Q0,
                                           uint32_t &Q1, uint32_t A0, uint32_t A1, uint32_t Rc0, uint32_t Rc1,
                                           uint32_t Rn0, uint32_t Rn1, uint32_t rmask, const BitsScoring &g,
                                           uint32_t X1r, uint32_t X0r) {
#pragma unroll
    for (int u = 0; u < 32; ++u)
        bits_step<GEN, RAMP>(u, H0, H1, V0, V1, Q0, Q1, A0, A1, __funnelshift_l(Rn0, Rc0, u),
                             __funnelshift_l(Rn1, Rc1, u), rmask, g, X1r, X0r);
}

template <bool GEN>
__global__ void __launch_bounds__(kBitsWarps * 32) k_bits_score(BitsArgs p) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint2 *rows = p.rows + (size_t)gw * p.rows_chunks * 32u + lane;
    for (;;) {
        uint32_t jid = 0;
        if (lane == 0) jid = atomicAdd(p.counter, 1u);
        jid = __shfl_sync(kFull, jid, 0);
        if (jid >= p.njobs) break;
        const BitsJob job = p.jobs[jid];
        const bool active = lane < job.cnt;
        const BatchTask tk = p.tasks[job.t0 + (active ? lane : 0u)];
        const uint32_t m = tk.m, n = tk.n;
        const uint32_t S = job.S, C = job.C;
        int32_t W = 0;
        if (S > 0) {
            const int64_t Ag = (int64_t)tk.a_off, Bg = (int64_t)tk.b_off;  // planar slots
            const int32_t top0 = (int32_t)m - 32 * (int32_t)S;  // row above bit 0 of stripe 0
            for (uint32_t s = 0; s < S; ++s) {
                const int32_t pad = min(max(-top0 - 32 * (int32_t)s, 0), 32);  // padding rows of this stripe
                const uint32_t rmask = pad >= 32 ? 0u : (~0u << pad);
                const int64_t abase = max(Ag + top0 + 32 * (int64_t)s, Ag - 32);
                const uint32_t A0 = plane_window(p.pl0, abase), A1 = plane_window(p.pl1, abase);
                const uint32_t X1r = p.g.X1 & rmask, X0r = p.g.X0 & rmask;
                const bool first = s == 0, last = s + 1 == S;
                uint32_t H0 = 0, H1 = 0, V0 = 0, V1 = 0;
                uint32_t Rc0 = __brev(plane_window(p.pl0, Bg - 31)), Rc1 = __brev(plane_window(p.pl1, Bg - 31));
                uint2 prev = first ? make_uint2(0u, 0u) : __ldcg(rows);
                for (uint32_t c = 0; c < C; ++c) {
                    const int64_t gb = Bg + 32 * (int64_t)c + 1;
                    const uint32_t Rn0 = __brev(plane_window(p.pl0, gb)), Rn1 = __brev(plane_window(p.pl1, gb));
                    uint32_t Q0 = 0, Q1 = 0;
                    if (!first) {
                        // input bits: the previous stripe's bottom row, columns 32c+1 .. 32c+32,
                        // column 32c+1 at bit 31
                        const uint2 nx = c + 1 < C ? __ldcg(rows + (size_t)(c + 1) * 32u) : make_uint2(0u, 0u);
                        Q0 = __funnelshift_r(nx.x, prev.x, 1);
                        Q1 = __funnelshift_r(nx.y, prev.y, 1);
                        prev = nx;
                    }
                    if (c == 0) bits_chunk<GEN, true>(H0, H1, V0, V1, Q0, Q1, A0, A1, Rc0, Rc1, Rn0, Rn1, rmask, p.g, X1r, X0r);
                    else bits_chunk<GEN, false>(H0, H1, V0, V1, Q0, Q1, A0, A1, Rc0, Rc1, Rn0, Rn1, rmask, p.g, X1r, X0r);
                    // outgoing bits: bit b is column 32c+1-b of the stripe's bottom row
                    if (!last) {
                        __stcg(rows + (size_t)c * 32u, make_uint2(Q0, Q1));
                    } else {
                        const int32_t lo = max(32 * (int32_t)c + 1 - (int32_t)n, 0), hi = min(31, 32 * (int32_t)c);
                        if (lo <= hi) {
                            const uint32_t mk = (hi == 31 ? ~0u : ((2u << hi) - 1u)) & (~0u << lo);
                            W += __popc(Q0 & mk) + 2 * __popc(Q1 & mk);
                        }
                    }
                    Rc0 = Rn0;
                    Rc1 = Rn1;
                }
            }
        }
        if (active) {
            const int32_t sc = W + p.gap * (int32_t)(m + n);
            if (in_range(tk.out0, p.score_cap, p.err, kSiteBatchScore)) p.scores[tk.out0] = sc;
            if (tk.out1 != ~0u && in_range(tk.out1, p.score_cap, p.err, kSiteBatchScore)) p.scores[tk.out1] = sc;
        }
    }
}

// Compacts the even bits of x into the low 32 bits.
__device__ __forceinline__ uint32_t even_bits(uint64_t x) {
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
    x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
    x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
    return (uint32_t)x;
}

// Planar copy of the launch's sequences: one warp per sequence; word w of
// its slot holds bit k of the codes of its bases 32w .. 32w+31 (bases past
// its end read as 0).
__global__ void k_planes(const uint8_t *pool, const PlaneSeg *segs, uint32_t nsegs, uint32_t *pl0, uint32_t *pl1) {
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t sg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sg < nsegs; sg += (gridDim.x * blockDim.x) >> 5) {
        const PlaneSeg seg = segs[sg];
        const uint8_t *src = pool ? pool + seg.src : reinterpret_cast<const uint8_t *>(seg.src);  // offset or address
        const uint32_t words = (seg.nbytes + 7) / 8;
        for (uint32_t w = lane; w < words; w += 32) {
            uint64_t v = 0;
            const uint32_t b0 = 8 * w;
            if (b0 + 8 <= seg.nbytes) {
#pragma unroll
                for (int k = 0; k < 8; ++k) v |= (uint64_t)src[b0 + k] << (8 * k);
            } else {
                for (uint32_t k = 0; b0 + k < seg.nbytes; ++k) v |= (uint64_t)src[b0 + k] << (8 * k);
            }
            pl0[seg.dst + w] = even_bits(v);
            pl1[seg.dst + w] = even_bits(v >> 1);
        }
    }
}

// ------------------------------------------------------------------ host
static size_t plane_hash(uint64_t off, uint32_t len) {
    uint64_t z = off * 0x9E3779B97F4A7C15ull ^ ((uint64_t)len << 17);
    z ^= z >> 31;
    z *= 0xBF58476D1CE4E5B9ull;
    return (size_t)(z ^ (z >> 29));
}

void PlaneSet::rehash(size_t size) {
    std::vector<Entry> old;
    old.swap(table_);
    table_.assign(size, Entry{0, 0, 0, 0});
    for (const Entry &e : old) {
        if (!e.used) continue;
        size_t h = plane_hash(e.off, e.len) & (size - 1);
        while (table_[h].used) h = (h + 1) & (size - 1);
        table_[h] = e;
    }
}

void PlaneSet::reserve(size_t n) {
    size_t size = 64;
    while (size < 2 * n) size *= 2;
    if (size > table_.size()) rehash(size);
    segs_.reserve(n);
}

int64_t PlaneSet::add(uint64_t off, uint32_t len) {
    if (2 * (count_ + 1) > table_.size()) rehash(std::max<size_t>(64, 2 * table_.size()));
    const size_t mask = table_.size() - 1;
    size_t h = plane_hash(off, len) & mask;
    for (; table_[h].used; h = (h + 1) & mask)
        if (table_[h].off == off && table_[h].len == len) return table_[h].slot;
    const uint32_t nbytes = (len + 3) / 4;
    const int64_t slot = (int64_t)words_ * 32 - kPlanePad;
    segs_.push_back(PlaneSeg{off, nbytes, (uint32_t)words_});
    words_ += (nbytes + 7) / 8 + 2;
    table_[h] = Entry{off, len, 1, slot};
    ++count_;
    return slot;
}

int PlaneSet::prepare(nw_ctx *ctx, const std::string &prefix) {
    int rc;
    void *v = nullptr;
    const uint64_t words = words_ + 4;  // room for the last window's second word
    if (words >= (1ull << 32)) return fail(ctx, NW_ERR_ARG, "planar copy of more than 2^37 bases");
    if ((rc = scratch(ctx, (prefix + "_planes").c_str(), (size_t)words * 8, &v))) return rc;
    planes_ = (uint32_t *)v;
    pl0 = planes_;
    pl1 = planes_ + words;
    max_base = (int64_t)words * 32 - kPlanePad - 64;
    if ((rc = scratch(ctx, (prefix + "_plane_segs").c_str(), segs_.size() * sizeof(PlaneSeg) + 16, &v))) return rc;
    dsegs_ = (PlaneSeg *)v;
    if (!segs_.empty()) {
        cudaError_t e = cudaMemcpyAsync(dsegs_, segs_.data(), segs_.size() * sizeof(PlaneSeg), cudaMemcpyHostToDevice,
                                        ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the table is host memory of this object
        if (e != cudaSuccess) return cuda_fail(ctx, e, "planar segments H2D");
    }
    return NW_OK;
}

int PlaneSet::enqueue(nw_ctx *ctx, const uint8_t *pool) const {
    if (segs_.empty()) return NW_OK;
    {
        LaunchTimer t(ctx, "planes");
        const uint32_t blocks = (uint32_t)std::min<size_t>((segs_.size() + 7) / 8, 4096);
        k_planes<<<blocks, 256, 0, ctx->stream>>>(pool, dsegs_, (uint32_t)segs_.size(), planes_,
                                                  planes_ + (words_ + 4));
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "planar copy launch");
}

int PlaneSet::launch(nw_ctx *ctx, const uint8_t *pool, const std::string &prefix) {
    const int rc = prepare(ctx, prefix);
    return rc ? rc : enqueue(ctx, pool);
}

bool bits_scoring_ok(const nw_scoring &sc) {
    const int32_t sm = sc.match - 2 * sc.gap, sx = sc.mismatch - 2 * sc.gap;
    return sx >= 0 && sx <= sm && sm <= 3;
}

template <typename T>
static int bits_upload(nw_ctx *ctx, const std::string &slot, const std::vector<T> &v, T **dev) {
    void *d = nullptr;
    int rc = scratch(ctx, slot.c_str(), v.size() * sizeof(T) + 16, &d);
    if (rc) return rc;
    if (!v.empty()) {
        cudaError_t e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the host vector is temporary
        if (e != cudaSuccess) return cuda_fail(ctx, e, "bit-sliced task upload");
    }
    *dev = (T *)d;
    return NW_OK;
}

int bits_prepare(nw_ctx *ctx, const uint8_t *pool, std::vector<BatchTask> &tasks, const nw_scoring &sc,
                 int32_t *scores, uint32_t score_cap, const std::string &prefix, BitsPlan *plan) {
    int rc;
    *plan = BitsPlan{};
    if (tasks.empty()) return NW_OK;
    // rows: the orientation with fewer stripe-chunks (the score is symmetric)
    auto S_of = [](uint32_t m) { return (m + 31) / 32; };
    auto C_of = [](uint32_t n) { return (n + 62) / 32; };
    for (auto &t : tasks) {
        if (t.m == 0 || t.n == 0) continue;
        if ((uint64_t)S_of(t.n) * C_of(t.m) < (uint64_t)S_of(t.m) * C_of(t.n)) {
            std::swap(t.a_off, t.b_off);
            std::swap(t.m, t.n);
        }
    }
    // jobs: equal stripe counts, widest first, at most 32 pairs each
    auto S_task = [&](const BatchTask &t) { return (t.m && t.n) ? S_of(t.m) : 0u; };
    std::stable_sort(tasks.begin(), tasks.end(), [&](const BatchTask &x, const BatchTask &y) {
        const uint32_t sx = S_task(x), sy = S_task(y);
        if (sx != sy) return sx > sy;
        return x.n > y.n;
    });
    std::vector<BitsJob> jobs;
    uint32_t maxC = 1;
    for (uint32_t k = 0; k < tasks.size();) {
        const uint32_t S = S_task(tasks[k]);
        BitsJob j{k, 0, S, S ? C_of(tasks[k].n) : 0};
        while (k < tasks.size() && j.cnt < 32 && S_task(tasks[k]) == S) {
            ++j.cnt;
            ++k;
        }
        maxC = std::max(maxC, j.C);
        jobs.push_back(j);
    }
    std::stable_sort(jobs.begin(), jobs.end(),
                     [](const BitsJob &x, const BitsJob &y) { return (uint64_t)x.S * x.C > (uint64_t)y.S * y.C; });

    void *v = nullptr;
    // the tasks address their sequences by planar slot
    for (auto &t : tasks) {
        if (!t.m || !t.n) continue;
        t.a_off = (uint64_t)plan->planes.add(t.a_off, t.m);
        t.b_off = (uint64_t)plan->planes.add(t.b_off, t.n);
    }
    if ((rc = plan->planes.prepare(ctx, prefix))) return rc;
    BitsArgs &ba = plan->ba;
    ba.pl0 = plan->planes.pl0;
    ba.pl1 = plan->planes.pl1;
    BatchTask *dt = nullptr;
    BitsJob *dj = nullptr;
    if ((rc = bits_upload(ctx, prefix + "_bits_tasks", tasks, &dt))) return rc;
    if ((rc = bits_upload(ctx, prefix + "_bits_jobs", jobs, &dj))) return rc;
    ba.tasks = dt;
    ba.jobs = dj;
    ba.njobs = (uint32_t)jobs.size();
    ba.scores = scores;
    ba.score_cap = score_cap;
    ba.gap = sc.gap;
    ba.err = ctx->d_err;
    const int32_t sm = sc.match - 2 * sc.gap, sx = sc.mismatch - 2 * sc.gap;
    ba.g.M1 = (sm & 2) ? ~0u : 0u;
    ba.g.M0 = (sm & 1) ? ~0u : 0u;
    ba.g.X1 = (sx & 2) ? ~0u : 0u;
    ba.g.X0 = (sx & 1) ? ~0u : 0u;
    plan->gen = !(sm == 3 && sx == 1);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, plan->gen ? k_bits_score<true> : k_bits_score<false>,
                                                  kBitsWarps * 32, 0);
    // One CTA of 8 warps per SM (two warps per scheduler), not the most the
    // registers allow: with more, the longest jobs -- taken first -- share
    // their scheduler with the rest and finish the launch alone.  Measured on
    // GB300 (all-vs-all of 512 sequences, CTAs per SM 8 / 3 / 2 / 1): 17.6k /
    // 17.7k / 22.4k / 23.7k GCUPS.  NW_BITS_OCC overrides (sweeps).
    int cap = 1;
    if (const char *e = getenv("NW_BITS_OCC")) cap = std::max(1, atoi(e));
    occ = std::min(occ, cap);
    if (occ < 1) occ = 1;
    uint32_t blocks = (uint32_t)occ * (uint32_t)ctx->sm_count;
    const uint32_t need = (ba.njobs + kBitsWarps - 1) / kBitsWarps;
    plan->blocks = std::max(1u, std::min(blocks, need));
    ba.rows_chunks = maxC;
    if ((rc = scratch(ctx, (prefix + "_bits_rows").c_str(),
                      (size_t)plan->blocks * kBitsWarps * maxC * 32 * sizeof(uint2), &v)))
        return rc;
    ba.rows = (uint2 *)v;
    if ((rc = scratch(ctx, (prefix + "_bits_counter").c_str(), 16, &v))) return rc;
    ba.counter = (uint32_t *)v;
    plan->pool = pool;
    return NW_OK;
}

int bits_launch(nw_ctx *ctx, const BitsPlan &plan) {
    if (plan.ba.njobs == 0) return NW_OK;
    cudaMemsetAsync(plan.ba.counter, 0, 4, ctx->stream);
    if (int rc = plan.planes.enqueue(ctx, plan.pool)) return rc;
    {
        LaunchTimer t(ctx, "bits_score");
        if (plan.gen) k_bits_score<true><<<plan.blocks, kBitsWarps * 32, 0, ctx->stream>>>(plan.ba);
        else k_bits_score<false><<<plan.blocks, kBitsWarps * 32, 0, ctx->stream>>>(plan.ba);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "bit-sliced launch");
}

}  // namespace nw
