// Bit-sliced fill of one long pair (a3/a4), spread over many warps: the
// Sec. 2.3 recurrence in the difference form of nw_bits.cu (two bit planes
// per anti-diagonal word), with pointer records for the Sec. 2.4 walk.
//
// Work split.  Stripes of 31 rows from the top of the grid (stripe s: rows
// 31s + 1 .. 31s + 31); a lane's word holds its stripe's rows in bits 0..30.
// Bit 31, and the rows of the last stripe past m, are spare rows: their
// differences stay in [0, 3] like any row's, and nothing reads them (they
// lie below every grid row of their word).  So the cell update needs no
// row mask.  Bit p at stripe step t is the cell of column t + 1 - p.
// Stripe s belongs to lane s % 32 of warp s / 32, and lane l runs its
// stripe 32 steps behind lane l - 1: at warp step tau it takes stripe step
// t = tau - 32l, so all lanes share the step within a chunk of 32 and the
// B window shifts stay compile-time constants.
//
// Bit 0 of a stripe needs, at step t, dH of the stripe above's bottom row
// (its bit 30) at column t + 1, which that stripe computed at its step
// t + 30: two warp steps earlier.  So a lane shuffles its neighbour's dH
// planes (shifted so that bit 30 lands on bit 31) at the start of a step
// and uses them at the next one: the shuffle's latency overlaps a whole
// step instead of lengthening every step's dependency chain.
//
// Between warps the bottom lane's outgoing words (32 steps of its bottom
// row, per chunk) pass through a ring in global memory: two 64-bit entries
// per chunk, each a data word and a tag (the launch's epoch), written and
// read as single 64-bit accesses, so a reader that sees the tag sees the
// data.  Lane 0 of the next warp needs the words of chunks c and c + 1 for
// its chunk c; it loads them one chunk ahead and waits (bounded) only when
// they are late.  A warp never waits for the warp below it, and the launch
// is cooperative, so every warp it waits for is resident.
//
// Records.  Per stripe and step the pair (L, Hb): bit p of L is 0 where the
// diagonal predecessor attains the maximum (T = s'), bit p of Hb is 0 where
// the upper one does (dV = 0).  They are laid out [warp][tau][lane], two
// steps per 16-byte store, so a warp's stores are contiguous.
#include <algorithm>
#include <cstdlib>
#include <numeric>
#include <vector>

#include "nw_bits.cuh"

namespace nw {

constexpr int kPairWarps = 4;        // most warps per CTA (one per scheduler)
constexpr uint32_t kPairRows = 31;   // rows per stripe (bits 0..30 of a word)
// Truth tables (from a = 0xF0, b = 0xCC, c = 0xAA) of the shallow update.
constexpr uint32_t kLutAndNotNot = lut(kA & ~kB & ~kC);  // a & !b & !c
constexpr uint32_t kLutAndNand = lut(kA & ~(kB & kC));   // a & !(b & c)
constexpr uint32_t kLutOrAndNot = lut((kA | kB) & ~kC);  // (a | b) & !c
constexpr uint32_t kLutXorAndNot = lut(kA ^ (kB & ~kC)); // a ^ (b & !c)

// One pair of a launch (device array).
struct PairDesc {
    int64_t Ag, Bg;             // slots of a (rows) and b (columns)
    uint32_t m, n, S, C;        // stripes, chunks of 32 steps per stripe
    uint32_t nwarps;
    uint32_t pm;                // bit of row m in the last stripe
    uint32_t rec_rows;          // step pairs per warp: the last lane's steps and a walk tile's overhang
    uint32_t pad;
    uint64_t rec_off;           // the pair's records: rec + rec_off (uint4 units)
    uint64_t ring_off;          // the pair's ring: ring + ring_off (64-bit words)
    int32_t *score;
};
// A CTA's pair and the index of its first warp in that pair.
struct PairBlock {
    uint32_t pair, w0;
};
// A launch: several pairs at once, each on its own warps, every warp of
// every pair resident (cooperative launch).
struct PairLaunch {
    const uint32_t *pl0, *pl1;  // planar sequences
    const PairDesc *pairs;
    const PairBlock *blocks;
    uint4 *rec;                 // records, per pair [warp][rec_rows][32 lanes] (two steps each), or null
    uint64_t *ring;             // per pair [warp][C][2] tagged outgoing words of lane 31
    uint32_t epoch;             // tag of this launch (never 0)
    int32_t gap;
    BitsScoring g;
    uint32_t *err;
};
// What one warp sees of its pair.
struct PairBitsArgs {
    const uint32_t *pl0, *pl1;
    int64_t Ag, Bg;
    uint32_t m, n, S, C, nwarps, pm;
    uint4 *rec;
    uint32_t rec_rows;
    uint64_t *ring;
    uint32_t epoch;
    int32_t *score;
    int32_t gap;
    BitsScoring g;
    uint32_t *err;
};

__device__ __forceinline__ uint64_t ld_relaxed64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_relaxed64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// x * k (a left shift by a power of two) as an integer multiply-add, which
// the multiply-add pipe can take while the logic pipe runs the cell update.
__device__ __forceinline__ uint32_t mul(uint32_t x, uint32_t k) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, 0;" : "=r"(d) : "r"(x), "r"(k));
    return d;
}

// Entries of ring chunk c: their tags match the epoch once written.
struct RingWords {
    uint64_t e0, e1;
    __device__ bool ready(uint32_t epoch) const {
        return (uint32_t)(e0 >> 32) == epoch && (uint32_t)(e1 >> 32) == epoch;
    }
    __device__ uint2 words() const { return make_uint2((uint32_t)e0, (uint32_t)e1); }
};

__device__ __forceinline__ RingWords ring_load(const uint64_t *ring, uint32_t c) {
    return RingWords{ld_relaxed64(ring + 2 * (size_t)c), ld_relaxed64(ring + 2 * (size_t)c + 1)};
}

// Waits until chunk c of the ring is written (bounded: two seconds or 2^24
// polls, or an error raised elsewhere).  Uniform across the warp: every lane
// reads the same words.
__device__ bool ring_wait(const uint64_t *ring, uint32_t c, uint32_t epoch, uint32_t *err, RingWords &r) {
    if (r.ready(epoch)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t spins = 1;; ++spins) {
        r = ring_load(ring, c);
        if (r.ready(epoch)) return true;
        if ((spins & 63u) == 0) {
            if (*(volatile uint32_t *)err != 0u) return false;
            if (spins >= kSpinLimit || global_ns() - t0 > kSpinNanos) {
                raise_error(err, NW_ERR_TIMEOUT, 0x60000u + c);
                return false;
            }
        }
        __nanosleep(32);
    }
}

// Per-lane state of the fill.  H, V: the dH, dV planes of the lane's last
// anti-diagonal; G = H shifted so that bit 31 is the bottom row's dH (bit
// 30, or row m's bit in the last stripe); Y: the word
// whose bit 31 is this step's input bit; Qi: lane 0's input bits of the
// chunk, the current one at bit 31; Qo: the bottom row's outgoing bits,
// the latest at bit 0.
struct PairState {
    uint32_t H0, H1, V0, V1, G0, G1, Y0, Y1, Qi0, Qi1, Qo0, Qo1;
};

// One anti-diagonal step of a lane's 31 rows (see bits_step in nw_bits.cu
// for the difference form).  Z: all ones on lane 0, which takes its input
// from Qi instead of the neighbour; gmul: 2^(31 - bottom bit).  RAMP: the
// first chunk of a lane (rz = 0 there), where bits p > u lie in column <= 0
// and their dV is forced to the boundary's 0.  L, Hb: the step's records.
template <bool GEN, bool RAMP>
__device__ __forceinline__ void pair_step(int u, PairState &st, uint32_t A0, uint32_t A1, uint32_t bw0, uint32_t bw1,
                                          uint32_t Z, uint32_t gmul, uint32_t rz, const BitsScoring &g, uint32_t &L,
                                          uint32_t &Hb) {
    // the neighbour's bottom row after the previous step: the next step's input
    const uint32_t N0 = __shfl_up_sync(kFull, st.G0, 1), N1 = __shfl_up_sync(kFull, st.G1, 1);
    const uint32_t eq = lop3<kLutEq>(A0, bw0, A1 ^ bw1);  // A_i == B_j
    const uint32_t a0 = __funnelshift_l(st.Y0, st.H0, 1), a1 = __funnelshift_l(st.Y1, st.H1, 1);  // dH above
    const uint32_t b0 = st.V0, b1 = st.V1;                                                        // dV left
    if constexpr (!GEN) {
        // s' = (eq, 1).  T = 3 where eq; else T = max(1, a, b), whose low bit
        // is 0 exactly where max(a, b) = 2.  Written so that T0 is two logic
        // levels after a (not three), and dV, dH one more:
        //   T0 = eq | !(a = 2, b < 3  or  b = 2, a < 3)
        //   dV1 = ((eq | b1) & !a1) ^ (a0 & !T0),  dH1 = ((eq | a1) & !b1) ^ (b0 & !T0)
        const uint32_t b2 = lop3<kLutAndNot>(b1, b0, 0u), b3 = b1 & b0;  // b = 2, b = 3
        const uint32_t x1 = lop3<kLutAndNotNot>(a1, a0, b3), x2 = lop3<kLutAndNand>(b2, a1, a0);
        const uint32_t sv = lop3<kLutOrAndNot>(eq, b1, a1), sh = lop3<kLutOrAndNot>(eq, a1, b1);
        const uint32_t T0 = lop3<kLutCOrNor>(x1, x2, eq);
        L = lop3<kLutOrAndNot>(a1, b1, eq) | ~T0;  // T != s'
        if constexpr (RAMP) {
            const uint32_t mk = ((2u << u) - 1u) | rz;
            st.V0 = lop3<kLutXorAnd>(T0, a0, mk);
            st.V1 = lop3<kLutXorAndNot>(sv, a0, T0) & mk;
        } else {
            st.V0 = T0 ^ a0;
            st.V1 = lop3<kLutXorAndNot>(sv, a0, T0);
        }
        st.H0 = T0 ^ b0;
        st.H1 = lop3<kLutXorAndNot>(sh, b0, T0);
    } else {
        const uint32_t p = lop3<kLutAndOrNot>(a0, a1, b1);
        const uint32_t q = lop3<kLutAndOrNot>(b0, b1, a1);
        const uint32_t e1 = lop3<kLutSel>(eq, g.M1, g.X1), e0 = lop3<kLutSel>(eq, g.M0, g.X0);
        const uint32_t m0 = p | q, m1 = a1 | b1;
        const uint32_t T0 = lop3<kLutAndNotOr>(m0, e1, m1) | lop3<kLutAndNotOr>(e0, m1, e1);
        const uint32_t T1 = m1 | e1;
        L = (T1 ^ e1) | (T0 ^ e0);
        const uint32_t ca = lop3<kLutAndNot>(a0, T0, 0u), cb = lop3<kLutAndNot>(b0, T0, 0u);
        if constexpr (RAMP) {
            const uint32_t mk = ((2u << u) - 1u) | rz;
            st.V0 = lop3<kLutXorAnd>(T0, a0, mk);
            st.V1 = lop3<kLutXor3>(T1, a1, ca) & mk;
        } else {
            st.V0 = T0 ^ a0;
            st.V1 = lop3<kLutXor3>(T1, a1, ca);
        }
        st.H0 = T0 ^ b0;
        st.H1 = lop3<kLutXor3>(T1, b1, cb);
    }
    Hb = st.V0 | st.V1;
    st.Qi0 = mul(st.Qi0, 2u);
    st.Qi1 = mul(st.Qi1, 2u);
    st.Y0 = lop3<kLutSel>(Z, st.Qi0, N0);
    st.Y1 = lop3<kLutSel>(Z, st.Qi1, N1);
    st.G0 = mul(st.H0, gmul);
    st.G1 = mul(st.H1, gmul);
    st.Qo0 = __funnelshift_l(st.G0, st.Qo0, 1);
    st.Qo1 = __funnelshift_l(st.G1, st.Qo1, 1);
}

// 32 steps; with PTR the records of steps 2v, 2v + 1 go to recp[v * 32].
template <bool GEN, bool RAMP, bool PTR>
__device__ __forceinline__ void pair_chunk(PairState &st, uint32_t A0, uint32_t A1, uint32_t Rc0, uint32_t Rc1,
                                           uint32_t Rn0, uint32_t Rn1, uint32_t Z, uint32_t gmul, uint32_t rz,
                                           const BitsScoring &g, uint4 *recp) {
    uint32_t Lp = 0, Hp = 0;
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        uint32_t L, Hb;
        pair_step<GEN, RAMP>(u, st, A0, A1, __funnelshift_l(Rn0, Rc0, u), __funnelshift_l(Rn1, Rc1, u), Z, gmul, rz,
                             g, L, Hb);
        if constexpr (PTR) {
            if (u & 1) __stcg(recp + (size_t)(u >> 1) * 32u, make_uint4(Lp, Hp, L, Hb));
            Lp = L;
            Hp = Hb;
        }
    }
}

template <bool GEN, bool PTR>
__global__ void __launch_bounds__(kPairWarps * 32, 1) k_bits_pair(PairLaunch L) {
    const uint32_t lane = threadIdx.x & 31u;
    const PairBlock bk = L.blocks[blockIdx.x];
    const PairDesc pd = L.pairs[bk.pair];
    const uint32_t w = bk.w0 + (threadIdx.x >> 5);
    if (w >= pd.nwarps) return;
    const PairBitsArgs p{L.pl0, L.pl1, pd.Ag, pd.Bg, pd.m, pd.n, pd.S, pd.C, pd.nwarps, pd.pm,
                         PTR ? L.rec + pd.rec_off : nullptr, pd.rec_rows, L.ring + pd.ring_off, L.epoch, pd.score,
                         L.gap, L.g, L.err};
    const uint32_t S = p.S, C = p.C;
    const uint32_t s = 32u * w + lane;
    const bool valid = s < S;
    const uint32_t K = C + min(31u, S - 1 - 32u * w);  // chunks until the warp's last lane is done
    const int64_t abase = valid ? p.Ag + (int64_t)kPairRows * s : p.Ag - 32;  // base of bit 0's row
    const uint32_t A0 = plane_window(p.pl0, abase), A1 = plane_window(p.pl1, abase);
    const uint32_t Z = lane == 0 ? ~0u : 0u;
    const bool last = s + 1 == S, out = lane == 31 && w + 1 < p.nwarps;
    const uint32_t gmul = 1u << (31u - (last ? p.pm : kPairRows - 1));  // bottom row -> bit 31 of G
    const uint64_t *rin = w ? p.ring + (size_t)(w - 1) * C * 2u : nullptr;
    uint64_t *rout = p.ring + (size_t)w * C * 2u;
    uint4 *recw = PTR ? p.rec + (size_t)w * p.rec_rows * 32u + lane : nullptr;
    PairState st{};
    int32_t W = 0;
    uint2 prev = make_uint2(0u, 0u);  // ring words of lane 0's current chunk
    RingWords ahead{0, 0};            // ring entries of the next chunk, loaded one chunk early
    if (rin) {
        RingWords r = ring_load(rin, 0);
        if (!ring_wait(rin, 0, p.epoch, p.err, r)) return;
        prev = r.words();
        if (C > 1) ahead = ring_load(rin, 1);
    }
    for (uint32_t k = 0; k < K; ++k) {
        // lane 0's input bits for chunk k: the stripe above's bottom row,
        // columns 32k + 1 .. 32k + 32, column 32k + 1 at bit 31 (the ring's
        // bit b of chunk c is column 32c + 2 - b); row 0's zero differences
        // for the first stripe
        uint32_t qin0 = 0, qin1 = 0;
        if (rin && k < C) {
            uint2 nx = make_uint2(0u, 0u);
            if (k + 1 < C) {
                if (!ring_wait(rin, k + 1, p.epoch, p.err, ahead)) return;
                nx = ahead.words();
                if (k + 2 < C) ahead = ring_load(rin, k + 2);
            }
            qin0 = __funnelshift_r(nx.x, prev.x, 2);
            qin1 = __funnelshift_r(nx.y, prev.y, 2);
            prev = nx;
        }
        if (lane == 0) {
            st.Qi0 = st.Y0 = qin0;
            st.Qi1 = st.Y1 = qin1;
        }
        const int32_t c = (int32_t)k - (int32_t)lane;  // this lane's chunk
        const bool act = valid && c >= 0 && c < (int32_t)C;
        const uint32_t cc = (uint32_t)min(max(c, 0), (int32_t)C - 1);
        const int64_t gb = p.Bg + 32 * (int64_t)cc;
        const uint32_t Rc0 = __brev(plane_window(p.pl0, gb - 31)), Rc1 = __brev(plane_window(p.pl1, gb - 31));
        const uint32_t Rn0 = __brev(plane_window(p.pl0, gb + 1)), Rn1 = __brev(plane_window(p.pl1, gb + 1));
        if (c == 0) {
            st.H0 = st.H1 = st.V0 = st.V1 = st.G0 = st.G1 = 0;
        }
        uint4 *recp = PTR ? recw + (size_t)k * 16u * 32u : nullptr;
        if (k < 32) {
            const uint32_t rz = c == 0 ? 0u : ~0u;
            pair_chunk<GEN, true, PTR>(st, A0, A1, Rc0, Rc1, Rn0, Rn1, Z, gmul, rz, p.g, recp);
        } else {
            pair_chunk<GEN, false, PTR>(st, A0, A1, Rc0, Rc1, Rn0, Rn1, Z, gmul, ~0u, p.g, recp);
        }
        // outgoing bits: bit b is column 32c + 2 - b of the stripe's bottom row
        if (act && out) {
            st_relaxed64(rout + 2 * (size_t)c, ((uint64_t)p.epoch << 32) | st.Qo0);
            st_relaxed64(rout + 2 * (size_t)c + 1, ((uint64_t)p.epoch << 32) | st.Qo1);
        }
        if (act && last) {
            // bit b of Qo: row m at step 32c + 31 - b, column 32c + 32 - b - pm
            const int32_t top = 32 * c + 32 - (int32_t)p.pm;
            const int32_t lo = max(top - (int32_t)p.n, 0), hi = min(31, top - 1);
            if (lo <= hi) {
                const uint32_t mk = (hi == 31 ? ~0u : ((2u << hi) - 1u)) & (~0u << lo);
                W += __popc(st.Qo0 & mk) + 2 * __popc(st.Qo1 & mk);
            }
        }
    }
    if (last) *p.score = W + p.gap * (int32_t)(p.m + p.n);
}

// ------------------------------------------------------------------ host
namespace {
struct PairGeom {
    uint32_t S, C, nwarps, rec_rows;
    uint64_t rec_bytes, ring_bytes;
};

PairGeom pair_geom(uint32_t m, uint32_t n) {
    PairGeom g;
    g.S = (m + kPairRows - 1) / kPairRows;
    g.C = (uint32_t)(((uint64_t)n + kPairRows - 1 + 31u) / 32u);  // steps 0 .. n + 29
    g.nwarps = (g.S + 31u) / 32u;
    // the last lane's steps end at warp step 32 (C + 31); a walk tile of 64
    // steps may start up to 63 steps before a stripe's last step
    g.rec_rows = 16u * (g.C + 33u);
    g.rec_bytes = (uint64_t)g.nwarps * g.rec_rows * 32u * 16u;
    g.ring_bytes = (uint64_t)g.nwarps * g.C * 16u;
    return g;
}

bool env_on(const char *name) {
    const char *v = getenv(name);
    return v && *v && *v != '0';
}

const void *pair_kernel(bool gen, bool want) {
    return want ? (gen ? (const void *)k_bits_pair<true, true> : (const void *)k_bits_pair<false, true>)
                : (gen ? (const void *)k_bits_pair<true, false> : (const void *)k_bits_pair<false, false>);
}

// Most warps of the kernel (one per CTA) that the device holds at once.
uint32_t resident_warps(nw_ctx *ctx, bool gen, bool want) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_kernel(gen, want), 32, 0) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    return (uint32_t)std::max(occ, 1) * (uint32_t)ctx->sm_count;
}

bool gen_of(const nw_scoring &sc) {
    return !(sc.match - 2 * sc.gap == 3 && sc.mismatch - 2 * sc.gap == 1);
}
}  // namespace

bool bits_pair_takes(nw_ctx *ctx, uint32_t m, uint32_t n, const nw_scoring &sc, bool want) {
    if (env_on("NW_PAIR_SCALAR") || !bits_scoring_ok(sc) || m == 0 || n == 0) return false;
    const char *mn = getenv("NW_BITS_PAIR_MIN");  // smallest side taken (test and sweep knob)
    const uint32_t min_side = mn ? (uint32_t)atoi(mn) : 64u;
    if (std::min(m, n) < min_side) return false;
    const PairGeom g = pair_geom(m, n);
    if (g.nwarps > resident_warps(ctx, gen_of(sc), want)) return false;
    uint64_t need = g.ring_bytes + 64;
    if (want) need += g.rec_bytes + (uint64_t)m + n + 64;
    return need <= scratch_headroom(ctx, "bpair_rec");
}

int bits_pairs(nw_ctx *ctx, const uint8_t *pool, const std::vector<PairJob> &jobs, const nw_scoring &sc, bool want,
               uint32_t mflag) {
    if (jobs.empty()) return NW_OK;
    int rc;
    const bool gen = gen_of(sc);
    PlaneSet ps;
    std::vector<int64_t> ag(jobs.size()), bg(jobs.size());
    for (size_t k = 0; k < jobs.size(); ++k) {
        ag[k] = ps.add(jobs[k].a_off, jobs[k].m);
        bg[k] = ps.add(jobs[k].b_off, jobs[k].n);
    }
    if ((rc = ps.launch(ctx, pool, "bpair"))) return rc;
    PairLaunch L{};
    L.pl0 = ps.pl0;
    L.pl1 = ps.pl1;
    L.gap = sc.gap;
    L.err = ctx->d_err;
    const int32_t sm = sc.match - 2 * sc.gap, sx = sc.mismatch - 2 * sc.gap;
    L.g.M1 = (sm & 2) ? ~0u : 0u;
    L.g.M0 = (sm & 1) ? ~0u : 0u;
    L.g.X1 = (sx & 2) ? ~0u : 0u;
    L.g.X0 = (sx & 1) ? ~0u : 0u;
    // longest chains first; a wave takes pairs while their warps are all
    // resident at once and their records fit the budget
    std::vector<size_t> order(jobs.size());
    std::iota(order.begin(), order.end(), (size_t)0);
    auto steps = [&](size_t k) { return (double)jobs[k].m + jobs[k].n + jobs[k].m / 31.0; };
    std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return steps(x) > steps(y); });
    const uint32_t cap_warps = resident_warps(ctx, gen, want);
    // half of what the records' slot may grow to: the walks and the rest of
    // a batch still need scratch after the waves (a lone pair may take more)
    const uint64_t room = scratch_headroom(ctx, "bpair_rec") / 2;
    size_t next = 0;
    while (next < order.size()) {
        std::vector<size_t> wave;
        uint64_t warps = 0, rec = 0, ring = 0, moves = 0;
        while (next < order.size()) {
            const size_t k = order[next];
            const PairGeom g = pair_geom(jobs[k].m, jobs[k].n);
            const uint64_t r = want ? g.rec_bytes : 0;
            if (!wave.empty() && (warps + g.nwarps > cap_warps || rec + r > room)) break;  // a first pair always goes
            if (g.nwarps > cap_warps)
                return fail(ctx, NW_ERR_ARG, "pair of %u rows needs %u resident warps", jobs[k].m, g.nwarps);
            wave.push_back(k);
            warps += g.nwarps;
            rec += r;
            ring += g.ring_bytes;
            moves += (uint64_t)jobs[k].m + jobs[k].n + 16;
            ++next;
        }
        // pair table and block table
        std::vector<PairDesc> descs;
        std::vector<PairBlock> blocks;
        uint64_t rec_off = 0, ring_off = 0;
        for (size_t q = 0; q < wave.size(); ++q) {
            const PairJob &j = jobs[wave[q]];
            const PairGeom g = pair_geom(j.m, j.n);
            PairDesc d{};
            d.Ag = ag[wave[q]];
            d.Bg = bg[wave[q]];
            d.m = j.m;
            d.n = j.n;
            d.S = g.S;
            d.C = g.C;
            d.nwarps = g.nwarps;
            d.pm = (j.m - 1) - kPairRows * (g.S - 1);
            d.rec_rows = g.rec_rows;
            d.rec_off = rec_off;
            d.ring_off = ring_off;
            d.score = j.score;
            descs.push_back(d);
            for (uint32_t w = 0; w < g.nwarps; ++w) blocks.push_back(PairBlock{(uint32_t)q, w});
            rec_off += want ? (uint64_t)g.nwarps * g.rec_rows * 32u : 0;
            ring_off += (uint64_t)g.nwarps * g.C * 2u;
        }
        void *v = nullptr;
        const size_t dbytes = descs.size() * sizeof(PairDesc), bbytes = blocks.size() * sizeof(PairBlock);
        if ((rc = scratch(ctx, "bpair_desc", dbytes + bbytes + 16, &v))) return rc;
        {
            cudaError_t e = cudaMemcpyAsync(v, descs.data(), dbytes, cudaMemcpyHostToDevice, ctx->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync((char *)v + dbytes, blocks.data(), bbytes, cudaMemcpyHostToDevice, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the tables are host memory of this call
            if (e != cudaSuccess) return cuda_fail(ctx, e, "pair table upload");
        }
        L.pairs = (const PairDesc *)v;
        L.blocks = (const PairBlock *)((char *)v + dbytes);
        if ((rc = scratch(ctx, "bpair_ring", ring + 64, &v))) return rc;
        if (v != ctx->bits_ring || ctx->bits_epoch == 0xffffffffu) {
            // a new ring may hold anything, also tags of an earlier context:
            // clear it and start the epochs again
            const cudaError_t e = cudaMemsetAsync(v, 0, ring + 64, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "ring clear");
            ctx->bits_ring = v;
            ctx->bits_epoch = 0;
        }
        L.ring = (uint64_t *)v;
        L.epoch = ++ctx->bits_epoch;
        L.rec = nullptr;
        if (want) {
            if ((rc = scratch(ctx, "bpair_rec", rec + 16, &v))) return rc;
            L.rec = (uint4 *)v;
        }
        void *args[] = {&L};
        {
            LaunchTimer t(ctx, want ? "bpair_fill_ptr" : "bpair_fill");
            const cudaError_t e = cudaLaunchCooperativeKernel(pair_kernel(gen, want), dim3((uint32_t)blocks.size()),
                                                              dim3(32), args, 0, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "bit-sliced pair launch");
        }
        if (!want) continue;
        void *mv = nullptr, *nm = nullptr, *dt = nullptr;
        if ((rc = scratch(ctx, "bpair_moves", moves + 16, &mv))) return rc;
        if ((rc = scratch(ctx, "bpair_nmoves", wave.size() * 8 + 16, &nm))) return rc;
        std::vector<TraceTask> tts;
        uint64_t moff = 0;
        for (size_t q = 0; q < wave.size(); ++q) {
            const PairJob &j = jobs[wave[q]];
            const uint8_t *a = pool ? pool + j.a_off : (const uint8_t *)(uintptr_t)j.a_off;
            const uint8_t *b = pool ? pool + j.b_off : (const uint8_t *)(uintptr_t)j.b_off;
            tts.push_back(TraceTask{(const uint32_t *)(L.rec + descs[q].rec_off), descs[q].rec_rows, j.m, j.n,
                                    (uint8_t *)mv + moff, (uint64_t *)nm + q, a, b, j.cigar, j.cigar_len, kNoBand, 0,
                                    nullptr, nullptr});
            moff += (uint64_t)j.m + j.n + 16;
        }
        if (tts.size() > 1) {
            if ((rc = scratch(ctx, "bpair_tt", tts.size() * sizeof(TraceTask), &dt))) return rc;
            cudaError_t e = cudaMemcpyAsync(dt, tts.data(), tts.size() * sizeof(TraceTask), cudaMemcpyHostToDevice,
                                            ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "pair trace upload");
        }
        if ((rc = launch_trace_bits(ctx, tts.data(), tts.size() > 1 ? (const TraceTask *)dt : nullptr,
                                    (uint32_t)tts.size(), mflag)))
            return rc;
    }
    return NW_OK;
}

int bits_pair(nw_ctx *ctx, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n, const nw_scoring &sc,
              bool want, uint32_t mflag, int32_t *score, char *cigar, uint64_t *cigar_len) {
    const std::vector<PairJob> jobs{PairJob{(uint64_t)(uintptr_t)a2b, (uint64_t)(uintptr_t)b2b, m, n, score,
                                            want ? cigar : nullptr, want ? cigar_len : nullptr}};
    return bits_pairs(ctx, nullptr, jobs, sc, want, mflag);
}

}  // namespace nw
