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

#include "nw_bits.cuh"

namespace nw {

constexpr int kPairWarps = 4;        // most warps per CTA (one per scheduler)
constexpr uint32_t kPairRows = 31;   // rows per stripe (bits 0..30 of a word)
// Truth tables (from a = 0xF0, b = 0xCC, c = 0xAA) of the shallow update.
constexpr uint32_t kLutAndNotNot = lut(kA & ~kB & ~kC);  // a & !b & !c
constexpr uint32_t kLutAndNand = lut(kA & ~(kB & kC));   // a & !(b & c)
constexpr uint32_t kLutOrAndNot = lut((kA | kB) & ~kC);  // (a | b) & !c
constexpr uint32_t kLutXorAndNot = lut(kA ^ (kB & ~kC)); // a ^ (b & !c)

struct PairBitsArgs {
    const uint32_t *pl0, *pl1;  // planar sequences
    int64_t Ag, Bg;             // slots of a (rows) and b (columns)
    uint32_t m, n, S, C;        // stripes, chunks of 32 steps per stripe
    uint32_t nwarps;
    uint32_t pm;                // bit of row m in the last stripe
    uint4 *rec;                 // records [warp][rec_rows][32 lanes] (two steps each), or null
    uint32_t rec_rows;          // step pairs per warp: the last lane's steps and a walk tile's overhang
    uint64_t *ring;             // [warp][C][2] tagged outgoing words of lane 31
    uint32_t epoch;             // tag of this launch (never 0)
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
__global__ void __launch_bounds__(kPairWarps * 32, 1) k_bits_pair(PairBitsArgs p) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= p.nwarps) return;
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
    uint32_t S, C, nwarps, per_cta, blocks, rec_rows;
    uint64_t rec_bytes, ring_bytes;
};

PairGeom pair_geom(uint32_t m, uint32_t n, int sms) {
    PairGeom g;
    g.S = (m + kPairRows - 1) / kPairRows;
    g.C = (uint32_t)(((uint64_t)n + kPairRows - 1 + 31u) / 32u);  // steps 0 .. n + 29
    g.nwarps = (g.S + 31u) / 32u;
    // a warp per SM while they fit (no warp shares an SM's memory pipes or
    // instruction cache), else kPairWarps per SM
    g.per_cta = g.nwarps <= (uint32_t)sms ? 1u : (uint32_t)kPairWarps;
    g.blocks = (g.nwarps + g.per_cta - 1) / g.per_cta;
    // the last lane's steps end at warp step 32 (C + 31); a walk tile of 64
    // steps may start up to 63 steps before a stripe's last step
    g.rec_rows = 16u * (g.C + 33u);
    g.rec_bytes = (uint64_t)g.nwarps * g.rec_rows * 32u * 16u;
    g.ring_bytes = (uint64_t)g.nwarps * g.C * 16u + 64;
    return g;
}

bool env_on(const char *name) {
    const char *v = getenv(name);
    return v && *v && *v != '0';
}
}  // namespace

bool bits_pair_takes(nw_ctx *ctx, uint32_t m, uint32_t n, const nw_scoring &sc, bool want) {
    if (env_on("NW_PAIR_SCALAR") || !bits_scoring_ok(sc) || m == 0 || n == 0) return false;
    const char *mn = getenv("NW_BITS_PAIR_MIN");  // smallest side taken (test and sweep knob)
    const uint32_t min_side = mn ? (uint32_t)atoi(mn) : 64u;
    if (std::min(m, n) < min_side) return false;
    const PairGeom g = pair_geom(m, n, ctx->sm_count);
    if (g.blocks > (uint32_t)ctx->sm_count) return false;  // one CTA per SM is always co-resident
    uint64_t need = g.ring_bytes;
    if (want) need += g.rec_bytes + (uint64_t)m + n + 64;
    return need <= scratch_headroom(ctx, "bpair_rec");
}

int bits_pair(nw_ctx *ctx, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n, const nw_scoring &sc,
              bool want, uint32_t mflag, int32_t *score, char *cigar, uint64_t *cigar_len) {
    int rc;
    const PairGeom g = pair_geom(m, n, ctx->sm_count);
    PlaneSet ps;
    PairBitsArgs pa{};
    pa.Ag = ps.add((uint64_t)(uintptr_t)a2b, m);
    pa.Bg = ps.add((uint64_t)(uintptr_t)b2b, n);
    if ((rc = ps.launch(ctx, nullptr, "bpair"))) return rc;
    pa.pl0 = ps.pl0;
    pa.pl1 = ps.pl1;
    pa.m = m;
    pa.n = n;
    pa.S = g.S;
    pa.C = g.C;
    pa.nwarps = g.nwarps;
    pa.pm = (m - 1) - kPairRows * (g.S - 1);
    pa.rec_rows = g.rec_rows;
    pa.score = score;
    pa.gap = sc.gap;
    pa.err = ctx->d_err;
    const int32_t sm = sc.match - 2 * sc.gap, sx = sc.mismatch - 2 * sc.gap;
    pa.g.M1 = (sm & 2) ? ~0u : 0u;
    pa.g.M0 = (sm & 1) ? ~0u : 0u;
    pa.g.X1 = (sx & 2) ? ~0u : 0u;
    pa.g.X0 = (sx & 1) ? ~0u : 0u;
    const bool gen = !(sm == 3 && sx == 1);
    void *v = nullptr;
    if ((rc = scratch(ctx, "bpair_ring", g.ring_bytes, &v))) return rc;
    if (v != ctx->bits_ring || ctx->bits_epoch == 0xffffffffu) {
        // a new ring may hold anything, also tags of an earlier context:
        // clear it and start the epochs again
        const cudaError_t e = cudaMemsetAsync(v, 0, g.ring_bytes, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "ring clear");
        ctx->bits_ring = v;
        ctx->bits_epoch = 0;
    }
    pa.ring = (uint64_t *)v;
    pa.epoch = ++ctx->bits_epoch;
    if (want) {
        if ((rc = scratch(ctx, "bpair_rec", g.rec_bytes, &v))) return rc;
        pa.rec = (uint4 *)v;
    }
    void *args[] = {&pa};
    const void *fn = want ? (gen ? (const void *)k_bits_pair<true, true> : (const void *)k_bits_pair<false, true>)
                          : (gen ? (const void *)k_bits_pair<true, false> : (const void *)k_bits_pair<false, false>);
    {
        LaunchTimer t(ctx, want ? "bpair_fill_ptr" : "bpair_fill");
        const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(g.blocks), dim3(g.per_cta * 32), args, 0,
                                                          ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "bit-sliced pair launch");
    }
    if (!want) return NW_OK;
    void *mv = nullptr, *nm = nullptr;
    if ((rc = scratch(ctx, "moves", (size_t)m + n + 16, &mv))) return rc;
    if ((rc = scratch(ctx, "nmoves", 16, &nm))) return rc;
    TraceTask tt{(const uint32_t *)pa.rec, g.rec_rows, m, n, (uint8_t *)mv, (uint64_t *)nm, a2b, b2b, cigar,
                 cigar_len, kNoBand, 0, nullptr, nullptr};
    return launch_trace_bits(ctx, &tt, nullptr, 1, mflag);
}

}  // namespace nw
