// One long pair: the fill (a3/a4) spread over many warps.
//
// Work split.  Stripes of 32*R rows go to warps; lane k of a warp owns R
// consecutive rows.  At step t lane k updates a register block of R rows x C
// columns (C = 16/R, so the block's 2-bit pointers make exactly one 32-bit
// word) for column block q = t - k.  The block's top row arrives from lane
// k-1 by C warp shuffles, its left column and corner stay in registers; the
// dependency chain through a block runs along its anti-diagonal (R+C-1
// cells), and one shuffle latency is paid per C columns instead of per
// column.
//
// Handoffs.  The NW warps of a CTA own NW consecutive stripes.  A stripe's
// bottom row goes to the next warp through a ring in shared memory (Q
// columns; the producer publishes a head every KQ columns after a CTA-scope
// fence, the consumer a tail; both waits are bounded).  The first warp of a
// CTA fills its own ring: from B for stripe 0, else from the previous CTA's
// last warp, which writes its bottom row to global memory and releases a
// gpu-scope progress counter every GQ columns.  Lane 0's input reaches it
// through the rotation shuffle: lane 31 loads the ring block (after storing
// its own finished block) and shuffles it to lane 0 with everything else.
// CTAs take CTA-stripes round robin; the grid never exceeds the co-resident
// CTA count, so every wait ends (and all of them are bounded regardless).
//
// The cell update (W domain: prmt + DPX add-max + max) and the pointer
// encoding (bit0: diagonal is the maximum, bit1: vertical >= horizontal) are
// those of the other kernels (the pointer bits are computed from differences
// rather than with the predicate-returning DPX max, whose dependent latency
// is several times longer); the pointer word layout [stripe][lane][block]
// with bit 2*(c*R + r) for block row r, column c is the one the traceback
// reads.  The step loop runs in three phases (lanes starting, all lanes busy,
// lanes finishing) so the busy phase has no per-lane tests.
#include <algorithm>

#include "nw_internal.cuh"

namespace nw {

constexpr int kPairQ = 256;      // ring columns per warp
constexpr int kPairKQ = 32;      // ring flag granularity (columns)
constexpr int kPairGQ = 64;      // global progress granularity (columns)
constexpr int kPairMaxWarps = 8;

struct PairArgs {
    const uint8_t *a;
    const uint8_t *b;
    uint32_t m, n;
    uint32_t prof[4];
    int32_t gap;
    uint32_t S;          // stripes
    uint32_t bstride;    // words per global boundary row (>= NB*C, multiple of 64)
    uint32_t *bnd;       // global boundary rows: row g = bottom of group g (0-based columns)
    uint32_t *progress;  // per group: columns of its global row released
    uint32_t *ptr;       // pointer words of stripes s_ptr0.. (null: score only)
    uint32_t ncg;        // pointer words per lane row (>= NB)
    uint32_t s_ptr0;     // first stripe with pointer words in `ptr`
    uint32_t cs_lo, cs_hi;   // groups (CTA-stripes) to run
    const uint32_t *ncols;   // null, or a device word: only columns [0, *ncols) are needed
    uint32_t recompute;      // groups start from kept rows and write none
    int32_t *score;          // null: no score
    uint32_t *err;
};

__device__ __forceinline__ uint32_t vld(const volatile uint32_t *p) { return *p; }

// Bounded wait on a shared-memory counter written by another warp of the CTA.
__device__ __forceinline__ bool smem_wait_geq(const volatile uint32_t *flag, uint32_t target, uint32_t *err,
                                              uint32_t where) {
    if (vld(flag) >= target) return true;
    const uint64_t t0 = global_ns();
    uint32_t spins = 0;
    while (vld(flag) < target) {
        if ((++spins & 255u) == 0) {
            if (vld(err) != 0u) return false;
            if (global_ns() - t0 > kSpinNanos) {
                raise_error(err, NW_ERR_TIMEOUT, where);
                return false;
            }
        }
    }
    return true;
}

template <int N>
__device__ __forceinline__ void st_vec(uint32_t *dst, const uint32_t (&v)[N]) {
    if constexpr (N == 4) {
        *reinterpret_cast<uint4 *>(dst) = make_uint4(v[0], v[1], v[2], v[3]);
    } else if constexpr (N == 2) {
        *reinterpret_cast<uint2 *>(dst) = make_uint2(v[0], v[1]);
    } else {
#pragma unroll
        for (int c = 0; c < N; c += 4) *reinterpret_cast<uint4 *>(dst + c) = make_uint4(v[c], v[c + 1], v[c + 2], v[c + 3]);
    }
}

template <int N>
__device__ __forceinline__ void ld_vec(uint32_t (&v)[N], const uint32_t *src) {
    if constexpr (N == 4) {
        const uint4 q = *reinterpret_cast<const uint4 *>(src);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (N == 2) {
        const uint2 q = *reinterpret_cast<const uint2 *>(src);
        v[0] = q.x; v[1] = q.y;
    } else {
#pragma unroll
        for (int c = 0; c < N; c += 4) {
            const uint4 q = *reinterpret_cast<const uint4 *>(src + c);
            v[c] = q.x; v[c + 1] = q.y; v[c + 2] = q.z; v[c + 3] = q.w;
        }
    }
}

// Per-warp state of one stripe.
template <int R, int C>
struct LaneState {
    uint32_t prof[R];  // row profiles (byte d = s'(row base, d))
    int32_t Wl[R];     // left column of the next block
    int32_t last[R];   // values of column n-1 (for the score)
    int32_t corner;    // W(top-1, left column)
    uint32_t outW[C];  // bottom row of the last block (lane 31: ring input for lane 0)
    uint32_t outS[C];  // column selectors travelling with it
};

// One step of a lane: block q = t - lane.  inW/inS: the ring block of
// column block t (lane 0's top row).  CHECK: lanes may be idle (lead / drain
// phases) and the last block may be in this step.  Cells are visited along
// anti-diagonals of the R x C block so consecutive instructions are
// independent.
template <int R, int C, bool PTR, bool CHECK>
__device__ __forceinline__ void pair_block(LaneState<R, C> &st, const uint32_t (&inW)[C], const uint32_t (&inS)[C],
                                           int32_t q, uint32_t NB, uint32_t qL, uint32_t cL, int lane,
                                           uint32_t *prow) {
    int32_t up[C];
    uint32_t sel[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint32_t w = __shfl_up_sync(kFull, st.outW[c], 1);
        const uint32_t x = __shfl_up_sync(kFull, st.outS[c], 1);
        up[c] = (int32_t)(lane == 0 ? inW[c] : w);
        sel[c] = lane == 0 ? inS[c] : x;
    }
    if (CHECK && !(q >= 0 && q < (int32_t)NB)) return;
    // V[r][c] after the step; inputs: left column st.Wl, top row up, corner
    int32_t V[R][C];
    uint32_t code = 0;
#pragma unroll
    for (int k = 0; k < R + C - 1; ++k) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int c = k - r;
            if (c < 0 || c >= C) continue;
            const int32_t u = r ? V[r - 1][c] : up[c];
            const int32_t l = c ? V[r][c - 1] : st.Wl[r];
            const int32_t d = r ? (c ? V[r - 1][c - 1] : st.Wl[r - 1]) : (c ? up[c - 1] : st.corner);
            const int32_t sv = (int32_t)prmt(st.prof[r], 0u, sel[c]);
            if constexpr (PTR) {
                // plain maxes on the dependency chain; the two pointer bits
                // come from differences off the chain: bit0 = diagonal is the
                // maximum (W == d+s'), bit1 = vertical >= horizontal, which
                // when the diagonal loses is W == u
                const int32_t t1 = d + sv;
                const int32_t wv = max(t1, max(u, l));
                V[r][c] = wv;
                const uint32_t bits = 3u - (uint32_t)min(wv - t1, 1) - (uint32_t)min(2 * (wv - u), 2);
                code |= bits << (2 * (c * R + r));
            } else {
                V[r][c] = max(__viaddmax_s32(d, sv, l), u);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        st.outW[c] = (uint32_t)V[R - 1][c];
        st.outS[c] = sel[c];
    }
    if (CHECK && (uint32_t)q == qL) {
#pragma unroll
        for (int c = 0; c < C; ++c)
            if ((uint32_t)c == cL) {
#pragma unroll
                for (int r = 0; r < R; ++r) st.last[r] = V[r][c];
            }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) st.Wl[r] = V[r][C - 1];
    st.corner = up[C - 1];
    if constexpr (PTR) prow[q] = code;
}

template <int R, bool PTR>
__global__ void __launch_bounds__(kPairMaxWarps * 32, 1) k_pair(PairArgs p) {
    constexpr int C = 16 / R;
    constexpr uint32_t SH = 32u * R;
    constexpr uint32_t QB = kPairQ / C;   // ring capacity in blocks
    constexpr uint32_t KB = kPairKQ / C;  // blocks per chunk (flags and self-fill)
    __shared__ __align__(16) uint32_t ringW[kPairMaxWarps][kPairQ];
    __shared__ __align__(16) uint32_t ringS[kPairMaxWarps][kPairQ];
    __shared__ uint32_t head[kPairMaxWarps];  // blocks written into ring[w]
    __shared__ uint32_t tail[kPairMaxWarps];  // blocks of ring[w] consumed

    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int NW = blockDim.x >> 5;
    const int src = (lane + 31) & 31;  // rotation: lane 0 hears lane 31
    const uint32_t m = p.m;
    // recompute passes need only the columns left of the traceback's entry
    const uint32_t n = p.ncols ? min(p.n, *p.ncols) : p.n;
    if (n == 0) return;
    const uint32_t NB = (n + C - 1) / C;
    const uint32_t NBC = NB * C;
    const uint32_t CS = (p.S + NW - 1) / NW;
    const uint32_t sM = (m - 1) / SH, lM = ((m - 1) % SH) / R, rM = (m - 1) % R;
    const uint32_t qL = NB - 1, cL = (n - 1) % C;

    const uint32_t cs_end = min(CS, p.cs_hi);
    for (uint32_t cs = p.cs_lo + blockIdx.x; cs < cs_end; cs += gridDim.x) {
        if (lane == 0) {
            head[w] = 0;
            tail[w] = 0;
        }
        __syncthreads();
        const uint32_t s = cs * NW + w;
        if (s < p.S) {
            LaneState<R, C> st;
            {
                const uint32_t row0 = s * SH + lane * R;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t i = row0 + r;
                    const uint32_t cb = i < m ? base_at(p.a, i) : 0u;
                    st.prof[r] = cb == 0 ? p.prof[0] : cb == 1 ? p.prof[1] : cb == 2 ? p.prof[2] : p.prof[3];
                    st.Wl[r] = 0;
                    st.last[r] = 0;
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    st.outW[c] = 0;
                    st.outS[c] = 0;
                }
                st.corner = 0;
            }
            const bool self_fill = w == 0;
            const bool has_next = s + 1 < p.S;
            const bool out_ring = has_next && w + 1 < NW;
            const bool out_glob = has_next && w + 1 == NW && !p.recompute;
            const uint32_t *ginW = (self_fill && cs > 0) ? p.bnd + (size_t)(cs - 1) * 2 * p.bstride : nullptr;
            const uint32_t *ginS = ginW ? ginW + p.bstride : nullptr;
            uint32_t *goutW = out_glob ? p.bnd + (size_t)cs * 2 * p.bstride : nullptr;
            uint32_t *goutS = goutW ? goutW + p.bstride : nullptr;
            uint32_t *prow = PTR ? p.ptr + (size_t)((s - p.s_ptr0) * 32u + lane) * p.ncg : nullptr;
            const int nx = w + 1 < NW ? w + 1 : w;
            volatile uint32_t *my_head = head + w;
            volatile uint32_t *my_tail = tail + w;
            volatile uint32_t *nx_head = head + nx;
            volatile uint32_t *nx_tail = tail + nx;
            uint32_t *myW = ringW[w], *myS = ringS[w], *nxW = ringW[nx], *nxS = ringS[nx];

            // Self-fill of ring[0]: chunks of 32 columns, lane l holds column
            // 32k + l; written two chunks ahead of use.
            uint32_t stW = 0, stS = 0;
            bool ok = true;
            auto load_chunk = [&](uint32_t k) -> bool {
                const uint32_t col = 32u * k + lane;
                if (32u * k >= NBC) return true;
                if (ginW) {
                    int good = 1;
                    if (lane == 0) good = wait_geq(&p.progress[cs - 1], min(32u * k + 32u, NBC), p.err, s) ? 1 : 0;
                    good = __shfl_sync(kFull, good, 0);
                    if (!good) return false;
                    (void)ld_acquire(&p.progress[cs - 1]);
                    stW = __ldcg(ginW + col);
                    stS = __ldcg(ginS + col);
                } else {
                    stW = 0;  // grid row 0
                    stS = sext_selector(col < n ? base_at(p.b, col) : 0u);
                }
                return true;
            };
            auto put_chunk = [&](uint32_t k) {
                const uint32_t slot = (32u * k + lane) & (kPairQ - 1);
                myW[slot] = stW;
                myS[slot] = stS;
            };
            if (self_fill) {
                ok = load_chunk(0);
                put_chunk(0);
                ok = ok && load_chunk(1);
                put_chunk(1);
                ok = ok && load_chunk(2);
                __syncwarp();
            }

            // Chunk bookkeeping before steps [t, t+KB) (warp-uniform).
            auto chunk_begin = [&](uint32_t t) -> bool {
                if (self_fill) {
                    const uint32_t k = t / KB + 2;
                    put_chunk(k);
                    if (!load_chunk(k + 1)) return false;
                    __syncwarp();
                } else if (t < NB) {
                    if (!smem_wait_geq(my_head, min(t + KB, NB), p.err, 0x10000u + s)) return false;
                    __threadfence_block();
                }
                if (out_ring) {
                    // lane 31 will write blocks [t-31, t-31+KB): their slots must be free
                    const int32_t need = (int32_t)t - 31 + (int32_t)KB - (int32_t)QB;
                    if (need > 0 && !smem_wait_geq(nx_tail, (uint32_t)need, p.err, 0x20000u + s)) return false;
                }
                return true;
            };
            // After steps [t, t+KB): publish what lane 31 wrote / lane 31 read.
            auto chunk_end = [&](uint32_t t) {
                if (lane == 31) {
                    if (!self_fill) *my_tail = t + KB;
                    const int32_t done = min((int32_t)t + (int32_t)KB - 31, (int32_t)NB);
                    if (done > 0) {
                        if (out_ring) {
                            __threadfence_block();
                            *nx_head = (uint32_t)done;
                        } else if (out_glob) {
                            st_release(&p.progress[cs], (uint32_t)done * C);
                        }
                    }
                }
            };
            // Input block t for lane 0 (all lanes read it: a broadcast), and
            // lane 31 hands block t-31 on.
            auto ring_in = [&](uint32_t t, uint32_t (&iw)[C], uint32_t (&is)[C]) {
                const uint32_t slot = (t % QB) * C;
                ld_vec<C>(iw, myW + slot);
                ld_vec<C>(is, myS + slot);
            };
            auto lane31_out = [&](uint32_t t) {
                const int32_t q31 = (int32_t)t - 31;
                const bool valid = lane == 31 && q31 >= 0 && q31 < (int32_t)NB;
                if (out_ring) {
                    if (valid) {
                        st_vec<C>(nxW + ((uint32_t)q31 % QB) * C, st.outW);
                        st_vec<C>(nxS + ((uint32_t)q31 % QB) * C, st.outS);
                    }
                } else if (out_glob) {
                    if (valid) {
                        st_vec<C>(goutW + (uint32_t)q31 * C, st.outW);
                        st_vec<C>(goutS + (uint32_t)q31 * C, st.outS);
                    }
                }
            };

            const uint32_t T = NB + 31;
            // busy chunks: every lane active, none on the last block
            const uint32_t busy_end = NB >= 1 ? NB - 1 : 0;
            uint32_t t = 0;
            uint32_t inW[C], inS[C];
            while (ok && t < T) {
                if (!chunk_begin(t)) {
                    ok = false;
                    break;
                }
                if (t >= 32 && t + KB <= busy_end) {
                    ring_in(t, inW, inS);
#pragma unroll
                    for (uint32_t u = 0; u < KB; ++u) {
                        uint32_t nW[C], nS[C];
                        if (u + 1 < KB) ring_in(t + u + 1, nW, nS);
                        pair_block<R, C, PTR, false>(st, inW, inS, (int32_t)(t + u) - lane, NB, qL, cL, lane, prow);
                        lane31_out(t + u);
                        if (u + 1 < KB) {
#pragma unroll
                            for (int c = 0; c < C; ++c) {
                                inW[c] = nW[c];
                                inS[c] = nS[c];
                            }
                        }
                    }
                } else {
                    for (uint32_t u = 0; u < KB; ++u) {
                        ring_in(t + u, inW, inS);
                        pair_block<R, C, PTR, true>(st, inW, inS, (int32_t)(t + u) - lane, NB, qL, cL, lane, prow);
                        lane31_out(t + u);
                    }
                }
                chunk_end(t);
                t += KB;
            }
            if (ok && p.score && s == sM && (uint32_t)lane == lM) {
                int32_t wmn = 0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if ((uint32_t)r == rM) wmn = st.last[r];
                *p.score = wmn + p.gap * (int32_t)(m + n);
            }
        }
        __syncthreads();
    }
}

template <int R, bool PTR>
static int launch_pair_R(nw_ctx *ctx, PairArgs &pa, int nw) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair<R, PTR>, nw * 32, 0);
    if (occ < 1) occ = 1;
    const uint32_t CS = (pa.S + nw - 1) / nw;
    const uint32_t hi = std::min(CS, pa.cs_hi);
    if (pa.cs_lo >= hi) return NW_OK;
    uint32_t blocks = hi - pa.cs_lo;
    const uint32_t cap = (uint32_t)occ * (uint32_t)ctx->sm_count;  // co-resident
    if (blocks > cap) blocks = cap;
    LaunchTimer t(ctx, pa.recompute ? "fill_recompute" : PTR ? "fill_ptr" : "fill_score");
    k_pair<R, PTR><<<blocks, nw * 32, 0, ctx->stream>>>(pa);
    return NW_OK;
}

uint32_t pair_bstride(uint32_t n) { return ((n + 64 + 63) / 64) * 64; }  // W row then selector row

int launch_pair_fill(nw_ctx *ctx, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n, const Profile &pf,
                     const PairFill &f) {
    PairArgs pa{};
    pa.a = a2b;
    pa.b = b2b;
    pa.m = m;
    pa.n = n;
    for (int c = 0; c < 4; ++c) pa.prof[c] = pf.prof[c];
    pa.gap = pf.gap;
    const int R = f.R;
    const int nw = std::max(1, std::min(f.nw, kPairMaxWarps));
    pa.S = (m + 32u * R - 1) / (32u * R);
    pa.bstride = pair_bstride(n);
    pa.ptr = f.ptr ? f.ptr_words : nullptr;
    pa.ncg = f.ncg;
    pa.cs_lo = f.cs_lo;
    pa.cs_hi = f.cs_hi;
    pa.s_ptr0 = f.cs_lo * (uint32_t)nw;
    pa.ncols = f.ncols;
    pa.recompute = f.recompute ? 1u : 0u;
    pa.score = f.score;
    pa.err = ctx->d_err;
    int rc;
    void *v = nullptr;
    const uint32_t CS = (pa.S + nw - 1) / nw;
    pa.bnd = f.bnd;
    if (!pa.bnd && CS > 1) {
        if ((rc = scratch(ctx, "pair_bnd", (size_t)(CS - 1) * 2 * pa.bstride * 4, &v))) return rc;
        pa.bnd = (uint32_t *)v;
    }
    pa.progress = f.progress;
    if (!pa.progress) {
        if ((rc = scratch(ctx, "pair_progress", (size_t)CS * 4 + 16, &v))) return rc;
        pa.progress = (uint32_t *)v;
    }
    if (!f.recompute) cudaMemsetAsync(pa.progress, 0, (size_t)CS * 4, ctx->stream);
    switch (R * 2 + (f.ptr ? 1 : 0)) {
        case 4: return launch_pair_R<2, false>(ctx, pa, nw);
        case 5: return launch_pair_R<2, true>(ctx, pa, nw);
        case 8: return launch_pair_R<4, false>(ctx, pa, nw);
        case 9: return launch_pair_R<4, true>(ctx, pa, nw);
        case 16: return launch_pair_R<8, false>(ctx, pa, nw);
        case 17: return launch_pair_R<8, true>(ctx, pa, nw);
        default: return fail(ctx, NW_ERR_ARG, "unsupported rows per lane %d", R);
    }
}

}  // namespace nw
