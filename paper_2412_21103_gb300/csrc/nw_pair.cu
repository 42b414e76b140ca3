// One long pair: the fill (a3/a4) spread over many warps.  It computes the
// Sec. 2.3 recurrence (Eq. 1, read as in standard NW: the match/mismatch
// score on the diagonal only, the gap on vertical and horizontal moves) from
// the Sec. 2.2 boundary, in the W domain of nw_internal.cuh.  Sec. 3.1
// parallelises the same fill with one thread per cell that polls its
// neighbours; here dependencies are met by construction instead.
//
// Work split.  Stripes of 32*R rows go to warps; lane k of a warp owns R
// consecutive rows.  At step t lane k updates a register block of R rows x C
// columns for column block q = t - k.  The block's top row arrives from lane
// k-1 by C warp shuffles, its left column and corner stay in registers, and
// the column selectors (which byte of the row profile a column's base picks)
// come from a per-column table that stays in L1.  The dependency chain
// through a block runs along its anti-diagonals (R+C-1 cells), and one
// shuffle latency is paid per C columns instead of per column.
//
// Handoffs.  The NW compute warps of a CTA own NW consecutive stripes (a
// "group").  A stripe's bottom row goes to the next warp through a ring in
// shared memory (Q columns; the producer publishes a head every KQ columns
// after a CTA-scope fence, the consumer a tail; both waits are bounded).
// One more warp per CTA, the courier, does all global-memory traffic: it
// fills the first warp's ring with the previous group's bottom row (zeros
// for grid row 0) as that group releases it, and drains the last warp's
// ring to global memory, releasing a gpu-scope progress counter; its L2
// round trips stall no compute warp.  Lane 0's input reaches it from the
// ring, broadcast to the warp; lane 31 stores its finished block into the
// next ring.  CTAs take groups round robin; the grid never exceeds the
// co-resident CTA count, so every wait ends (and all of them are bounded
// regardless).
//
// The kept group rows double as the checkpoints of the recompute traceback:
// a launch may run a range of groups, each starting from the previous
// group's kept row, write no rows, and compute only the columns left of a
// device-resident column count.
//
// The cell update is W = max(d + s', max(u, l)) in the W domain (one prmt,
// one max, one DPX add-max); with pointers each cell also appends the sign
// bits of d + s' - max(u, l) and u - l (ptr_append), and words of R rows x
// 16/R columns are stored [stripe][lane][word].  The step loop runs in three
// phases (lanes starting, all lanes busy, lanes finishing) so the busy phase
// has no per-lane tests.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "nw_internal.cuh"

namespace nw {

constexpr int kPairQ = 256;   // ring columns per warp
constexpr int kPairKQ = 16;   // ring flag granularity (columns)
constexpr int kPairMaxWarps = 8;

struct PairArgs {
    const uint8_t *a;
    const uint32_t *sel;  // column selectors (sext_selector of each base of B), >= NB*C entries
    uint32_t m, n;
    uint32_t prof[4];
    int32_t gap;
    uint32_t S;              // stripes
    uint32_t bstride;        // words per global group row (>= NB*C)
    uint32_t *bnd;           // global rows: row g = bottom W row of group g (0-based columns)
    uint32_t *progress;      // per group: columns of its global row released
    uint32_t *ptr;           // pointer words of stripes s_ptr0.. (null: score only)
    uint32_t ncg;            // pointer words per lane row (>= NB*C/(16/R))
    uint32_t s_ptr0;         // first stripe with pointer words in `ptr`
    uint32_t cs_lo, cs_hi;   // groups (CTA-stripes) to run
    const uint32_t *ncols;   // null, or a device word: only columns [0, *ncols) are needed
    uint32_t recompute;      // groups start from kept rows and write none
    uint32_t keep_rows;      // every group's bottom row must reach global memory (checkpoints)
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

// Shared memory at cluster scope.  Ring counters and ring data may belong to
// this CTA or to a neighbour CTA of the same thread-block cluster; every
// access goes through a 32-bit shared::cluster address (mapa of the local
// address to a CTA rank), so one instruction serves both cases.
__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_map(const void *local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ uint32_t ld_acq_cl(uint32_t a) {
    uint32_t v;
    asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_cl(uint32_t a, uint32_t v) {
    asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Predicated vector store to a shared::cluster address (no branch).
template <int N>
__device__ __forceinline__ void st_cl_if(bool p, uint32_t a, const uint32_t (&v)[N]) {
    if constexpr (N == 2) {
        asm volatile("{.reg .pred q; setp.ne.b32 q, %0, 0; @q st.shared::cluster.v2.u32 [%1], {%2, %3};}" ::"r"((uint32_t)p),
                     "r"(a), "r"(v[0]), "r"(v[1])
                     : "memory");
    } else {
#pragma unroll
        for (int c = 0; c < N; c += 4)
            asm volatile(
                "{.reg .pred q; setp.ne.b32 q, %0, 0; @q st.shared::cluster.v4.u32 [%1], {%2, %3, %4, %5};}" ::"r"(
                    (uint32_t)p),
                "r"(a + 16u * (c / 4)), "r"(v[c]), "r"(v[c + 1]), "r"(v[c + 2]), "r"(v[c + 3])
                : "memory");
    }
}
// Bounded wait on a shared::cluster counter (acquire: the ring data written
// before its release is visible afterwards).
__device__ __forceinline__ bool cl_wait_geq(uint32_t a, uint32_t target, uint32_t *err, uint32_t where) {
    if (ld_acq_cl(a) >= target) return true;
    const uint64_t t0 = global_ns();
    uint32_t spins = 0;
    while (ld_acq_cl(a) < target) {
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
    } else if constexpr (N == 1) {
        *dst = v[0];
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
    } else if constexpr (N == 1) {
        v[0] = *src;
    } else {
#pragma unroll
        for (int c = 0; c < N; c += 4) {
            const uint4 q = *reinterpret_cast<const uint4 *>(src + c);
            v[c] = q.x; v[c + 1] = q.y; v[c + 2] = q.z; v[c + 3] = q.w;
        }
    }
}

// Predicated vector store through a generic address: one store instruction
// with a predicate, no branch (a lane-divergent branch around the store
// costs a warp tens of cycles per step).
template <int N>
__device__ __forceinline__ void st_vec_if(bool p, uint32_t *dst, const uint32_t (&v)[N]) {
    if constexpr (N == 4) {
        asm volatile("{.reg .pred q; setp.ne.b32 q, %0, 0; @q st.v4.u32 [%1], {%2, %3, %4, %5};}" ::"r"((uint32_t)p),
                     "l"(dst), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
                     : "memory");
    } else if constexpr (N == 2) {
        asm volatile("{.reg .pred q; setp.ne.b32 q, %0, 0; @q st.v2.u32 [%1], {%2, %3};}" ::"r"((uint32_t)p), "l"(dst),
                     "r"(v[0]), "r"(v[1])
                     : "memory");
    } else {
#pragma unroll
        for (int c = 0; c < N; c += 4)
            asm volatile("{.reg .pred q; setp.ne.b32 q, %0, 0; @q st.v4.u32 [%1], {%2, %3, %4, %5};}" ::"r"((uint32_t)p),
                         "l"(dst + c), "r"(v[c]), "r"(v[c + 1]), "r"(v[c + 2]), "r"(v[c + 3])
                         : "memory");
    }
}

// Column selectors of block q (read-only path: the table stays in L1).
template <int C>
__device__ __forceinline__ void ld_sel(uint32_t (&v)[C], const uint32_t *tab, uint32_t q) {
    if constexpr (C == 4) {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(tab) + q);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else if constexpr (C == 2) {
        const uint2 x = __ldg(reinterpret_cast<const uint2 *>(tab) + q);
        v[0] = x.x; v[1] = x.y;
    } else {
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = __ldg(tab + q * C + c);
    }
}

// Per-warp state of one stripe.
template <int R, int C>
struct LaneState {
    uint32_t prof[R];  // row profiles (byte d = s'(row base, d))
    int32_t Wl[R];     // left column of the next block
    int32_t last[R];   // values of column n-1 (for the score)
    int32_t corner;    // W(top-1, left column)
    uint32_t outW[C];  // bottom row of the last block (lane 31: the next stripe's input)
    uint32_t accL, accH;  // pointer bits of the word being filled
};

// One step of a lane: block q = t - lane.  inW: the ring block of column
// block t (lane 0's top row); sel: the selectors of block q.  CHECK: lanes
// may be idle (lead / drain phases) and the last block may be in this step.
// Cells are visited along anti-diagonals of the R x C block so consecutive
// instructions are independent.
template <int R, int C, bool PTR, bool CHECK>
__device__ __forceinline__ void pair_block(LaneState<R, C> &st, const uint32_t (&inW)[C], const uint32_t (&sel)[C],
                                           int32_t q, uint32_t NB, uint32_t qL, uint32_t cL, int lane,
                                           uint32_t *prow) {
    constexpr uint32_t SPW = (16u / R) / C;  // steps per pointer word
    int32_t up[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint32_t w = __shfl_up_sync(kFull, st.outW[c], 1);
        up[c] = (int32_t)(lane == 0 ? inW[c] : w);
    }
    if (CHECK && !(q >= 0 && q < (int32_t)NB)) return;
    int32_t V[R][C];
    int32_t DL[R][C], DH[R][C];
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
            const int32_t m2 = max(u, l);
            V[r][c] = __viaddmax_s32(d, sv, m2);
            if constexpr (PTR) {
                DL[r][c] = d + sv - m2;  // < 0: the diagonal candidate loses
                DH[r][c] = u - l;        // < 0: horizontal beats vertical
            }
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) st.outW[c] = (uint32_t)V[R - 1][c];
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
    if constexpr (PTR) {
        // two independent chains of funnel shifts, cells in word order
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                st.accL = ptr_append(st.accL, DL[r][c]);
                st.accH = ptr_append(st.accH, DH[r][c]);
            }
        const uint32_t qq = (uint32_t)q;
        if (SPW == 1 || qq % SPW == SPW - 1) {
            prow[qq / SPW] = ptr_word(st.accL, st.accH);
        } else if (CHECK && qq == NB - 1) {
            const uint32_t miss = (SPW - 1 - qq % SPW) * R * C;  // the row's last word is short
            prow[qq / SPW] = ptr_word(st.accL << miss, st.accH << miss);
        }
    }
}

// The courier warp of a CTA: all global-memory traffic of the group's rows.
// Incoming (do_in): the previous group's kept bottom row (or the zeros of
// grid row 0) into ring 0, published by head[0] as the producer releases it.
// Outgoing (do_out): the last compute warp's bottom row from ring NW to
// global memory, released every few chunks.  The compute warps only ever
// wait on shared-memory counters; the round trips to L2 stall this warp.
template <int C>
__device__ __forceinline__ void pair_courier(const PairArgs &p, uint32_t cs, uint32_t NW, uint32_t NB, bool do_in,
                                             bool do_out, uint32_t (*ringW)[kPairQ], uint32_t *head, uint32_t *tail,
                                             uint32_t me) {
    constexpr uint32_t QB = kPairQ / C;
    constexpr uint32_t KB = kPairKQ / C;
    constexpr uint32_t MAXB = 8 * KB;  // blocks moved per step of the loop (128 columns)
    const int lane = threadIdx.x & 31;
    const bool in_glob = do_in && cs > 0;
    const uint32_t *gin = in_glob ? p.bnd + (size_t)(cs - 1) * p.bstride : nullptr;
    uint32_t *gout = do_out ? p.bnd + (size_t)cs * p.bstride : nullptr;
    (void)me;  // (the courier's rings are this CTA's: CTA-scope ordering)
    volatile uint32_t *v_head = head, *v_tail = tail;
    uint32_t delivered = do_in ? 0u : NB, forwarded = do_out ? 0u : NB;
    uint32_t avail_in = in_glob ? 0u : NB * C;  // columns released upstream (as last seen)
    uint64_t t_moved = global_ns();
    uint32_t idle = 0;
    while (delivered < NB || forwarded < NB) {
        bool moved = false;
        if (delivered < NB) {
            uint32_t next = min(delivered + MAXB, NB);
            next = min(next, vld(v_tail) + QB);  // ring 0 space
            if (in_glob && avail_in < next * C && avail_in < NB * C) {
                uint32_t v = 0;
                if (lane == 0) v = ld_acquire(&p.progress[cs - 1]);
                avail_in = __shfl_sync(kFull, v, 0);
            }
            next = min(next, avail_in / C);
            if (next > delivered) {
                if (in_glob) (void)ld_acquire(&p.progress[cs - 1]);  // every lane's loads after the flag
#pragma unroll
                for (uint32_t k = 0; k < MAXB * C / 32; ++k) {
                    const uint32_t col = delivered * C + k * 32u + lane;
                    if (col < next * C) ringW[0][col % kPairQ] = in_glob ? __ldcg(gin + col) : 0u;
                }
                __syncwarp();
                __threadfence_block();
                if (lane == 0) v_head[0] = next;
                delivered = next;
                moved = true;
            }
        }
        if (forwarded < NB) {
            const uint32_t avail = vld(v_head + NW);
            if (avail > forwarded) {
                __threadfence_block();
                const uint32_t upto = min(avail, forwarded + MAXB);
                uint32_t v[MAXB * C / 32];
#pragma unroll
                for (uint32_t k = 0; k < MAXB * C / 32; ++k) {
                    const uint32_t col = forwarded * C + k * 32u + lane;
                    v[k] = col < upto * C ? ringW[NW][col % kPairQ] : 0u;
                }
                __syncwarp();
                if (lane == 0) v_tail[NW] = upto;  // the slots are free once read
#pragma unroll
                for (uint32_t k = 0; k < MAXB * C / 32; ++k) {
                    const uint32_t col = forwarded * C + k * 32u + lane;
                    if (col < upto * C) __stcg(gout + col, v[k]);
                }
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&p.progress[cs], upto * C);
                forwarded = upto;
                moved = true;
            }
        }
        if (moved) {
            idle = 0;
            t_moved = global_ns();
        } else {
            if (vld(p.err) != 0u) break;
            if ((++idle & 63u) == 0 && global_ns() - t_moved > kSpinNanos) {
                if (lane == 0) raise_error(p.err, NW_ERR_TIMEOUT, 0x30000u + cs);
                break;
            }
            __nanosleep(20);
        }
    }
}

// CLS: CTAs per thread-block cluster (1: no cluster).  With clusters the
// groups of one cluster are consecutive and hand their rows over through
// distributed shared memory: the last compute warp of rank r stores its
// bottom row straight into ring 0 of rank r+1 and releases rank r+1's
// head[0]; rank r+1's first warp returns its consumption into rank r's
// `tail_rem`.  Only the first and last rank of a cluster use the courier.
template <int R, int C, bool PTR, int CLS>
__global__ void __launch_bounds__((kPairMaxWarps + 1) * 32, 1) k_pair(PairArgs p) {
    constexpr uint32_t SH = 32u * R;
    constexpr uint32_t QB = kPairQ / C;   // ring capacity in blocks
    constexpr uint32_t KB = kPairKQ / C;  // blocks per chunk (flags)
    // ring w < NW: input of compute warp w (ring 0 filled by the courier or
    // by the previous rank); ring NW: output of the last compute warp,
    // drained by the courier
    __shared__ __align__(16) uint32_t ringW[kPairMaxWarps + 1][kPairQ];
    __shared__ uint32_t head[kPairMaxWarps + 1];  // blocks written into ring[w]
    __shared__ uint32_t tail[kPairMaxWarps + 1];  // blocks of ring[w] consumed
    __shared__ uint32_t tail_rem;                 // blocks of the next rank's ring 0 consumed

    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int NW = (int)(blockDim.x >> 5) - 1;  // compute warps; warp NW is the courier
    const uint32_t m = p.m;
    // recompute passes need only the columns left of the traceback's entry
    const uint32_t n = p.ncols ? min(p.n, *p.ncols) : p.n;
    if (n == 0) return;  // (uniform over the grid: every CTA returns)
    const uint32_t NB = (n + C - 1) / C;
    const uint32_t CS = (p.S + NW - 1) / NW;
    const uint32_t sM = (m - 1) / SH, lM = ((m - 1) % SH) / R, rM = (m - 1) % R;
    const uint32_t qL = NB - 1, cL = (n - 1) % C;
    const uint32_t me = CLS > 1 ? cl_rank() : 0u;
    const uint32_t cs_end = min(CS, p.cs_hi);
    const uint32_t first = CLS > 1 ? cl_id() * CLS : blockIdx.x;
    const uint32_t stride = CLS > 1 ? cl_count() * CLS : gridDim.x;

    for (uint32_t base = p.cs_lo + first; base < cs_end; base += stride) {
        const uint32_t cs = base + me;  // this CTA's group (past cs_end: idle this round)
        const bool active = cs < cs_end;
        if (lane == 0) {
            head[w] = 0;
            tail[w] = 0;
            if (w == 0) tail_rem = 0;
        }
        __syncthreads();
        if (CLS > 1) cluster_sync();  // every rank reset before any remote write
        // hand-overs inside the cluster (never in recompute passes: there
        // every group starts from its kept row)
        const bool in_dsm = CLS > 1 && me > 0 && active && !p.recompute;
        const bool next_here = CLS > 1 && me + 1 < CLS && cs + 1 < cs_end;
        const uint32_t last_s = min((cs + 1) * NW, p.S) - 1;
        const bool out_any = active && !p.recompute && last_s + 1 < p.S;
        const bool out_dsm = out_any && next_here;
        const uint32_t s = cs * NW + w;
        if (w == NW) {
            if (active) pair_courier<C>(p, cs, NW, NB, !in_dsm, out_any && !out_dsm, ringW, head, tail, me);
        } else if (active && s < p.S) {
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
                for (int c = 0; c < C; ++c) st.outW[c] = 0;
                st.corner = 0;
                st.accL = 0;
                st.accH = 0;
            }
            const bool has_next = s + 1 < p.S;
            const bool last_w = w + 1 == NW;
            // output: ring w+1 of this CTA, ring NW (the courier's), or ring 0
            // of the next rank (not in recompute passes)
            const bool out_ring = has_next && (!last_w || out_any);
            const bool remote_out = last_w && out_dsm;
            uint32_t *prow = PTR ? p.ptr + (size_t)((s - p.s_ptr0) * 32u + lane) * p.ncg : nullptr;
            // Same-CTA rings: volatile counters and CTA-scope fences.  The ring
            // to / from a neighbour rank: shared::cluster addresses with
            // cluster-scope release / acquire.
            const bool remote_in = w == 0 && in_dsm;
            volatile uint32_t *my_head = head + w;
            volatile uint32_t *my_tail = tail + w;
            volatile uint32_t *nx_head = head + w + 1;
            volatile uint32_t *nx_tail = tail + w + 1;
            uint32_t *nxW = ringW[w + 1];
            const uint32_t a_my_head = cl_map(head + w, me);
            const uint32_t a_rem_tail = remote_in ? cl_map(&tail_rem, me - 1) : 0u;
            const uint32_t a_nx_head = remote_out ? cl_map(head, me + 1) : 0u;
            const uint32_t a_nx_tail = cl_map(&tail_rem, me);
            const uint32_t a_nx_ring = remote_out ? cl_map(ringW[0], me + 1) : 0u;
            const uint32_t *myW = ringW[w];
            bool ok = true;

            // Chunk bookkeeping before steps [t, t+KB) (warp-uniform).
            auto chunk_begin = [&](uint32_t t) -> bool {
                if (t < NB) {
                    if (remote_in) {
                        if (!cl_wait_geq(a_my_head, min(t + KB, NB), p.err, 0x10000u + s)) return false;
                    } else {
                        if (!smem_wait_geq(my_head, min(t + KB, NB), p.err, 0x10000u + s)) return false;
                        __threadfence_block();
                    }
                }
                if (out_ring) {
                    // lane 31 will write blocks [t-31, t-31+KB): their slots must be free
                    const int32_t need = (int32_t)t - 31 + (int32_t)KB - (int32_t)QB;
                    if (need > 0) {
                        const bool ok2 = remote_out ? cl_wait_geq(a_nx_tail, (uint32_t)need, p.err, 0x20000u + s)
                                                    : smem_wait_geq(nx_tail, (uint32_t)need, p.err, 0x20000u + s);
                        if (!ok2) return false;
                    }
                }
                return true;
            };
            // After steps [t, t+KB): publish what lane 31 wrote / what was read.
            auto chunk_end = [&](uint32_t t) {
                if (lane == 31) {
                    if (remote_in) st_rel_cl(a_rem_tail, t + KB);
                    else *my_tail = t + KB;
                    const int32_t done = min((int32_t)t + (int32_t)KB - 31, (int32_t)NB);
                    if (out_ring && done > 0) {
                        if (remote_out) {
                            st_rel_cl(a_nx_head, (uint32_t)done);
                        } else {
                            __threadfence_block();
                            *nx_head = (uint32_t)done;
                        }
                    }
                }
            };
            // Input block t for lane 0 (all lanes read it: a broadcast).
            auto ring_in = [&](uint32_t t, uint32_t (&iw)[C]) { ld_vec<C>(iw, myW + (t % QB) * C); };

            // The step loop, instantiated for a local or a remote output ring
            // (lane 31's predicated store; no branch per step).
            auto run = [&](auto remote_tag) {
                constexpr bool RO = decltype(remote_tag)::value;
                auto lane31_out = [&](uint32_t t) {
                    const int32_t q31 = (int32_t)t - 31;
                    const bool valid = out_ring && lane == 31 && q31 >= 0 && q31 < (int32_t)NB;
                    const uint32_t qv = valid ? (uint32_t)q31 : 0u;
                    if constexpr (RO) st_cl_if<C>(valid, a_nx_ring + (qv % QB) * C * 4u, st.outW);
                    else st_vec_if<C>(valid, nxW + (qv % QB) * C, st.outW);
                };
                const uint32_t T = NB + 31;
                // busy chunks: every lane active, none on the last block
                const uint32_t busy_end = NB >= 1 ? NB - 1 : 0;
                uint32_t t = 0;
                uint32_t inW[C], sel[C];
                while (ok && t < T) {
                    if (!chunk_begin(t)) {
                        ok = false;
                        break;
                    }
                    if (t >= 32 && t + KB <= busy_end) {
                        // selectors two steps ahead (an L1 miss costs more than a step)
                        uint32_t sel1[C];
                        ring_in(t, inW);
                        ld_sel<C>(sel, p.sel, t - (uint32_t)lane);
                        ld_sel<C>(sel1, p.sel, t + 1 - (uint32_t)lane);
#pragma unroll
                        for (uint32_t u = 0; u < KB; ++u) {
                            uint32_t nW[C], nS[C];
                            if (u + 1 < KB) ring_in(t + u + 1, nW);
                            if (u + 2 < KB) ld_sel<C>(nS, p.sel, t + u + 2 - (uint32_t)lane);
                            pair_block<R, C, PTR, false>(st, inW, sel, (int32_t)(t + u) - lane, NB, qL, cL, lane,
                                                         prow);
                            lane31_out(t + u);
#pragma unroll
                            for (int c = 0; c < C; ++c) {
                                if (u + 1 < KB) inW[c] = nW[c];
                                sel[c] = sel1[c];
                                if (u + 2 < KB) sel1[c] = nS[c];
                            }
                        }
                    } else {
                        for (uint32_t u = 0; u < KB; ++u) {
                            ring_in(t + u, inW);
                            const int32_t q = (int32_t)(t + u) - lane;
                            ld_sel<C>(sel, p.sel, (uint32_t)min(max(q, 0), (int32_t)NB - 1));
                            pair_block<R, C, PTR, true>(st, inW, sel, q, NB, qL, cL, lane, prow);
                            lane31_out(t + u);
                        }
                    }
                    chunk_end(t);
                    t += KB;
                }
            };
            if (CLS > 1 && remote_out) run(std::true_type{});
            else run(std::false_type{});
            if (ok && p.score && s == sM && (uint32_t)lane == lM) {
                int32_t wmn = 0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if ((uint32_t)r == rM) wmn = st.last[r];
                *p.score = wmn + p.gap * (int32_t)(m + n);
            }
        }
        __syncthreads();
        if (CLS > 1) cluster_sync();  // no rank resets while a neighbour still reads or writes it
    }
}

// Column selectors of B: entry j = sext_selector(B_j), zero-code past n.
__global__ void k_selectors(const uint8_t *b, uint32_t n, uint32_t count, uint32_t *sel) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x)
        sel[j] = sext_selector(j < n ? base_at(b, j) : 0u);
}

// Cluster launch of CLS CTAs per cluster; grid = the resident clusters (or
// fewer), so every wait across clusters ends.  Returns 1 (nothing launched)
// when the cluster shape cannot be scheduled.
template <int R, int C, bool PTR, int CLS>
static int launch_pair_cl(nw_ctx *ctx, PairArgs &pa, int nw, uint32_t groups) {
    auto kern = k_pair<R, C, PTR, CLS>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CLS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.blockDim = dim3((unsigned)(nw + 1) * 32u);
    cfg.stream = ctx->stream;
    // unused dynamic shared memory so that each SM takes one CTA of the
    // cluster (the scheduler would otherwise stack several on one SM, whose
    // compute warps then share schedulers)
    int pad_kb = 110;
    if (const char *e = getenv("NW_PAIR_CL_PAD")) pad_kb = atoi(e);
    cfg.dynamicSmemBytes = (size_t)pad_kb * 1024;
    if (pad_kb > 0 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.dynamicSmemBytes) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    uint32_t want = (groups + CLS - 1) / CLS;
    cfg.gridDim = dim3(want * CLS);
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        return 1;
    }
    if (want > (uint32_t)ncl) want = (uint32_t)ncl;
    cfg.gridDim = dim3(want * CLS);
    cudaError_t e;
    {
        LaunchTimer t(ctx, PTR ? "fill_ptr" : "fill_score");
        e = cudaLaunchKernelEx(&cfg, kern, pa);
    }
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "cluster launch");
}

template <int R, int C, bool PTR>
static int launch_pair_R(nw_ctx *ctx, PairArgs &pa, int nw) {
    const uint32_t CS = (pa.S + nw - 1) / nw;
    const uint32_t hi = std::min(CS, pa.cs_hi);
    if (pa.cs_lo >= hi) return NW_OK;
    const uint32_t groups = hi - pa.cs_lo;
    // Optional (NW_PAIR_CLUSTER = 2, 4 or 8): consecutive groups in one
    // thread-block cluster hand rows over through distributed shared memory.
    // Measured on GB300 it is slower than the courier path (32k x 32k: 6.6
    // vs 4.6 ms): the cluster-scope release that publishes each chunk also
    // waits for the warp's outstanding global pointer stores.  Never for
    // recompute passes or checkpoint fills (every group's row must reach
    // global memory there).
    int cls = 1;
    if (const char *e = getenv("NW_PAIR_CLUSTER")) cls = atoi(e);
    if (pa.recompute || pa.keep_rows || groups < 2) cls = 1;
    int rc = 1;
    if (cls == 8) rc = launch_pair_cl<R, C, PTR, 8>(ctx, pa, nw, groups);
    else if (cls == 4) rc = launch_pair_cl<R, C, PTR, 4>(ctx, pa, nw, groups);
    else if (cls == 2) rc = launch_pair_cl<R, C, PTR, 2>(ctx, pa, nw, groups);
    if (rc != 1) return rc;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair<R, C, PTR, 1>, (nw + 1) * 32, 0);
    if (occ < 1) occ = 1;
    uint32_t blocks = groups;
    const uint32_t cap = (uint32_t)occ * (uint32_t)ctx->sm_count;  // co-resident
    if (blocks > cap) blocks = cap;
    LaunchTimer t(ctx, pa.recompute ? "fill_recompute" : PTR ? "fill_ptr" : "fill_score");
    k_pair<R, C, PTR, 1><<<blocks, (nw + 1) * 32, 0, ctx->stream>>>(pa);
    return NW_OK;
}

uint32_t pair_bstride(uint32_t n) { return ((n + 64 + 63) / 64) * 64; }

int launch_pair_fill(nw_ctx *ctx, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n, const Profile &pf,
                     const PairFill &f) {
    PairArgs pa{};
    pa.a = a2b;
    pa.m = m;
    pa.n = n;
    for (int c = 0; c < 4; ++c) pa.prof[c] = pf.prof[c];
    pa.gap = pf.gap;
    const int R = f.R, C = f.C;
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
    pa.keep_rows = f.keep_rows ? 1u : 0u;
    pa.score = f.score;
    pa.err = ctx->d_err;
    int rc;
    void *v = nullptr;
    const uint32_t CS = (pa.S + nw - 1) / nw;
    pa.bnd = f.bnd;
    if (!pa.bnd && CS > 1) {
        if ((rc = scratch(ctx, "pair_bnd", (size_t)(CS - 1) * pa.bstride * 4, &v))) return rc;
        pa.bnd = (uint32_t *)v;
    }
    pa.progress = f.progress;
    if (!pa.progress) {
        if ((rc = scratch(ctx, "pair_progress", (size_t)CS * 4 + 16, &v))) return rc;
        pa.progress = (uint32_t *)v;
    }
    if (!f.recompute) cudaMemsetAsync(pa.progress, 0, (size_t)CS * 4, ctx->stream);
    pa.sel = f.sel;
    if (!pa.sel) {
        const uint32_t count = pa.bstride;  // >= NB*C for every C
        if ((rc = scratch(ctx, "pair_sel", (size_t)count * 4, &v))) return rc;
        LaunchTimer t(ctx, "selectors");
        k_selectors<<<(count + 255) / 256, 256, 0, ctx->stream>>>(b2b, n, count, (uint32_t *)v);
        pa.sel = (const uint32_t *)v;
    }
    switch (R * 100 + C * 10 + (f.ptr ? 1 : 0)) {
        case 220: return launch_pair_R<2, 2, false>(ctx, pa, nw);
        case 221: return launch_pair_R<2, 2, true>(ctx, pa, nw);
        case 240: return launch_pair_R<2, 4, false>(ctx, pa, nw);
        case 241: return launch_pair_R<2, 4, true>(ctx, pa, nw);
        case 280: return launch_pair_R<2, 8, false>(ctx, pa, nw);
        case 281: return launch_pair_R<2, 8, true>(ctx, pa, nw);
        case 420: return launch_pair_R<4, 2, false>(ctx, pa, nw);
        case 421: return launch_pair_R<4, 2, true>(ctx, pa, nw);
        case 440: return launch_pair_R<4, 4, false>(ctx, pa, nw);
        case 441: return launch_pair_R<4, 4, true>(ctx, pa, nw);
        case 820: return launch_pair_R<8, 2, false>(ctx, pa, nw);
        case 821: return launch_pair_R<8, 2, true>(ctx, pa, nw);
        default: return fail(ctx, NW_ERR_ARG, "unsupported block shape %d x %d", R, C);
    }
}

}  // namespace nw
