// Traceback (a5) and CIGAR assembly, shared by the single-pair and the
// batched paths.  A task describes one pair: its pointer words (layout
// [stripe][lane][column group], R rows x 16/R columns per word), its
// sequences and where its moves and CIGAR go.  One CTA per task.
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
                const uint32_t code = (word >> (2u * (((b1 - cb) % CPW) * R + (a1 % R)))) & 3u;
                const uint32_t mv = (code & 1u) ? 0u : ((code & 2u) ? 1u : 2u);
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
    uint64_t ci = 0, cj = 0;   // bases of A / B consumed before this chunk
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

int launch_trace(nw_ctx *ctx, int R, const TraceTask &one, const TraceTask *many, uint32_t ntasks, uint32_t mflag) {
    const int rc = launch_traceback(ctx, R, one, many, ntasks);
    return rc ? rc : launch_finish(ctx, one, many, ntasks, mflag);
}

}  // namespace nw
