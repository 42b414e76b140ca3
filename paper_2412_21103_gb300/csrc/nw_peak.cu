// Integer-pipe peak microbenchmark: the denominator of the roofline.
//
// Every thread runs kChains independent dependency chains of one instruction
// kind, so each SM sub-partition always has ready instructions; the grid is
// a multiple of the SM count.  The rate is reported in warp-lane operations
// per second (one 32-lane instruction = 32 operations).
#include "nw_bits.cuh"
#include "nw_internal.cuh"

namespace nw {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

// Kinds 0-4, 8 (LOP3), 9 (IMAD), 10 (funnel shift) time one instruction;
// 5-7 time one score-only cell in three formulations; 11 (below) one step
// of the bit-sliced update.  Every chain reads a neighbouring chain so the
// compiler cannot fold or strength-reduce the loop.
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak(uint64_t iters, int32_t seed, int32_t *sink) {
    int32_t x[kChains], y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = (int32_t)threadIdx.x * 3 + c + seed;
        y[c] = (int32_t)threadIdx.x - c;
    }
    const int32_t k1 = (seed & 3) + 1;
    const uint32_t sel = sext_selector((uint32_t)seed & 3u);
    const uint32_t prof = 0x01030103u + (uint32_t)seed;
    for (uint64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const int c1 = (c + 1) % kChains, c2 = (c + 2) % kChains;
            if constexpr (KIND == 0) {
                x[c] = __viaddmax_s32(x[c], k1, x[c1]);
            } else if constexpr (KIND == 1) {
                x[c] = __vimax3_s32(x[c], x[c1], x[c2]);
            } else if constexpr (KIND == 2) {
                x[c] = max(x[c], x[c1]);
            } else if constexpr (KIND == 3) {
                x[c] = (int32_t)((uint32_t)x[c] + (uint32_t)x[c1] + (uint32_t)k1);
            } else if constexpr (KIND == 4) {
                x[c] = (int32_t)prmt((uint32_t)x[c], (uint32_t)x[c1], sel);
            } else if constexpr (KIND == 5) {
                // prmt + DPX add-max + max
                const int32_t s = (int32_t)prmt(prof ^ (uint32_t)y[c], 0u, sel);
                const int32_t t = __viaddmax_s32(y[c], s, x[c]);
                y[c] = x[c];
                x[c] = max(t, x[c1]);
            } else if constexpr (KIND == 6) {
                // prmt + add + 3-input max
                const int32_t s = (int32_t)prmt(prof ^ (uint32_t)y[c], 0u, sel);
                const int32_t t = y[c] + s;
                y[c] = x[c];
                x[c] = __vimax3_s32(t, x[c], x[c1]);
            } else if constexpr (KIND == 7) {
                // prmt + add + two 2-input max
                const int32_t s = (int32_t)prmt(prof ^ (uint32_t)y[c], 0u, sel);
                const int32_t t = y[c] + s;
                y[c] = x[c];
                x[c] = max(max(t, x[c]), x[c1]);
            } else if constexpr (KIND == 8) {
                x[c] = (int32_t)lop3<kLutXor3>((uint32_t)x[c], (uint32_t)x[c1], (uint32_t)x[c2]);  // one LOP3
            } else if constexpr (KIND == 10) {
                x[c] = (int32_t)__funnelshift_l((uint32_t)x[c1], (uint32_t)x[c], (uint32_t)k1);  // one SHF
            } else {
                x[c] = (int32_t)((uint32_t)x[c] * (uint32_t)k1 + (uint32_t)x[c1]);  // IMAD
            }
        }
    }
    int32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= x[c] ^ y[c];
    if (acc == 0x7f3a5c11) *sink = acc;  // practically never true; keeps the work live
}

// Kind 11: one anti-diagonal step of the bit-sliced difference update (the
// step of nw_bits.cu: two window shifts, the match word, the two shifted
// upper inputs, T, dV, dH and the boundary shift register; 32 cells) on
// four independent lanes' words per thread.
constexpr int kBitsChains = 4;
__global__ void __launch_bounds__(kPeakThreads) k_peak_bits(uint64_t iters, uint32_t seed, int32_t *sink) {
    uint32_t H0[kBitsChains], H1[kBitsChains], V0[kBitsChains], V1[kBitsChains], Q0[kBitsChains], Q1[kBitsChains];
    const uint32_t A0 = seed * 0x9E3779B9u + threadIdx.x, A1 = A0 * 2654435761u;
    uint32_t Rc0 = ~A0, Rc1 = A1 ^ 0x5bd1e995u, Rn0 = A0 ^ 0x27d4eb2fu, Rn1 = ~A1;
    const uint32_t rmask = ~(seed & 1u);
#pragma unroll
    for (int c = 0; c < kBitsChains; ++c) {
        H0[c] = A0 >> c;
        H1[c] = 0;
        V0[c] = A1 >> c;
        V1[c] = 0;
        Q0[c] = Rc0 + c;
        Q1[c] = Rn1 - c;
    }
    for (uint64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kBitsChains; ++c) {
            const uint32_t bw0 = __funnelshift_l(Rn0, Rc0, c + 1), bw1 = __funnelshift_l(Rn1, Rc1, c + 1);
            const uint32_t x = lop3<kLutXorOrNotC>(A1, bw1, rmask);
            const uint32_t eq = lop3<kLutEq>(A0, bw0, x);
            const uint32_t a0 = __funnelshift_l(Q0[c], H0[c], 1), a1 = __funnelshift_l(Q1[c], H1[c], 1);
            const uint32_t b0 = V0[c], b1 = V1[c];
            const uint32_t p = lop3<kLutAndOrNot>(a0, a1, b1);
            const uint32_t q = lop3<kLutAndOrNot>(b0, b1, a1);
            const uint32_t v = lop3<kLutCOrNor>(a1, b1, eq);
            const uint32_t T0 = p | lop3<kLutOrAnd>(q, v, rmask);
            const uint32_t T1 = lop3<kLutOr3>(a1, b1, eq);
            const uint32_t ca = lop3<kLutAndNot>(a0, T0, 0u), cb = lop3<kLutAndNot>(b0, T0, 0u);
            V0[c] = T0 ^ a0;
            V1[c] = lop3<kLutXor3>(T1, a1, ca);
            H0[c] = T0 ^ b0;
            H1[c] = lop3<kLutXor3>(T1, b1, cb);
            Q0[c] = __funnelshift_l(H0[c], Q0[c], 1);
            Q1[c] = __funnelshift_l(H1[c], Q1[c], 1);
        }
        Rc0 = Rn0 ^ Rc0;  // keep the windows moving (two ops per step of 4 x 32 cells)
        Rn1 = Rc1 + Rn1;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kBitsChains; ++c) acc ^= H0[c] ^ H1[c] ^ V0[c] ^ V1[c] ^ Q0[c] ^ Q1[c];
    if (acc == 0x7f3a5c11u) *sink = (int32_t)acc;  // practically never true; keeps the work live
}

template <int KIND>
static float run_peak(nw_ctx *ctx, uint64_t iters, int32_t *sink) {
    const int blocks = ctx->sm_count * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](uint64_t n) {
        if constexpr (KIND == 11) k_peak_bits<<<blocks, kPeakThreads, 0, ctx->stream>>>(n, 1u, sink);
        else k_peak<KIND><<<blocks, kPeakThreads, 0, ctx->stream>>>(n, 1, sink);
    };
    launch(iters / 16 + 1);  // warm-up
    cudaEventRecord(e0, ctx->stream);
    {
        LaunchTimer t(ctx, "peak");
        launch(iters);
    }
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace nw

using namespace nw;

extern "C" int nw_peak_int(nw_ctx *ctx, int kind, uint64_t iters, double *gops) {
    if (!ctx || !gops || kind < 0 || kind > 11 || iters == 0) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    void *sink = nullptr;
    int rc = scratch(ctx, "peak_sink", 16, &sink);
    if (rc) return rc;
    float ms = 0.f;
    switch (kind) {
        case 0: ms = run_peak<0>(ctx, iters, (int32_t *)sink); break;
        case 1: ms = run_peak<1>(ctx, iters, (int32_t *)sink); break;
        case 2: ms = run_peak<2>(ctx, iters, (int32_t *)sink); break;
        case 3: ms = run_peak<3>(ctx, iters, (int32_t *)sink); break;
        case 4: ms = run_peak<4>(ctx, iters, (int32_t *)sink); break;
        case 5: ms = run_peak<5>(ctx, iters, (int32_t *)sink); break;
        case 6: ms = run_peak<6>(ctx, iters, (int32_t *)sink); break;
        case 7: ms = run_peak<7>(ctx, iters, (int32_t *)sink); break;
        case 8: ms = run_peak<8>(ctx, iters, (int32_t *)sink); break;
        case 9: ms = run_peak<9>(ctx, iters, (int32_t *)sink); break;
        case 10: ms = run_peak<10>(ctx, iters, (int32_t *)sink); break;
        default: ms = run_peak<11>(ctx, iters, (int32_t *)sink); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "peak kernel");
    // kinds 5-7 count cells, kind 11 cells (32 per word step), the others
    // instructions (per lane)
    const double per = kind == 11 ? (double)kBitsChains * 32 : (double)kChains;
    const double ops = (double)ctx->sm_count * 8 * kPeakThreads * per * (double)iters;
    *gops = ms > 0 ? ops / (ms * 1e-3) / 1e9 : 0.0;
    return NW_OK;
}
