// Integer-pipe peak microbenchmark: the denominator of the roofline.
//
// Every thread runs kChains independent dependency chains of one instruction
// kind, so each SM sub-partition always has ready instructions; the grid is
// a multiple of the SM count.  The rate is reported in warp-lane operations
// per second (one 32-lane instruction = 32 operations).
#include "nw_internal.cuh"

namespace nw {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

// Kinds 0-4, 8, 9 time one instruction; 5-7 time one score-only cell in
// three formulations.  Every chain reads a neighbouring chain so the
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
                x[c] = (x[c] ^ x[c1]) & (x[c2] | k1);  // one LOP3
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

template <int KIND>
static float run_peak(nw_ctx *ctx, uint64_t iters, int32_t *sink) {
    const int blocks = ctx->sm_count * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_peak<KIND><<<blocks, kPeakThreads, 0, ctx->stream>>>(iters / 16 + 1, 1, sink);  // warm-up
    cudaEventRecord(e0, ctx->stream);
    {
        LaunchTimer t(ctx, "peak");
        k_peak<KIND><<<blocks, kPeakThreads, 0, ctx->stream>>>(iters, 1, sink);
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
    if (!ctx || !gops || kind < 0 || kind > 9 || iters == 0) return NW_ERR_ARG;
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
        default: ms = run_peak<9>(ctx, iters, (int32_t *)sink); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "peak kernel");
    // kinds 5-7 count cells, the others instructions (per lane)
    const double ops = (double)ctx->sm_count * 8 * kPeakThreads * kChains * (double)iters;
    *gops = ms > 0 ? ops / (ms * 1e-3) / 1e9 : 0.0;
    return NW_OK;
}
