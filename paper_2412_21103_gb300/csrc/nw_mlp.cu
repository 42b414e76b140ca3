// Learned band (a9): 4-mer diagonal-histogram features and a small BF16 MLP
// that predicts the band half-width of a pair.  Not in the paper.
//
// Features of a pair (A: m bases, B: n bases, L = max(m,n), delta = n - m):
//   K = min(256, m-3) anchors i_k = floor(k*(m-4)/(K-1)) in A; anchor i's
//   expected diagonal is e(i) = round(delta*i/m); every j in B within
//   W = max(1, L/8) of i + e(i) whose 4-mer equals A's 4-mer at i adds one to
//   bin floor((j - i - e(i) + W) * 64 / (2W+1)).  f[b] = log1p(count_b) /
//   log1p(K) for the 64 bins, f[64] = delta / L.  (Pairs with m < 4 or n < 4
//   get an all-zero histogram.)
//
// Network: 65 -> 128 (ReLU) -> 128 (ReLU) -> 1, weights and activations in
// BF16, accumulation and biases in FP32; the output is log(w) of the band
// half-width.  Parameters (FP32 masters, flat): W1[128][65], b1[128],
// W2[128][128], b2[128], W3[128], b3.  Loss: 0.5 * mean((y - t)^2).  Training
// uses Adam (beta 0.9 / 0.999, eps 1e-8) on the FP32 masters; the BF16
// copies used by forward and backward are refreshed after every step.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <vector>

#include "nw_internal.cuh"

namespace nw {

constexpr int kF = 65, kH = 128;
constexpr int kNW1 = kH * kF, kNB1 = kH, kNW2 = kH * kH, kNB2 = kH, kNW3 = kH, kNB3 = 1;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kNW1, kOffW2 = kOffB1 + kNB1, kOffB2 = kOffW2 + kNW2,
              kOffW3 = kOffB2 + kNB2, kOffB3 = kOffW3 + kNW3, kNParams = kOffB3 + kNB3;
constexpr int kAnchors = 256, kBins = 64;

struct BandModel {
    float *master = nullptr;      // kNParams
    __nv_bfloat16 *wb = nullptr;  // BF16 copies of W1, W2, W3 (same offsets)
    float *adam_m = nullptr, *adam_v = nullptr;
    float *grad = nullptr;        // kNParams
    int64_t step = 0;
};

// ---------------------------------------------------------------- features
__global__ void __launch_bounds__(kAnchors) k_features(const uint8_t *pool, const uint64_t *a_off,
                                                       const uint32_t *a_len, const uint64_t *b_off,
                                                       const uint32_t *b_len, uint32_t npairs, float *feat) {
    extern __shared__ uint8_t bcode[];  // 4-mer code of B at every position
    __shared__ uint32_t hist[kBins];
    for (uint32_t p = blockIdx.x; p < npairs; p += gridDim.x) {
        const uint32_t m = a_len[p], n = b_len[p];
        const uint8_t *A = pool + a_off[p], *B = pool + b_off[p];
        if (threadIdx.x < kBins) hist[threadIdx.x] = 0;
        const bool ok = m >= 4 && n >= 4;
        const uint32_t nk = ok ? n - 3 : 0;
        for (uint32_t j = threadIdx.x; j < nk; j += blockDim.x)
            bcode[j] = (uint8_t)(base_at(B, j) | (base_at(B, j + 1) << 2) | (base_at(B, j + 2) << 4) |
                                 (base_at(B, j + 3) << 6));
        __syncthreads();
        const uint32_t L = max(m, n);
        const int32_t delta = (int32_t)n - (int32_t)m;
        const uint32_t K = ok ? min((uint32_t)kAnchors, m - 3) : 0;
        if (threadIdx.x < K) {
            const uint32_t i = K > 1 ? (uint32_t)(((uint64_t)threadIdx.x * (m - 4)) / (K - 1)) : 0u;
            const uint32_t ac = base_at(A, i) | (base_at(A, i + 1) << 2) | (base_at(A, i + 2) << 4) |
                                (base_at(A, i + 3) << 6);
            const int32_t e = (int32_t)llrint((double)delta * (double)i / (double)m);
            const int32_t W = max(1, (int32_t)(L / 8));
            const int32_t c0 = (int32_t)i + e;
            const int32_t jlo = max(0, c0 - W), jhi = min((int32_t)nk - 1, c0 + W);
            // four codes per 32-bit load; a byte of x is zero exactly where
            // the code equals ac (hi: its high bit set for every nonzero byte)
            const uint32_t acx4 = ac * 0x01010101u;
            const uint32_t *bw = reinterpret_cast<const uint32_t *>(bcode);
            for (int32_t w = jlo >> 2; w <= (jhi >> 2); ++w) {
                const uint32_t x = bw[w] ^ acx4;
                uint32_t zero = ~((((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u) & 0x80808080u;
                while (zero) {
                    const int32_t j = 4 * w + ((__ffs(zero) - 1) >> 3);
                    zero &= zero - 1;
                    if (j < jlo || j > jhi) continue;
                    const int32_t bin = (int32_t)(((int64_t)(j - c0 + W) * kBins) / (2 * W + 1));
                    atomicAdd(&hist[min(max(bin, 0), kBins - 1)], 1u);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < kBins) {
            const float norm = K ? log1pf((float)K) : 1.f;
            feat[(size_t)p * kF + threadIdx.x] = log1pf((float)hist[threadIdx.x]) / norm;
        }
        if (threadIdx.x == kBins) feat[(size_t)p * kF + kBins] = L ? (float)delta / (float)L : 0.f;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- network
__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Forward of one layer for a tile of samples: out[b][u] = act(sum_k W[u][k]
// in[b][k] + bias[u]) rounded to BF16 (act = ReLU) or left in FP32 (last).
// One thread per (sample, unit).
__global__ void k_layer_fwd(const float *in, int nin, const __nv_bfloat16 *W, const float *bias, int nout,
                            uint32_t nb, float *out, int relu, int round_in) {
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nb * (uint32_t)nout) return;
    const uint32_t b = idx / nout, u = idx % nout;
    const float *x = in + (size_t)b * nin;
    const __nv_bfloat16 *w = W + (size_t)u * nin;
    float acc = 0.f;
    for (int k = 0; k < nin; ++k) acc = fmaf(__bfloat162float(w[k]), round_in ? bf(x[k]) : x[k], acc);
    acc += bias[u];
    out[idx] = relu ? bf(fmaxf(acc, 0.f)) : acc;
}

// dy = (y - t) / B and the loss.
__global__ void k_dloss(const float *y, const float *t, uint32_t nb, float *dy, float *loss) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const float e = y[b] - t[b];
    dy[b] = e / (float)nb;
    atomicAdd(loss, 0.5f * e * e / (float)nb);
}

// dIn[b][k] = sum_u dOut[b][u] W[u][k], masked by ReLU'(act_in[b][k] > 0).
__global__ void k_layer_bwd_data(const float *dout, int nout, const __nv_bfloat16 *W, int nin, const float *act_in,
                                 uint32_t nb, float *din) {
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nb * (uint32_t)nin) return;
    const uint32_t b = idx / nin, k = idx % nin;
    float acc = 0.f;
    for (int u = 0; u < nout; ++u) acc = fmaf(dout[(size_t)b * nout + u], __bfloat162float(W[(size_t)u * nin + k]), acc);
    din[idx] = act_in[idx] > 0.f ? acc : 0.f;
}

// dW[u][k] = sum_b dOut[b][u] in[b][k] (in rounded to BF16 when asked),
// dBias[u] = sum_b dOut[b][u].  One thread per weight.
__global__ void k_layer_bwd_w(const float *dout, int nout, const float *in, int nin, uint32_t nb, float *dW,
                              float *dbias, int round_in) {
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nw = (uint32_t)nout * nin;
    if (idx < nw) {
        const uint32_t u = idx / nin, k = idx % nin;
        float acc = 0.f;
        for (uint32_t b = 0; b < nb; ++b) {
            const float x = in[(size_t)b * nin + k];
            acc = fmaf(dout[(size_t)b * nout + u], round_in ? bf(x) : x, acc);
        }
        dW[idx] = acc;
    } else if (idx < nw + (uint32_t)nout) {
        const uint32_t u = idx - nw;
        float acc = 0.f;
        for (uint32_t b = 0; b < nb; ++b) acc += dout[(size_t)b * nout + u];
        dbias[u] = acc;
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int n, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void k_refresh_bf16(const float *p, __nv_bfloat16 *wb, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(p[i]);
}

// He-style initialisation from a counter-based SplitMix64 stream: value k
// is mix64(seed + (k+1) * 0x9E3779B97F4A7C15), mapped to a uniform in
// [-1, 1) and scaled by sqrt(6 / fan_in); biases start at 0 except b3.
__device__ __forceinline__ uint64_t splitmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_init(float *p, uint64_t seed, float b3) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParams) return;
    float fan = 0.f;
    if (i < kOffB1) fan = kF;
    else if (i >= kOffW2 && i < kOffB2) fan = kH;
    else if (i >= kOffW3 && i < kOffB3) fan = kH;
    if (fan == 0.f) {
        p[i] = i == kOffB3 ? b3 : 0.f;
        return;
    }
    const uint64_t r = splitmix(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
    const float u = (float)((double)(r >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
    p[i] = u * sqrtf(6.f / fan);
}

// ------------------------------------------------------------------- host
static unsigned blocks_for(uint64_t n, unsigned t = 256) { return (unsigned)((n + t - 1) / t); }

static int model_of(nw_ctx *ctx, BandModel **out, bool create) {
    if (!ctx->band_model) {
        if (!create) return fail(ctx, NW_ERR_ARG, "no band model: call nw_band_model_init or nw_band_model_set");
        BandModel *bm = new BandModel();
        cudaError_t e = cudaMalloc(&bm->master, kNParams * 4);
        if (e == cudaSuccess) e = cudaMalloc(&bm->wb, kNParams * 2);
        if (e == cudaSuccess) e = cudaMalloc(&bm->adam_m, kNParams * 4);
        if (e == cudaSuccess) e = cudaMalloc(&bm->adam_v, kNParams * 4);
        if (e == cudaSuccess) e = cudaMalloc(&bm->grad, kNParams * 4);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, NW_ERR_OOM, "band model allocation failed");
        }
        cudaMemsetAsync(bm->adam_m, 0, kNParams * 4, ctx->stream);
        cudaMemsetAsync(bm->adam_v, 0, kNParams * 4, ctx->stream);
        ctx->band_model = bm;
    }
    *out = (BandModel *)ctx->band_model;
    return NW_OK;
}

void free_band_model(nw_ctx *ctx) {
    BandModel *bm = (BandModel *)ctx->band_model;
    if (!bm) return;
    cudaFree(bm->master);
    cudaFree(bm->wb);
    cudaFree(bm->adam_m);
    cudaFree(bm->adam_v);
    cudaFree(bm->grad);
    delete bm;
    ctx->band_model = nullptr;
}

static void refresh(nw_ctx *ctx, BandModel *bm) {
    k_refresh_bf16<<<blocks_for(kNParams), 256, 0, ctx->stream>>>(bm->master, bm->wb, kNParams);
}

// Activations for a batch: h1, h2 (BF16-rounded floats) and y.
struct Acts {
    float *h1, *h2, *y;
};

static int forward(nw_ctx *ctx, BandModel *bm, const float *x, uint32_t nb, Acts &a) {
    void *v = nullptr;
    int rc = scratch(ctx, "mlp_acts", (size_t)nb * (2 * kH + 1) * 4 + 64, &v);
    if (rc) return rc;
    a.h1 = (float *)v;
    a.h2 = a.h1 + (size_t)nb * kH;
    a.y = a.h2 + (size_t)nb * kH;
    LaunchTimer t(ctx, "mlp_forward", 3);
    k_layer_fwd<<<blocks_for((uint64_t)nb * kH), 256, 0, ctx->stream>>>(x, kF, bm->wb + kOffW1, bm->master + kOffB1,
                                                                         kH, nb, a.h1, 1, 1);
    k_layer_fwd<<<blocks_for((uint64_t)nb * kH), 256, 0, ctx->stream>>>(a.h1, kH, bm->wb + kOffW2, bm->master + kOffB2,
                                                                         kH, nb, a.h2, 1, 0);
    k_layer_fwd<<<blocks_for(nb), 256, 0, ctx->stream>>>(a.h2, kH, bm->wb + kOffW3, bm->master + kOffB3, 1, nb, a.y,
                                                          0, 0);
    return NW_OK;
}

static int gradients(nw_ctx *ctx, BandModel *bm, const float *x, const float *t, uint32_t nb, float *loss) {
    Acts a;
    int rc = forward(ctx, bm, x, nb, a);
    if (rc) return rc;
    void *v = nullptr;
    if ((rc = scratch(ctx, "mlp_grads", (size_t)nb * (2 * kH + 1) * 4 + 64, &v))) return rc;
    float *dy = (float *)v, *dh2 = dy + nb, *dh1 = dh2 + (size_t)nb * kH;
    cudaMemsetAsync(loss, 0, 4, ctx->stream);
    LaunchTimer lt(ctx, "mlp_backward", 6);
    k_dloss<<<blocks_for(nb), 256, 0, ctx->stream>>>(a.y, t, nb, dy, loss);
    // layer 3: dW3, db3; dh2 = W3^T dy masked by h2 > 0
    k_layer_bwd_w<<<blocks_for(kNW3 + 1), 256, 0, ctx->stream>>>(dy, 1, a.h2, kH, nb, bm->grad + kOffW3,
                                                                 bm->grad + kOffB3, 0);
    k_layer_bwd_data<<<blocks_for((uint64_t)nb * kH), 256, 0, ctx->stream>>>(dy, 1, bm->wb + kOffW3, kH, a.h2, nb, dh2);
    // layer 2
    k_layer_bwd_w<<<blocks_for(kNW2 + kH), 256, 0, ctx->stream>>>(dh2, kH, a.h1, kH, nb, bm->grad + kOffW2,
                                                                  bm->grad + kOffB2, 0);
    k_layer_bwd_data<<<blocks_for((uint64_t)nb * kH), 256, 0, ctx->stream>>>(dh2, kH, bm->wb + kOffW2, kH, a.h1, nb,
                                                                            dh1);
    // layer 1 (inputs rounded to BF16 as in the forward)
    k_layer_bwd_w<<<blocks_for(kNW1 + kH), 256, 0, ctx->stream>>>(dh1, kH, x, kF, nb, bm->grad + kOffW1,
                                                                  bm->grad + kOffB1, 1);
    return NW_OK;
}

}  // namespace nw

using namespace nw;

// The feature kernel keeps B in dynamic shared memory (one byte per base).
// Its limit above the default 48 KiB is a per-function attribute of the
// process, which concurrent callers (the server's workers) share: it is
// always set to the one value that covers every accepted B, never to a
// call's own need, so a launch never meets a smaller limit set by another
// thread.
constexpr uint32_t kFeatMaxB = 200000;
static int features_smem(nw_ctx *ctx, uint32_t maxn) {
    if (maxn <= 48 * 1024) return NW_OK;
    const cudaError_t e = cudaFuncSetAttribute(k_features, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFeatMaxB);
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "feature kernel shared memory");
}

// Features -> network -> half-widths (with a safety factor), on the host.
uint32_t band_start_width(float y, uint32_t m, uint32_t n, double margin, double probe_cap, bool skip);

// `overlap` runs on the host once the feature and network kernels are
// queued, before the copy of their output (a copy into pageable memory
// returns only when it is done); not at all when the call keeps the fixed
// start.
int learned_band_widths(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                        const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, std::vector<uint32_t> &w,
                        const std::function<int()> &overlap) {
    w.assign(npairs, 64u);
    BandModel *bm = nullptr;
    if (!ctx->band_model) return NW_OK;  // no model: fixed starting width 64
    // The first round's width is 0.75x the predicted one: a round that fails
    // its certificate is followed by one at the smallest width the failed
    // score proves sufficient, so under-predicting costs one narrow pass
    // while over-predicting widens every band.  Measured on GB300 (20,000
    // pairs of 2-20 kb, same context and memory budget): 0.25 -> 6,526,
    // 0.5 -> 6,100, 0.75 -> 5,691, 1 -> 5,285 effective GCUPS, against 6,962
    // from the fixed start 64; 0.75 is kept because it is the smallest
    // margin at which the network certifies more pairs in the first round
    // than the fixed start on held-out pairs while sweeping fewer banded
    // cells there.  NW_BAND_MARGIN and NW_BAND_PROBE_CAP for sweeps.
    double margin = 0.75;
    if (const char *e = getenv("NW_BAND_MARGIN")) margin = std::max(0.25, atof(e));
    int rc = model_of(ctx, &bm, false);
    if (rc) return rc;
    void *v = nullptr;
    if ((rc = scratch(ctx, "lb_meta", (size_t)npairs * 24 + 64, &v))) return rc;
    uint64_t *dao = (uint64_t *)v, *dbo = dao + npairs;
    uint32_t *dal = (uint32_t *)(dbo + npairs), *dbl = dal + npairs;
    cudaMemcpyAsync(dao, a_off, (size_t)npairs * 8, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dbo, b_off, (size_t)npairs * 8, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dal, a_len, (size_t)npairs * 4, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dbl, b_len, (size_t)npairs * 4, cudaMemcpyHostToDevice, ctx->stream);
    void *f = nullptr;
    if ((rc = scratch(ctx, "lb_feat", (size_t)npairs * kF * 4 + 64, &f))) return rc;
    uint32_t maxn = 4;
    for (uint32_t k = 0; k < npairs; ++k) maxn = std::max(maxn, b_len[k]);
    if (maxn > kFeatMaxB) return NW_OK;  // features need B <= 200,000 bases: keep the fixed start
    if ((rc = features_smem(ctx, maxn))) return rc;
    {
        LaunchTimer t(ctx, "features");
        k_features<<<std::min<uint32_t>(npairs, (uint32_t)ctx->sm_count * 8), kAnchors, maxn, ctx->stream>>>(
            pool, dao, dal, dbo, dbl, npairs, (float *)f);
    }
    if (const cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_fail(ctx, e, "features launch");
    Acts a;
    if ((rc = forward(ctx, bm, (const float *)f, npairs, a))) return rc;
    if (overlap && (rc = overlap())) return rc;
    std::vector<float> y(npairs);
    cudaMemcpyAsync(y.data(), a.y, (size_t)npairs * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if ((rc = nw_ctx_sync(ctx))) return rc;
    // Probe cap (NW_BAND_PROBE_CAP, 0 = none) and the straight-to-full rule
    // (NW_BAND_SKIP: a pair whose predicted band would cover most of the
    // grid starts at that width, which sends it to the full kernel).
    double probe_cap = 0.0;
    if (const char *e = getenv("NW_BAND_PROBE_CAP")) probe_cap = atof(e);
    const bool skip = getenv("NW_BAND_SKIP") != nullptr;
    for (uint32_t k = 0; k < npairs; ++k) w[k] = band_start_width(y[k], a_len[k], b_len[k], margin, probe_cap, skip);
    return NW_OK;
}

// First half-width of a pair from the network's output y = log w:
// ceil(margin * e^y), clamped to [8, max(m, n)].  (Sweep knobs: a probe cap
// on the width, and the straight-to-full rule for a predicted band that would
// cover most of the grid.)
uint32_t band_start_width(float y, uint32_t m, uint32_t n, double margin, double probe_cap, bool skip) {
    const double full_pred = std::exp((double)y);
    double pred = full_pred * margin;
    const double cap = (double)std::max(m, n);
    const double delta = std::fabs((double)n - (double)m);
    if (skip && (512.0 + 2.0 * full_pred + delta) * 20.0 >= (double)n * 17.0) pred = cap;
    else if (probe_cap > 0 && pred > probe_cap) pred = probe_cap;
    return (uint32_t)std::min(cap, std::max(8.0, std::ceil(pred)));
}

extern "C" {

int nw_band_features(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                     const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, float *feat) {
    if (!ctx) return NW_ERR_ARG;
    if (npairs == 0) return NW_OK;
    if (!pool2b || !a_off || !a_len || !b_off || !b_len || !feat) return fail(ctx, NW_ERR_ARG, "null argument");
    cudaSetDevice(ctx->device);
    void *v = nullptr;
    int rc = scratch(ctx, "feat_meta", (size_t)npairs * 24 + 64, &v);
    if (rc) return rc;
    uint64_t *dao = (uint64_t *)v, *dbo = dao + npairs;
    uint32_t *dal = (uint32_t *)(dbo + npairs), *dbl = dal + npairs;
    cudaMemcpyAsync(dao, a_off, (size_t)npairs * 8, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dbo, b_off, (size_t)npairs * 8, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dal, a_len, (size_t)npairs * 4, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dbl, b_len, (size_t)npairs * 4, cudaMemcpyHostToDevice, ctx->stream);
    uint32_t maxn = 4;
    for (uint32_t k = 0; k < npairs; ++k) maxn = std::max(maxn, b_len[k]);
    if (maxn > kFeatMaxB) return fail(ctx, NW_ERR_ARG, "features need B <= 200,000 bases");
    if (int rc2 = features_smem(ctx, maxn)) return rc2;
    {
        LaunchTimer t(ctx, "features");
        k_features<<<std::min<uint32_t>(npairs, (uint32_t)ctx->sm_count * 8), kAnchors, maxn, ctx->stream>>>(
            pool2b, dao, dal, dbo, dbl, npairs, feat);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "features launch");
    // the metadata copies read host arrays the caller may free on return
    e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "features sync");
}

int nw_band_model_init(nw_ctx *ctx, uint64_t seed) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    BandModel *bm = nullptr;
    int rc = model_of(ctx, &bm, true);
    if (rc) return rc;
    k_init<<<blocks_for(kNParams), 256, 0, ctx->stream>>>(bm->master, seed, std::log(64.f));
    cudaMemsetAsync(bm->adam_m, 0, kNParams * 4, ctx->stream);
    cudaMemsetAsync(bm->adam_v, 0, kNParams * 4, ctx->stream);
    bm->step = 0;
    refresh(ctx, bm);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "model init");
}

uint32_t nw_band_start_width(float y, uint64_t m, uint64_t n) {
    if (m >= (1ull << 31) || n >= (1ull << 31)) return 0;
    return band_start_width(y, (uint32_t)m, (uint32_t)n, 0.75, 0.0, false);
}

uint64_t nw_band_model_size(void) { return kNParams; }

int nw_band_model_set(nw_ctx *ctx, const float *params, uint64_t count) {
    if (!ctx || !params || count != (uint64_t)kNParams) return ctx ? fail(ctx, NW_ERR_ARG, "need %d params", kNParams) : NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    BandModel *bm = nullptr;
    int rc = model_of(ctx, &bm, true);
    if (rc) return rc;
    cudaMemcpyAsync(bm->master, params, kNParams * 4, cudaMemcpyHostToDevice, ctx->stream);
    refresh(ctx, bm);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "model set");
}

// File format of a saved model: the 8 bytes "NWBAND01", the parameter
// count as a little-endian uint64, then the FP32 master parameters in the
// layout nw_band_model_get returns (little-endian IEEE-754).
int nw_band_model_save(nw_ctx *ctx, const char *path) {
    if (!ctx || !path) return NW_ERR_ARG;
    std::vector<float> p(kNParams);
    int rc = nw_band_model_get(ctx, p.data(), p.size());
    if (rc) return rc;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ctx, NW_ERR_ARG, "cannot open '%s' for writing", path);
    const uint64_t count = kNParams;
    const bool ok = fwrite("NWBAND01", 1, 8, f) == 8 && fwrite(&count, 8, 1, f) == 1 &&
                    fwrite(p.data(), 4, p.size(), f) == p.size();
    const bool closed = fclose(f) == 0;
    return ok && closed ? NW_OK : fail(ctx, NW_ERR_ARG, "short write to '%s'", path);
}

int nw_band_model_load(nw_ctx *ctx, const char *path) {
    if (!ctx || !path) return NW_ERR_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ctx, NW_ERR_ARG, "cannot open '%s'", path);
    char magic[8] = {0};
    uint64_t count = 0;
    std::vector<float> p(kNParams);
    const bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "NWBAND01", 8) == 0 && fread(&count, 8, 1, f) == 1 &&
                    count == (uint64_t)kNParams && fread(p.data(), 4, p.size(), f) == p.size() && fgetc(f) == EOF;
    fclose(f);
    if (!ok) return fail(ctx, NW_ERR_ARG, "'%s' is not a saved band model of %d parameters", path, kNParams);
    return nw_band_model_set(ctx, p.data(), p.size());
}

int nw_band_model_clear(nw_ctx *ctx) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);  // no kernel still reads the parameters
    free_band_model(ctx);
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "model clear");
}

int nw_band_model_get(nw_ctx *ctx, float *params, uint64_t count) {
    if (!ctx || !params || count != (uint64_t)kNParams) return ctx ? fail(ctx, NW_ERR_ARG, "need %d params", kNParams) : NW_ERR_ARG;
    BandModel *bm = nullptr;
    int rc = model_of(ctx, &bm, false);
    if (rc) return rc;
    cudaMemcpyAsync(params, bm->master, kNParams * 4, cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "model get");
}

int nw_band_model_forward(nw_ctx *ctx, const float *feat, uint32_t n, float *out) {
    if (!ctx || (n && (!feat || !out))) return NW_ERR_ARG;
    if (!n) return NW_OK;
    cudaSetDevice(ctx->device);
    BandModel *bm = nullptr;
    int rc = model_of(ctx, &bm, false);
    if (rc) return rc;
    Acts a;
    if ((rc = forward(ctx, bm, feat, n, a))) return rc;
    cudaMemcpyAsync(out, a.y, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "model forward");
}

int nw_band_model_grad(nw_ctx *ctx, const float *feat, const float *target, uint32_t n, float *grad, float *loss) {
    if (!ctx || !feat || !target || !grad || !loss || !n) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    BandModel *bm = nullptr;
    int rc = model_of(ctx, &bm, false);
    if (rc) return rc;
    if ((rc = gradients(ctx, bm, feat, target, n, loss))) return rc;
    cudaMemcpyAsync(grad, bm->grad, kNParams * 4, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "model grad");
}

int nw_band_model_train_step(nw_ctx *ctx, const float *feat, const float *target, uint32_t n, float lr, float *loss) {
    if (!ctx || !feat || !target || !loss || !n) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    BandModel *bm = nullptr;
    int rc = model_of(ctx, &bm, false);
    if (rc) return rc;
    if ((rc = gradients(ctx, bm, feat, target, n, loss))) return rc;
    bm->step += 1;
    const float c1 = 1.f - std::pow(0.9f, (float)bm->step), c2 = 1.f - std::pow(0.999f, (float)bm->step);
    {
        LaunchTimer t(ctx, "adam");
        k_adam<<<blocks_for(kNParams), 256, 0, ctx->stream>>>(bm->master, bm->grad, bm->adam_m, bm->adam_v, kNParams,
                                                               lr, c1, c2);
    }
    refresh(ctx, bm);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "train step");
}

}  // extern "C"
