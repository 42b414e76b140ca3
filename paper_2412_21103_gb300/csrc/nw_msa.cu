// Center-star multiple alignment (the paper's Sec. 3.2) on one GPU.
//
// Stage 1, the scoring matrix: the n(n-1)/2 pairwise scores of Eq. 2 by the
// batched kernel (nw_score_all_pairs).  Stage 2, the center: the sequence
// most similar to the rest -- the largest sum of its scores against the
// other sequences (the diagonal len*match is left out), lowest index on
// ties -- found by a row-sum kernel and an arg-max kernel.  Stage 3: every
// sequence aligned (as the query, rows) with the center (the reference,
// columns) by the batched CIGAR path.  Stage 4, the merge with the aligned
// center as the reference ("once a gap, always a gap"): before center base
// p (p = 0..|C|, |C| = after the last base) the merged alignment keeps G[p]
// columns, the most 'I' ops any alignment puts there; center base p lands in
// column p + G[0] + ... + G[p]; a row's I-bases fill their slot from its
// left; a 'D' op leaves '-' in the center's column.  The merge reads the
// RLE CIGARs on the device: one thread per sequence finds its insertion
// runs (atomic max into G), one block scans G into column offsets, one
// thread per sequence writes its row.
#include <algorithm>
#include <vector>

#include "nw_internal.cuh"

namespace nw {

// Sum of row i over j != i (int64), one warp per row.
__global__ void k_row_sums(const int32_t *M, uint32_t nseq, int64_t *sums) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nseq; i += warps) {
        const int32_t *row = M + (size_t)i * nseq;
        int64_t s = 0;
        for (uint32_t j = lane; j < nseq; j += 32u)
            if (j != i) s += row[j];
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (lane == 0) sums[i] = s;
    }
}

// Index of the largest sum, the lowest index on ties (one block).
__global__ void k_argmax(const int64_t *sums, uint32_t nseq, uint32_t *center) {
    __shared__ int64_t bv[32];
    __shared__ uint32_t bi[32];
    int64_t v = INT64_MIN;
    uint32_t idx = 0xffffffffu;
    for (uint32_t i = threadIdx.x; i < nseq; i += blockDim.x)
        if (sums[i] > v) {  // i grows: strict keeps the first maximum of this thread
            v = sums[i];
            idx = i;
        }
    auto better = [](int64_t v1, uint32_t i1, int64_t v2, uint32_t i2) { return v1 > v2 || (v1 == v2 && i1 < i2); };
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const int64_t v2 = __shfl_xor_sync(kFull, v, o);
        const uint32_t i2 = __shfl_xor_sync(kFull, idx, o);
        if (better(v2, i2, v, idx)) {
            v = v2;
            idx = i2;
        }
    }
    const uint32_t w = threadIdx.x >> 5, nw_ = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31u) == 0) {
        bv[w] = v;
        bi[w] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (uint32_t k = 1; k < nw_; ++k)
            if (better(bv[k], bi[k], v, idx)) {
                v = bv[k];
                idx = bi[k];
            }
        *center = idx;
    }
}

// Calls f(op, count) for every run of a run-length encoded CIGAR; returns
// false on a character that is neither a digit nor an op.
template <typename F>
__device__ bool for_runs(const char *c, uint64_t len, F f) {
    uint64_t num = 0;
    for (uint64_t q = 0; q < len; ++q) {
        const char ch = c[q];
        if (ch >= '0' && ch <= '9') {
            num = num * 10u + (uint64_t)(ch - '0');
            continue;
        }
        if (ch != '=' && ch != 'X' && ch != 'M' && ch != 'I' && ch != 'D') return false;
        if (!f(ch, num)) return false;
        num = 0;
    }
    return true;
}

// G[p] = max over sequences of the 'I' ops placed before center base p.
// Checks that alignment k consumes exactly len[k] bases and the C center
// bases (NW_ERR_ARG into the error word, detail k, otherwise).
__global__ void k_slot_gaps(const char *cigar_pool, const uint64_t *cigar_off, const uint64_t *cigar_len,
                            const uint32_t *len, uint32_t nseq, uint32_t C, uint32_t *G, uint32_t *err) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nseq; k += gridDim.x * blockDim.x) {
        uint64_t p = 0, i = 0, ins = 0;
        const bool ok = for_runs(cigar_pool + cigar_off[k], cigar_len[k], [&](char op, uint64_t cnt) {
            if (op == 'I') {
                ins += cnt;
                i += cnt;
            } else {
                if (ins && p <= C) atomicMax(G + p, ins < 0xffffffffull ? (uint32_t)ins : 0xffffffffu);
                ins = 0;
                p += cnt;
                if (op != 'D') i += cnt;
            }
            return p <= C && i <= len[k];
        });
        if (ins && p <= C) atomicMax(G + p, ins < 0xffffffffull ? (uint32_t)ins : 0xffffffffu);
        if (!ok || p != C || i != len[k]) raise_error(err, NW_ERR_ARG, k);
    }
}

// start[p] = p + G[0] + ... + G[p-1] (first column of slot p) for p =
// 0..count-1, and the column count (count-1) + sum(G) (one block).
__global__ void k_slot_scan(const uint32_t *G, uint32_t count, uint64_t *start, uint64_t *ncols) {
    __shared__ uint64_t wsum[32];
    __shared__ uint64_t carry_s;
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (uint32_t base = 0; base < count; base += blockDim.x) {
        const uint32_t p = base + threadIdx.x;
        const uint64_t v = p < count ? (uint64_t)G[p] : 0u;
        uint64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            uint64_t t = lane < nwarps ? wsum[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(kFull, t, o);
                if ((int)lane >= o) t += y;
            }
            if (lane < nwarps) wsum[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        const uint64_t before = carry_s + (w ? wsum[w - 1] : 0u) + (incl - v);
        if (p < count) start[p] = before + p;
        __syncthreads();
        if (threadIdx.x == 0) carry_s += wsum[nwarps - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *ncols = carry_s + (count - 1);
}

// Row k of the merged alignment: the caller set every byte to '-'.
__global__ void k_merge_rows(const uint8_t *pool, const uint64_t *off, const uint32_t *len, const char *cigar_pool,
                             const uint64_t *cigar_off, const uint64_t *cigar_len, uint32_t nseq, const uint32_t *G,
                             const uint64_t *start, const uint64_t *ncols, char *msa, uint64_t ld,
                             uint32_t *err) {
    if (*(volatile const uint32_t *)err) return;  // a CIGAR failed its check
    const uint64_t cols = *ncols;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nseq; k += gridDim.x * blockDim.x) {
        char *row = msa + (uint64_t)k * ld;
        const uint8_t *s = pool + off[k];
        uint64_t p = 0, i = 0, used = 0;
        for_runs(cigar_pool + cigar_off[k], cigar_len[k], [&](char op, uint64_t cnt) {
            for (uint64_t r = 0; r < cnt; ++r) {
                if (op == 'I') {
                    const uint64_t col = start[p] + used++;
                    if (in_range(col, cols, err, kSiteMsaRow)) row[col] = "ACGT"[base_at(s, i)];
                    ++i;
                } else if (op == 'D') {
                    ++p;
                    used = 0;
                } else {
                    const uint64_t col = start[p] + G[p];
                    if (in_range(col, cols, err, kSiteMsaRow)) row[col] = "ACGT"[base_at(s, i)];
                    ++i;
                    ++p;
                    used = 0;
                }
            }
            return true;
        });
        if (ld > cols) row[cols] = '\0';
    }
}

// The merge on device buffers (metadata arrays on the host).
static int merge_device(nw_ctx *ctx, const uint8_t *pool, const uint64_t *off, const uint32_t *len, uint32_t nseq,
                        uint32_t center, const char *cigar_pool, const uint64_t *cigar_off, const uint64_t *cigar_len,
                        char *msa, uint64_t ld, uint64_t *msa_cols) {
    int rc;
    const uint32_t C = len[center];
    void *doff = nullptr, *dlen = nullptr, *dcoff = nullptr, *dG = nullptr, *dstart = nullptr, *dn = nullptr;
    if ((rc = to_device(ctx, off, (size_t)nseq * 8, "msa_off", &doff))) return rc;
    if ((rc = to_device(ctx, len, (size_t)nseq * 4, "msa_len", &dlen))) return rc;
    if ((rc = to_device(ctx, cigar_off, (size_t)nseq * 8, "msa_coff", &dcoff))) return rc;
    if ((rc = scratch(ctx, "msa_G", ((size_t)C + 1) * 4, &dG))) return rc;
    if ((rc = scratch(ctx, "msa_start", ((size_t)C + 1) * 8, &dstart))) return rc;
    if ((rc = scratch(ctx, "msa_ncols", 16, &dn))) return rc;
    cudaError_t e = cudaMemsetAsync(dG, 0, ((size_t)C + 1) * 4, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "msa memset");
    const uint32_t blocks = std::max<uint32_t>(1, (nseq + 127) / 128);
    {
        LaunchTimer t(ctx, "msa_gaps");
        k_slot_gaps<<<blocks, 128, 0, ctx->stream>>>(cigar_pool, (const uint64_t *)dcoff, cigar_len,
                                                     (const uint32_t *)dlen, nseq, C, (uint32_t *)dG, ctx->d_err);
    }
    {
        LaunchTimer t(ctx, "msa_scan");
        k_slot_scan<<<1, 1024, 0, ctx->stream>>>((const uint32_t *)dG, C + 1, (uint64_t *)dstart, (uint64_t *)dn);
    }
    uint64_t cols = 0;
    e = cudaMemcpyAsync(&cols, dn, 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "msa column count D2H");
    if ((rc = nw_ctx_sync(ctx))) return rc;
    *msa_cols = cols;
    if (!msa) return NW_OK;
    if (ld < cols) return fail(ctx, NW_ERR_CIGAR_TRUNC, "merged alignment has %llu columns, row stride is %llu",
                               (unsigned long long)cols, (unsigned long long)ld);
    if (nseq && (e = cudaMemsetAsync(msa, '-', (size_t)nseq * ld, ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "msa fill");
    {
        LaunchTimer t(ctx, "msa_rows");
        k_merge_rows<<<blocks, 128, 0, ctx->stream>>>(pool, (const uint64_t *)doff, (const uint32_t *)dlen,
                                                      cigar_pool, (const uint64_t *)dcoff, cigar_len, nseq,
                                                      (const uint32_t *)dG, (const uint64_t *)dstart,
                                                      (const uint64_t *)dn, msa, ld, ctx->d_err);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "msa launch");
}

static uint64_t pool_extent(const uint64_t *off, const uint32_t *len, uint32_t nseq) {
    uint64_t b = 16;
    for (uint32_t k = 0; k < nseq; ++k) b = std::max<uint64_t>(b, off[k] + (len[k] + 3) / 4);
    return b;
}

}  // namespace nw

using namespace nw;

extern "C" int nw_msa_merge(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *off, const uint32_t *len,
                            uint32_t nseq, uint32_t center, uint32_t flags, const char *cigar_pool,
                            const uint64_t *cigar_off, const uint64_t *cigar_len, char *msa, uint64_t msa_ld,
                            uint64_t *msa_cols) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (nseq == 0) return fail(ctx, NW_ERR_ARG, "no sequences");
    if (!pool2b || !off || !len || !cigar_pool || !cigar_off || !cigar_len || !msa_cols || center >= nseq)
        return fail(ctx, NW_ERR_ARG, "null argument or center out of range");
    if (!(flags & NW_HOST_IO))
        return merge_device(ctx, pool2b, off, len, nseq, center, cigar_pool, cigar_off, cigar_len, msa, msa_ld,
                            msa_cols);
    int rc;
    void *dp = nullptr, *dc = nullptr, *dl = nullptr, *dm = nullptr;
    if ((rc = to_device(ctx, pool2b, pool_extent(off, len, nseq), "hio_pool", &dp))) return rc;
    uint64_t extent = 16;
    for (uint32_t k = 0; k < nseq; ++k) extent = std::max<uint64_t>(extent, cigar_off[k] + cigar_len[k]);
    if ((rc = to_device(ctx, cigar_pool, extent, "hio_cigar", &dc))) return rc;
    if ((rc = to_device(ctx, cigar_len, (size_t)nseq * 8, "hio_cigar_len", &dl))) return rc;
    if (msa && (rc = scratch(ctx, "hio_msa", (size_t)nseq * msa_ld + 16, &dm))) return rc;
    if ((rc = merge_device(ctx, (const uint8_t *)dp, off, len, nseq, center, (const char *)dc, cigar_off,
                           (const uint64_t *)dl, msa ? (char *)dm : nullptr, msa_ld, msa_cols)))
        return rc;
    if (!msa) return NW_OK;
    cudaError_t e = cudaMemcpyAsync(msa, dm, (size_t)nseq * msa_ld, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "msa D2H");
    return nw_ctx_sync(ctx);
}

extern "C" int nw_center_star(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *off, const uint32_t *len,
                              uint32_t nseq, nw_scoring sc, uint32_t flags, uint32_t *center, int64_t *row_sums,
                              int32_t *scores, char *cigar_pool, const uint64_t *cigar_off, uint64_t *cigar_len,
                              char *msa, uint64_t msa_ld, uint64_t *msa_cols) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    int rc = check_scoring(ctx, sc);
    if (rc) return rc;
    if (nseq == 0 || nseq > 65535) return fail(ctx, NW_ERR_ARG, "1 to 65535 sequences");
    if (!pool2b || !off || !len || !center || !scores || !cigar_pool || !cigar_off || !cigar_len || !msa_cols)
        return fail(ctx, NW_ERR_ARG, "null argument");
    for (uint32_t k = 0; k < nseq; ++k)
        if (cigar_off[k + 1] < cigar_off[k]) return fail(ctx, NW_ERR_ARG, "CIGAR offsets must not decrease");
    const bool host = flags & NW_HOST_IO;
    const uint8_t *pool = pool2b;
    int32_t *d_scores = scores;
    char *d_cig = cigar_pool;
    uint64_t *d_clen = cigar_len;
    int64_t *d_sums = row_sums;
    if (host) {
        void *p = nullptr;
        if ((rc = to_device(ctx, pool2b, pool_extent(off, len, nseq), "hio_pool", &p))) return rc;
        pool = (const uint8_t *)p;
        if ((rc = scratch(ctx, "hio_scores", (size_t)nseq * 4, &p))) return rc;
        d_scores = (int32_t *)p;
        if ((rc = scratch(ctx, "hio_cigar", cigar_off[nseq] + 16, &p))) return rc;
        d_cig = (char *)p;
        if ((rc = scratch(ctx, "hio_cigar_len", (size_t)nseq * 8, &p))) return rc;
        d_clen = (uint64_t *)p;
        d_sums = nullptr;
    }
    // stage 1: the scoring matrix (Eq. 2 pairs)
    void *dM = nullptr, *dS = nullptr, *dc = nullptr;
    cudaError_t e0 = cudaSuccess;
    if ((rc = scratch(ctx, "cs_matrix", (size_t)nseq * nseq * 4, &dM))) return rc;
    if (!d_sums) {
        if ((rc = scratch(ctx, "cs_sums", (size_t)nseq * 8, &dS))) return rc;
        d_sums = (int64_t *)dS;
    }
    if ((rc = scratch(ctx, "cs_center", 16, &dc))) return rc;
    if (nseq == 1) {  // no pair to score: the one sequence is the center
        if ((e0 = cudaMemsetAsync(dM, 0, 4, ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e0, "matrix");
    } else if ((rc = nw_score_all_pairs(ctx, pool, off, len, nseq, sc, flags & NW_GRAPH, (int32_t *)dM))) {
        return rc;
    }
    // stage 2: the center
    {
        LaunchTimer t(ctx, "center", 2);
        const uint32_t blocks = std::min<uint32_t>((nseq + 7) / 8, (uint32_t)ctx->sm_count * 8);
        k_row_sums<<<blocks, 256, 0, ctx->stream>>>((const int32_t *)dM, nseq, d_sums);
        k_argmax<<<1, 1024, 0, ctx->stream>>>(d_sums, nseq, (uint32_t *)dc);
    }
    uint32_t c = 0;
    cudaError_t e = cudaMemcpyAsync(&c, dc, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "center D2H");
    if ((rc = nw_ctx_sync(ctx))) return rc;
    *center = c;
    // stage 3: every sequence (query) against the center (reference)
    std::vector<uint64_t> b_off(nseq, off[c]);
    std::vector<uint32_t> b_len(nseq, len[c]);
    for (uint32_t k = 0; k < nseq; ++k)
        if (cigar_off[k + 1] - cigar_off[k] < nw_cigar_bound(len[k], len[c]))
            return fail(ctx, NW_ERR_ARG, "CIGAR capacity of sequence %u below nw_cigar_bound", k);
    if ((rc = nw_align_batch(ctx, pool, off, len, b_off.data(), b_len.data(), nseq, sc,
                             NW_CIGAR | (flags & NW_CIGAR_M), d_scores, d_cig, cigar_off, d_clen)))
        return rc;
    // stage 4: the merge
    char *d_msa = msa;
    if (host && msa) {
        void *p = nullptr;
        if ((rc = scratch(ctx, "hio_msa", (size_t)nseq * msa_ld + 16, &p))) return rc;
        d_msa = (char *)p;
    }
    if ((rc = merge_device(ctx, pool, off, len, nseq, c, d_cig, cigar_off, d_clen, d_msa, msa_ld, msa_cols)))
        return rc;
    if (!host) return NW_OK;
    e = cudaMemcpyAsync(scores, d_scores, (size_t)nseq * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cigar_len, d_clen, (size_t)nseq * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cigar_pool, d_cig, cigar_off[nseq], cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && row_sums)
        e = cudaMemcpyAsync(row_sums, d_sums, (size_t)nseq * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && msa) e = cudaMemcpyAsync(msa, d_msa, (size_t)nseq * msa_ld, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "center-star D2H");
    return nw_ctx_sync(ctx);
}
