// Batched pairs (a7): many independent alignments in one persistent launch
// (the kernel is in nw_batch_kernel.cuh), straggler routing, the certified
// banded rounds (a8), CUDA graphs, and the C entry points.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <numeric>
#include <vector>

#include "nw_batch_kernel.cuh"
#include "nw_bits.cuh"
#include "nw_internal.cuh"
#include "nw_order.h"

namespace nw {

// ------------------------------------------------------------------- host
// Score slots the tasks of a launch may write (the checked build compares
// every score store against it).
static uint32_t score_slots(const BatchTask *host, uint32_t n) {
    uint32_t cap = 0;
    for (uint32_t k = 0; k < n; ++k) {
        cap = std::max(cap, host[k].out0 + 1);
        if (host[k].out1 != ~0u) cap = std::max(cap, host[k].out1 + 1);
    }
    return cap;
}

template <int R, bool PTR, int BAND>
static int launch_batch_R(nw_ctx *ctx, BatchArgs &ba, uint32_t max_n, const std::string &prefix) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<R, PTR, BAND>, kBatchWarps * 32, 0);
    if (occ < 1) occ = 1;
    uint32_t blocks = (uint32_t)occ * (uint32_t)ctx->sm_count;
    const uint32_t need = (ba.ntasks + kBatchWarps - 1) / kBatchWarps;
    if (blocks > need) blocks = need ? need : 1;
    const uint32_t warps = blocks * kBatchWarps;
    ba.ring_stride = ((max_n + 31) / 32) * 32 + 32;
    void *v = nullptr;
    int rc = scratch(ctx, (prefix + "_ring").c_str(), (size_t)warps * ba.ring_stride * 4, &v);
    if (rc) return rc;
    ba.ring = (uint32_t *)v;
    if ((rc = scratch(ctx, (prefix + "_counter").c_str(), 16, &v))) return rc;
    ba.counter = (uint32_t *)v;
    cudaMemsetAsync(ba.counter, 0, 4, ctx->stream);
    LaunchTimer t(ctx, BAND ? (PTR ? "band_fill_ptr" : "band_score") : (PTR ? "batch_fill_ptr" : "batch_score"));
    k_batch<R, PTR, BAND><<<blocks, kBatchWarps * 32, 0, ctx->stream>>>(ba);
    return NW_OK;
}

// band: 0 full grid, 1 strict band, 2 band region (see k_batch)
static int launch_batch(nw_ctx *ctx, int R, bool ptr, BatchArgs &ba, uint32_t max_n, int band = 0,
                        const std::string &prefix = "batch") {
#define NW_BATCH_CASES(PTRV, BANDV)                                                 \
    switch (R) {                                                                   \
        case 4: return launch_batch_R<4, PTRV, BANDV>(ctx, ba, max_n, prefix);     \
        case 8: return launch_batch_R<8, PTRV, BANDV>(ctx, ba, max_n, prefix);     \
        default: return launch_batch_R<16, PTRV, BANDV>(ctx, ba, max_n, prefix);   \
    }
    if (band == 2) {
        if (ptr) NW_BATCH_CASES(true, 2)
        NW_BATCH_CASES(false, 2)
    }
    if (band == 1) NW_BATCH_CASES(false, 1)  // strict band: score-only inspection
    if (ptr) NW_BATCH_CASES(true, 0)
    NW_BATCH_CASES(false, 0)
#undef NW_BATCH_CASES
}

// Rows per lane for a set of pairs: the one that wastes the fewest padded
// rows per useful row, counting a per-column overhead of ~10 instructions
// against 3 per cell.
static int pick_rows(const std::vector<BatchTask> &tasks) {
    double best = 1e300;
    int bestR = 8;
    for (int R : {4, 8, 16}) {
        double cost = 0;
        const uint32_t SH = 32u * R;
        for (const auto &t : tasks) {
            const double rows = (double)((t.m + SH - 1) / SH) * SH;
            const double P = std::max<uint32_t>(t.n, kMinPeriod);
            cost += rows * P * (3.0 + 10.0 / R);
        }
        if (cost < best) {
            best = cost;
            bestR = R;
        }
    }
    return bestR;
}

// Autotuner for the rows per lane of a score-only batch: the first call of a
// workload signature (mean lengths and pair count, bucketed by powers of
// two) runs the launch with each candidate, times it with CUDA events and
// keeps the fastest; later calls of the signature take the kept choice.
// Every candidate computes the same scores, so the timed runs are real work.
// Rows per lane 32 names the bit-sliced score-only kernel (one 32-row word
// per lane, nw_bits.cu); it is a candidate only where `bits` allows it (a
// score-only launch whose scoring fits two bit planes).
template <typename F>
static int tune_rows(nw_ctx *ctx, const std::vector<BatchTask> &tasks, int fallback, F launch, int *R,
                     bool bits = false) {
    *R = fallback;
    if (!ctx->autotune || tasks.empty()) return NW_OK;
    double sm = 0, sn = 0;
    for (const auto &t : tasks) {
        sm += t.m;
        sn += t.n;
    }
    const std::string key = "batch_rows:m" + size_bucket((uint64_t)(sm / tasks.size())) + ":n" +
                            size_bucket((uint64_t)(sn / tasks.size())) + ":p" + size_bucket(tasks.size());
    uint32_t c = 0;
    if (tuned(ctx, key, &c)) {
        if (c != 4 && c != 8 && c != 16 && c != 32)
            return fail(ctx, NW_ERR_ARG, "tuning %s: rows per lane %u", key.c_str(), c);
        *R = c == 32 && !bits ? 16 : (int)c;  // a pointer fill has no 32-row kernel
        return NW_OK;
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    int rc = NW_OK;
    for (int r : {4, 8, 16, 32}) {
        if (r == 32 && !bits) continue;
        cudaEventRecord(a, ctx->stream);
        if ((rc = launch(r))) break;
        cudaEventRecord(b, ctx->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
            best = ms;
            *R = r;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!rc) set_tuned(ctx, key, (uint32_t)*R);
    return rc;
}

// Graph-cache key of a batch call: the entry point, every device pointer it
// bakes in, the sizes and host metadata it was planned from.
static std::string batch_key(const char *what, const void *pool, const void *out, uint32_t count, const nw_scoring &sc,
                             uint32_t flags, uint64_t meta_hash) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%p|%p|%u|%d,%d,%d|%x|%016llx", what, pool, out, count, sc.match, sc.mismatch, sc.gap,
             flags, (unsigned long long)meta_hash);
    return buf;
}

template <typename T>
static int upload(nw_ctx *ctx, const char *slot, const std::vector<T> &v, T **dev) {
    void *d = nullptr;
    int rc = scratch(ctx, slot, v.size() * sizeof(T) + 16, &d);
    if (rc) return rc;
    if (!v.empty()) {
        cudaError_t e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "task upload");
        // the host vector may be freed right after: wait for the copy
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "task upload sync");
    }
    *dev = (T *)d;
    return NW_OK;
}

static void sort_lpt(std::vector<BatchTask> &tasks) {
    std::stable_sort(tasks.begin(), tasks.end(), [](const BatchTask &x, const BatchTask &y) {
        return (uint64_t)x.m * std::max(x.n, kMinPeriod) > (uint64_t)y.m * std::max(y.n, kMinPeriod);
    });
}

static int check_common(nw_ctx *ctx, const nw_scoring &sc) {
    if (!ctx) return NW_ERR_ARG;
    cudaSetDevice(ctx->device);
    return check_scoring(ctx, sc);
}

static int check_len(nw_ctx *ctx, const nw_scoring &sc, uint64_t m, uint64_t n) {
    if (m >= (1ull << 30) || n >= (1ull << 30)) return fail(ctx, NW_ERR_ARG, "sequence longer than 2^30");
    const uint64_t mn = m < n ? m : n;
    // W <= max(match - 2*gap, 0) * min(i, j): nothing to bound when the
    // diagonal never beats two gaps
    const uint64_t sp = sc.match > 2 * sc.gap ? (uint64_t)(sc.match - 2 * sc.gap) : 0;
    if (sp * mn >= (1ull << 29))
        return fail(ctx, NW_ERR_ARG, "(match - 2*gap) * min(m,n) must stay below 2^29");
    return NW_OK;
}

// The certified band's exit bound needs fewer gap moves to score higher:
// with G gap moves a path scores at most match*(m+n-G)/2 + gap*G, which
// falls with G only when match >= 2*gap.
static int check_band_scoring(nw_ctx *ctx, const nw_scoring &sc) {
    if (sc.match < 2 * sc.gap)
        return fail(ctx, NW_ERR_ARG, "the certified band needs match >= 2*gap (its exit bound assumes fewer gaps "
                                     "score higher)");
    return NW_OK;
}

// ------------------------------------------------------ straggler routing
// One warp per pair is efficient while the batch fills the GPU, but a pair
// much longer than the rest (or a long pair in a small batch) leaves the GPU
// idle while one warp grinds through it.  The longest pairs go to the
// multi-warp single-pair kernels instead: with pairs sorted by one-warp
// time, routing the first k costs the routed pairs' time + max(the rest's
// ideal batch time, the (k+1)-th one-warp time), and the k with the lowest
// estimate is taken.  Routed pairs on the bit-sliced single-pair kernel run
// together, each on its own warps (m/992 of them), so they cost the larger
// of their longest chain and their warp-seconds spread over the GPU's
// schedulers (1.5 warps at full speed on each); pairs on the scalar kernel
// run one after another.  Rates are GB300 measurements (cells/s): one warp
// of the batched kernels, the whole batched kernel, and the scalar
// single-pair kernel on a long pair; the bit-sliced one runs a chain of
// m + n + m/31 steps of about 40 ns, then its walk.
constexpr double kWarpRate = 2e9, kBatchRate = 3.5e12, kPairRate = 2e11, kPairFixed = 1e-3;
constexpr double kBitsStepSeconds = 40e-9, kBitsPairFixed = 0.3e-3;

struct PairCost {
    double secs;   // time of the pair on the single-pair path
    double warps;  // its warps on the bit-sliced kernel (0: the scalar kernel, one pair at a time)
};

static PairCost single_pair_cost(uint32_t m, uint32_t n, const nw_scoring &sc) {
    if (bits_scoring_ok(sc) && std::min(m, n) >= 64)
        return PairCost{((double)m + n + m / 31.0) * kBitsStepSeconds + kBitsPairFixed,
                        std::ceil(std::ceil(m / 31.0) / 32.0)};
    return PairCost{(double)m * n / kPairRate + kPairFixed, 0.0};
}

// warp_cells[k]: cells pair k costs on one warp (scaled for slower
// kernels), full_cells[k]: its full grid, costs[k] (or, when empty,
// full_cells[k] / kPairRate + kPairFixed on the scalar kernel): its cost on
// the single-pair path; sms: the GPU's SMs.  Returns the indices to route.
static std::vector<size_t> pick_stragglers(const std::vector<double> &warp_cells, const std::vector<double> &full_cells,
                                           const std::vector<PairCost> &costs, int sms,
                                           double batch_rate = kBatchRate) {
    std::vector<uint64_t> keys(warp_cells.size());
    for (size_t k = 0; k < keys.size(); ++k) keys[k] = order_key(warp_cells[k]);
    const std::vector<uint32_t> ord = radix_order_desc(std::move(keys));  // largest first, index order among equals
    const std::vector<size_t> order(ord.begin(), ord.end());
    double rest = 0;
    for (double c : warp_cells) rest += c;
    const double lanes = 6.0 * std::max(sms, 1);  // warps at full speed on the GPU's schedulers
    double serial = 0, conc_sum = 0, conc_max = 0, best = 1e300;
    size_t best_k = 0;
    for (size_t k = 0; k <= order.size(); ++k) {
        const double tail = k < order.size() ? warp_cells[order[k]] / kWarpRate : 0.0;
        const double est = serial + std::max(conc_max, conc_sum / lanes) + std::max(rest / batch_rate, tail);
        if (est < best) {
            best = est;
            best_k = k;
        }
        if (k == order.size()) break;
        const PairCost c = costs.empty() ? PairCost{full_cells[order[k]] / kPairRate + kPairFixed, 0.0}
                                         : costs[order[k]];
        if (c.warps > 0) {
            conc_sum += c.secs * c.warps;
            conc_max = std::max(conc_max, c.secs);
        } else {
            if (full_cells[order[k]] < 1e7) break;  // small pairs are not worth the scalar kernel's launches
            serial += c.secs;
        }
        rest -= warp_cells[order[k]];
    }
    return std::vector<size_t>(order.begin(), order.begin() + best_k);
}

// NW_BAND_KEEP=1 keeps every pair in the banded rounds (none leaves them for
// scheduling), so that what the rounds certify measures the band widths
// alone; small batches otherwise send wide-band pairs to the full-grid
// single-pair kernel, which runs them together.
static bool band_keep_all() {
    const char *e = getenv("NW_BAND_KEEP");
    return e && *e && *e != '0';
}

// Run one pair on the single-pair kernels, writing into the batch outputs.
static int run_straggler(nw_ctx *ctx, const uint8_t *pool, uint64_t a_off, uint32_t m, uint64_t b_off, uint32_t n,
                         const nw_scoring &sc, uint32_t flags, int32_t *score, char *cigar, uint64_t cigar_cap,
                         uint64_t *cigar_len) {
    LaunchTimer t(ctx, "straggler", 0);  // spans the single-pair kernels, which count themselves
    return align_single(ctx, pool + a_off, m, pool + b_off, n, sc, flags & (NW_CIGAR | NW_CIGAR_M | NW_RECOMPUTE), score,
                        (flags & NW_CIGAR) ? cigar : nullptr, cigar_cap, (flags & NW_CIGAR) ? cigar_len : nullptr);
}

// Runs tasks on the single-pair path, writing into the batch outputs: the
// pairs the bit-sliced single-pair kernel takes run together, each on its
// own warps, in waves; the others one after another.
static int run_stragglers(nw_ctx *ctx, const uint8_t *pool, const std::vector<BatchTask> &ts, const nw_scoring &sc,
                          uint32_t flags, int32_t *scores, char *cigar_pool, const uint64_t *cigar_off,
                          uint64_t *cigar_len) {
    const bool want = flags & NW_CIGAR;
    std::vector<PairJob> jobs;
    for (const BatchTask &t : ts) {
        const uint32_t id = t.out0;
        if (!(flags & NW_RECOMPUTE) && bits_pair_takes(ctx, t.m, t.n, sc, want)) {
            jobs.push_back(PairJob{t.a_off, t.b_off, t.m, t.n, scores + id, want ? cigar_pool + cigar_off[id] : nullptr,
                                   want ? cigar_len + id : nullptr});
            continue;
        }
        const int rc = run_straggler(ctx, pool, t.a_off, t.m, t.b_off, t.n, sc, flags, scores + id,
                                     want ? cigar_pool + cigar_off[id] : nullptr,
                                     want ? cigar_off[id + 1] - cigar_off[id] : 0, want ? cigar_len + id : nullptr);
        if (rc) return rc;
    }
    LaunchTimer t(ctx, "straggler", 0);  // spans the single-pair kernels, which count themselves
    return bits_pairs(ctx, pool, jobs, sc, want, (flags & NW_CIGAR_M) ? 1u : 0u);
}

// ------------------------------------------------------- certified band
// Closed-form bound on the score of any path that leaves the band of
// half-width w: such a path reaches diagonal hi+1 (then needs at least
// (hi+1) + (hi+1-delta) horizontal/vertical moves) or lo-1 (at least
// (1-lo) + (delta-lo+1)); with G gap moves it has (m+n-G)/2 diagonal moves
// worth at most `match` each, and match >= 0 >= gap makes fewer gaps better.
// Returns false when no path can leave the band (no bound needed).
bool band_exit_bound(int64_t m, int64_t n, int64_t w, int32_t match, int32_t gap, int64_t *bound) {
    const int64_t delta = n - m;
    const int64_t lo = std::min<int64_t>(0, delta) - w, hi = std::max<int64_t>(0, delta) + w;
    bool any = false;
    int64_t best = 0;
    const int64_t g_up = (hi + 1) + (hi + 1 - delta);   // visits diagonal hi+1
    const int64_t g_dn = (1 - lo) + (delta - lo + 1);   // visits diagonal lo-1
    const bool up_ok = hi + 1 <= n && g_up <= m + n;
    const bool dn_ok = 1 - lo <= m && g_dn <= m + n;
    for (int side = 0; side < 2; ++side) {
        if (side == 0 ? !up_ok : !dn_ok) continue;
        const int64_t g = side == 0 ? g_up : g_dn;
        const int64_t k = (m + n - g) / 2;
        const int64_t v = (int64_t)match * k + (int64_t)gap * (m + n - 2 * k);
        best = any ? std::max(best, v) : v;
        any = true;
    }
    *bound = best;
    return any;
}

// The certificate on a banded score S_b of half-width w: the score is exact
// when S_b >= U, the alignment when S_b > U (a tie outside the band could
// win the diagonal-first order); no bound when no path can leave the band.
bool band_certifies(int64_t m, int64_t n, int64_t w, int32_t sb, const nw_scoring &sc, bool want) {
    int64_t U = 0;
    const bool leave = band_exit_bound(m, n, w, sc.match, sc.gap, &U);
    return !leave || (want ? (int64_t)sb > U : (int64_t)sb >= U);
}

// The next half-width after S_b failed at w: at least double, and at least
// the smallest w' whose bound lies below S_b -- a wider band scores no less,
// so w' certifies for sure.
uint32_t band_next_width(uint32_t m, uint32_t n, uint32_t w, int32_t sb, const nw_scoring &sc, bool want) {
    uint32_t lo_w = w + 1, hi_w = std::max(m, n) + 1;
    while (lo_w < hi_w) {
        const uint32_t mid = lo_w + (hi_w - lo_w) / 2;
        if (band_certifies(m, n, mid, sb, sc, want)) hi_w = mid;
        else lo_w = mid + 1;
    }
    return std::max(2 * w, lo_w);
}

// Band of half-width w for an m x n pair: diagonals and the stripe period.
static void band_task(BatchTask &t, int R, uint32_t w) {
    const int64_t delta = (int64_t)t.n - t.m;
    t.lo = (int32_t)(std::min<int64_t>(0, delta) - w);
    t.hi = (int32_t)(std::max<int64_t>(0, delta) + w);
    const uint32_t SH = 32u * R;
    const uint64_t width = std::min<uint64_t>((uint64_t)t.n, (uint64_t)SH + (uint64_t)(t.hi - t.lo));
    t.period = (uint32_t)std::max<uint64_t>(width, SH + kMinPeriod);
}

// Cell slots the banded warp steps through (its time and pointer memory).
static uint64_t band_cells(const BatchTask &t, int R) {
    const uint32_t SH = 32u * R;
    return (uint64_t)((t.m + SH - 1) / SH) * SH * t.period;
}

// Cells the banded kernel actually updates: per stripe, 32R rows times its
// columns [max(0, s*32R + lo), min(n-1, s*32R + 32R - 1 + hi)].
static uint64_t band_cells_updated(const BatchTask &t, int R) {
    const int64_t SH = 32 * R;
    const int64_t S = ((int64_t)t.m + SH - 1) / SH;
    uint64_t cells = 0;
    for (int64_t s = 0; s < S; ++s) {
        const int64_t cb = std::max<int64_t>(0, s * SH + t.lo);
        const int64_t ce = std::min<int64_t>((int64_t)t.n - 1, s * SH + SH - 1 + t.hi);
        if (ce >= cb) cells += (uint64_t)(ce - cb + 1) * (uint64_t)SH;
    }
    return cells;
}

static uint64_t full_cells(const BatchTask &t, int R) {
    const uint32_t SH = 32u * R;
    return (uint64_t)((t.m + SH - 1) / SH) * SH * std::max(t.n, kMinPeriod);
}

}  // namespace nw

using namespace nw;

// Full-grid batch over the pairs ids[0..count) (ids == nullptr: 0..count-1)
// of the caller's arrays; results go to the caller's slots of those ids.
int batch_device_impl(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                      const uint64_t *b_off, const uint32_t *b_len, const uint32_t *ids, uint32_t count,
                      const nw_scoring &sc, uint32_t flags, int32_t *scores, char *cigar_pool,
                      const uint64_t *cigar_off, uint64_t *cigar_len);

// One banded round on the bit-sliced window kernel (nw_bits_band.cu) for
// the items (half-widths iw): pairs that would keep the GPU waiting on one
// warp go to `rest` (the full kernels), the others run in waves bounded by
// pointer memory; each wave's certified pairs are walked into CIGARs, the
// others return in next / nextw with their next widths.
static int bits_round(nw_ctx *ctx, const uint8_t *pool, const PlaneSet &planes, std::vector<BandBitsItem> &items, std::vector<uint32_t> &iw, int round, const nw_scoring &sc,
                      uint32_t flags, int32_t *scores, uint32_t score_cap, char *cigar_pool, const uint64_t *cigar_off,
                      uint64_t *cigar_len, std::vector<uint32_t> &next, std::vector<uint32_t> &nextw,
                      std::vector<uint32_t> &rest) {
    const bool want = flags & NW_CIGAR;
    int rc;
    HostTimer ht_prep(ctx, "bband_round_prep");
    {
        // pairs that would take longer on their warp than the whole round
        // ideally takes (the GPU's 4 x 152 schedulers busy) spread their
        // window over more lanes (NW_BBAND_FAST=0 keeps every pair on the
        // throughput shape)
        const char *fe = getenv("NW_BBAND_FAST");
        const bool fast_on = !(fe && *fe == '0');
        double total = 0;
        for (const auto &it : items) total += band_bits_seconds(it.shape);
        const double ideal = total / (4.0 * ctx->sm_count);
        for (auto &it : items)
            if (fast_on && band_bits_seconds(it.shape) > ideal) band_bits_fast(&it.shape);
    }
    {
        // one warp of this kernel runs its pair at about the scalar batch
        // kernel's per-warp rate; the whole kernel fills the GPU's 4 x 152
        // schedulers
        std::vector<double> wc(items.size()), fc(items.size());
        std::vector<PairCost> ps(items.size());
        for (size_t q = 0; q < items.size(); ++q) {
            wc[q] = band_bits_seconds(items[q].shape) * kWarpRate;
            fc[q] = (double)items[q].m * items[q].n;
            ps[q] = single_pair_cost(items[q].m, items[q].n, sc);
        }
        const std::vector<size_t> strag = band_keep_all()
                                              ? std::vector<size_t>()
                                              : pick_stragglers(wc, fc, ps, ctx->sm_count, kWarpRate * 4.0 * ctx->sm_count);
        if (!strag.empty()) {
            std::vector<char> routed(items.size(), 0);
            for (size_t q : strag) {
                routed[q] = 1;
                rest.push_back(items[q].out0);
            }
            std::vector<BandBitsItem> keep;
            std::vector<uint32_t> keep_w;
            for (size_t q = 0; q < items.size(); ++q)
                if (!routed[q]) {
                    keep.push_back(items[q]);
                    keep_w.push_back(iw[q]);
                }
            items.swap(keep);
            iw.swap(keep_w);
        }
    }
    if (round == 0) ctx->band_stats[0] += items.size();
    ht_prep.stop();
    const uint64_t wave_budget = scratch_headroom(ctx, "bband_ptr") / 2;
    size_t k0 = 0;
    while (k0 < items.size()) {
        std::vector<BandBitsItem> wave;
        std::vector<uint32_t> ww;
        uint64_t recs = 0;
        size_t k = k0;
        for (; k < items.size(); ++k) {
            BandBitsItem it = items[k];
            const uint64_t r = band_bits_records(it.shape);
            if (want) {
                if (!wave.empty() && (recs + r) * 16 > wave_budget) break;
                it.ptr_off = recs;
                recs += r;
            }
            ctx->band_stats[6] += r * 64u;  // cells: 2 anti-diagonals x 32 rows per record
            wave.push_back(it);
            ww.push_back(iw[k]);
        }
        void *pv = nullptr;
        if (want && (rc = scratch(ctx, "bband_ptr", recs * 16 + 16, &pv))) return rc;
        std::vector<int32_t> hs;
        if ((rc = band_bits_fill(ctx, planes, wave, want, sc.gap, scores, score_cap, pv, recs, hs)))
            return rc;
        std::vector<uint32_t> cert;
        for (size_t q = 0; q < wave.size(); ++q) {
            const BandBitsItem &it = wave[q];
            const uint32_t w = ww[q];
            if (!band_certifies(it.m, it.n, w, hs[q], sc, want)) {
                // the next round's width, kept within the window kernel's
                // reach while this round was below it: a narrower band than
                // the guaranteed one often certifies too, and a failed round
                // on this kernel costs less than the scalar banded kernel
                uint32_t nwid = band_next_width(it.m, it.n, w, hs[q], sc, want);
                const uint32_t cap = band_bits_max_width(it.m, it.n);
                if (nwid > cap && w < cap) nwid = cap;
                next.push_back(it.out0);
                nextw.push_back(nwid);
                continue;
            }
            ctx->band_stats[1 + round] += 1;
            if (it.out0 < ctx->band_round.size()) {
                ctx->band_round[it.out0] = (uint8_t)(round + 1);
                ctx->band_w_cert[it.out0] = w;
            }
            cert.push_back((uint32_t)q);
        }
        if (want && (rc = band_bits_walk(ctx, pv, wave, cert, pool, cigar_pool, cigar_off, cigar_len,
                                         (flags & NW_CIGAR_M) ? 1u : 0u)))
            return rc;
        k0 = k;
    }
    return NW_OK;
}

// The planar copy of a call's sequences for the window kernel, with each
// pair's two slots by pair id.  Its table (the distinct sequences and their
// slots) is built on the host once per call: by the learned-band entry while
// the feature and network kernels run, else by the rounds, which then
// upload it and launch the copy.
struct BandPlanes {
    bool added = false;
    PlaneSet planes;
    std::vector<int64_t> a_slot, b_slot;  // by pair id
};

static void add_band_planes(nw_ctx *ctx, const uint64_t *a_off, const uint32_t *a_len, const uint64_t *b_off,
                            const uint32_t *b_len, const std::vector<uint32_t> &ids, BandPlanes &bp) {
    HostTimer htp(ctx, "bband_planes");
    uint32_t cap = 0;
    for (uint32_t id : ids) cap = std::max(cap, id + 1);
    bp.planes.reserve(2 * ids.size());
    bp.a_slot.assign(cap, 0);
    bp.b_slot.assign(cap, 0);
    for (uint32_t id : ids) {
        bp.a_slot[id] = bp.planes.add(a_off[id], a_len[id]);
        bp.b_slot[id] = bp.planes.add(b_off[id], b_len[id]);
    }
    bp.added = true;
}

// Banded rounds for the pairs in `ids` with starting half-widths w0[k]; the
// pairs no round certifies are appended to `rest` for the full kernel.  `bp`
// holds the planar copy of the pairs' sequences when the caller built it.
static int band_rounds(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                       const uint64_t *b_off, const uint32_t *b_len, const std::vector<uint32_t> &ids,
                       const std::vector<uint32_t> &w0, const nw_scoring &sc, uint32_t flags, int32_t *scores,
                       char *cigar_pool, const uint64_t *cigar_off, uint64_t *cigar_len, std::vector<uint32_t> &rest,
                       BandPlanes &bp) {
    HostTimer ht_all(ctx, "band_rounds");
    const Profile pf = make_profile(sc);
    const bool want = flags & NW_CIGAR;
    // 512-row stripes: measured on GB300 (20,000 pairs of 2-20 kb) the
    // banded kernel takes 2.3x less time than with 256-row stripes for about
    // the same cells (NW_BAND_R = 4 or 8 for sweeps)
    int R = 16;
    if (const char *e = getenv("NW_BAND_R")) R = atoi(e) == 8 ? 8 : atoi(e) == 4 ? 4 : 16;
    constexpr int kRounds = 3;
    int rc;
    std::vector<uint32_t> pending(ids), width(w0);
    std::vector<int32_t> hs;
    uint32_t npairs_total = 0;  // banded scores by pair id
    for (uint32_t id : ids) npairs_total = std::max(npairs_total, id + 1);
    std::vector<int32_t> by_id;
    const bool band_log = getenv("NW_BAND_LOG") != nullptr;
    // the full kernels' pointer slots are idle until the fallback: give their
    // memory to the banded waves (it stays in the context's pool)
    if (want) {
        free_prefix(ctx, "batch_ptr");
        free_prefix(ctx, "ptr");
    }
    // the paper's scoring (s' = 3 on a match, 1 on a mismatch) runs on the
    // bit-sliced window kernel, from a planar copy of the pool;
    // NW_BAND_SCALAR=1 keeps every round on the scalar banded kernel (for
    // comparisons)
    const bool use_bits = sc.match - 2 * sc.gap == 3 && sc.mismatch - 2 * sc.gap == 1 && !getenv("NW_BAND_SCALAR");
    uint32_t score_cap_all = 0;
    for (uint32_t id : ids) score_cap_all = std::max(score_cap_all, id + 1);
    if (use_bits) {
        if (!bp.added) add_band_planes(ctx, a_off, a_len, b_off, b_len, ids, bp);
        HostTimer htp(ctx, "bband_planes_copy");
        if ((rc = bp.planes.launch(ctx, pool, "bband"))) return rc;
    }
    const PlaneSet &planes = bp.planes;
    for (int round = 0; round < kRounds && !pending.empty(); ++round) {
        size_t routed_full = 0;
        // the previous round's pointer words are traced already (stream
        // order): the scalar kernel's slot does not count against this
        // round's waves.  The window kernel's slot is kept and reused: its
        // waves budget it by its own headroom, and freeing it while the last
        // walk still reads it would have the pool map fresh memory for the
        // next round instead of reusing it.
        if (want) free_prefix(ctx, "band_ptr");
        // pairs whose band would cover most of the grid go straight to full
        HostTimer hti(ctx, "bband_items");
        std::vector<BatchTask> tasks;
        std::vector<uint32_t> tw;  // width used per task
        std::vector<uint32_t> next, nextw;  // rejected pairs and their next widths
        for (size_t q = 0; q < pending.size(); ++q) {
            const uint32_t id = pending[q];
            BatchTask t{};
            t.a_off = a_off[id];
            t.b_off = b_off[id];
            t.m = a_len[id];
            t.n = b_len[id];
            t.out0 = id;
            t.out1 = ~0u;
            const uint32_t w = width[q];
            if (t.m == 0 || t.n == 0) {
                rest.push_back(id);
                continue;
            }
            band_task(t, R, w);
            // (a banded cell costs about what a full-grid cell costs, so the
            // band pays off up to ~85% of the grid)
            if (band_cells(t, R) * 20 >= full_cells(t, R) * 17 ||
                (want && band_cells(t, R) / 4 > (ctx->budget - std::min(ctx->budget, ctx->used)) / 2)) {
                rest.push_back(id);
                continue;
            }
            tasks.push_back(t);
            tw.push_back(width[q]);
        }
        if (use_bits && !tasks.empty()) {
            // every pair whose band fits the window kernel (at most 8,192 rows)
            std::vector<BandBitsItem> items;
            std::vector<uint32_t> iw, keep_w;
            std::vector<BatchTask> keep;
            const int max_q = band_bits_max_q();
            for (size_t q = 0; q < tasks.size(); ++q) {
                const BatchTask &t = tasks[q];
                BandBitsShape sh;
                BatchTask tb = t;
                uint32_t wq = tw[q];
                const uint32_t cap = band_bits_max_width(t.m, t.n);
                if (wq > cap && cap > 0) {
                    if (round == 0) {
                        // a starting width beyond the window (a prediction that
                        // the pair needs a wider band): straight to the full kernel
                        rest.push_back(t.out0);
                        continue;
                    }
                    // a next width beyond it: the window's widest band first
                    // (the guaranteed width is often wider than needed)
                    wq = cap;
                    band_task(tb, R, wq);
                }
                if (band_bits_shape(tb.m, tb.n, tb.lo, tb.hi, &sh, max_q)) {
                    items.push_back(BandBitsItem{tb.a_off, tb.b_off, 0, bp.a_slot[tb.out0], bp.b_slot[tb.out0], tb.m,
                                                 tb.n, tb.out0, sh});
                    iw.push_back(wq);
                } else {
                    keep.push_back(t);
                    keep_w.push_back(tw[q]);
                }
            }
            tasks.swap(keep);
            tw.swap(keep_w);
            hti.stop();
            if (!items.empty() &&
                (rc = bits_round(ctx, pool, planes, items, iw, round, sc, flags, scores, score_cap_all,
                                 cigar_pool, cigar_off, cigar_len, next, nextw, rest)))
                return rc;
        }
        {
            // banded pairs that would leave the GPU idle on one warp run full
            // on the single-pair kernel instead (counted as fallbacks); a
            // banded warp is ~1.5x slower per cell than a full-grid one
            std::vector<double> wc(tasks.size()), fc(tasks.size());
            std::vector<PairCost> ps(tasks.size());
            for (size_t q = 0; q < tasks.size(); ++q) {
                wc[q] = 1.5 * (double)band_cells(tasks[q], R);
                fc[q] = (double)tasks[q].m * tasks[q].n;
                ps[q] = single_pair_cost(tasks[q].m, tasks[q].n, sc);
            }
            const std::vector<size_t> strag =
                band_keep_all() ? std::vector<size_t>() : pick_stragglers(wc, fc, ps, ctx->sm_count);
            routed_full = strag.size();
            if (!strag.empty()) {
                std::vector<char> routed(tasks.size(), 0);
                for (size_t q : strag) {
                    routed[q] = 1;
                    rest.push_back(tasks[q].out0);
                }
                std::vector<BatchTask> keep;
                std::vector<uint32_t> keep_w;
                for (size_t q = 0; q < tasks.size(); ++q)
                    if (!routed[q]) {
                        keep.push_back(tasks[q]);
                        keep_w.push_back(tw[q]);
                    }
                tasks.swap(keep);
                tw.swap(keep_w);
            }
        }
        ctx->band_stats[0] += round == 0 ? tasks.size() : 0;
        // waves bounded by pointer memory (score-only: one wave)
        const uint64_t wave_budget = (ctx->budget - std::min(ctx->budget, ctx->used)) / 2;
        size_t k0 = 0;
        while (k0 < tasks.size()) {
            std::vector<BatchTask> wave;
            uint64_t words = 0, mvbytes = 0;
            uint32_t max_n = 1;
            size_t k = k0;
            for (; k < tasks.size(); ++k) {
                BatchTask t = tasks[k];
                if (want) {
                    const uint32_t SH = 32u * R;
                    t.ncg = ptr_words_per_lane_row(t.period, R);
                    const uint64_t wds = (uint64_t)((t.m + SH - 1) / SH) * 32u * t.ncg;
                    if (!wave.empty() && (words + wds) * 4 > wave_budget) break;
                    t.ptr_off = words;
                    words += wds;
                    mvbytes += (uint64_t)t.m + t.n + 16;
                }
                max_n = std::max(max_n, t.n);
                ctx->band_stats[6] += band_cells_updated(t, R);
                wave.push_back(t);
            }
            void *pv = nullptr, *mv = nullptr, *nm = nullptr;
            if (want) {
                if ((rc = scratch(ctx, "band_ptr", words * 4 + 16, &pv))) return rc;
                if ((rc = scratch(ctx, "band_moves", mvbytes + 16, &mv))) return rc;
                if ((rc = scratch(ctx, "band_nmoves", wave.size() * 8 + 16, &nm))) return rc;
            }
            std::vector<BatchTask> fill = wave;
            sort_lpt(fill);
            const auto wave_t0 = std::chrono::steady_clock::now();
            BatchTask *dt = nullptr;
            if ((rc = upload(ctx, "band_tasks", fill, &dt))) return rc;
            BatchArgs ba{};
            ba.pool = pool;
            for (int c = 0; c < 4; ++c) ba.prof[c] = pf.prof[c];
            ba.gap = pf.gap;
            ba.scores = scores;
            ba.err = ctx->d_err;
            ba.tasks = dt;
            ba.ntasks = (uint32_t)fill.size();
            ba.ptr = (uint32_t *)pv;
            ba.ptr_cap = words;
            ba.score_cap = score_slots(fill.data(), (uint32_t)fill.size());
            if ((rc = launch_batch(ctx, R, want, ba, max_n, 2))) return rc;
            // certificate on the banded scores: one gather, one copy back
            {
                void *g = nullptr;
                if ((rc = scratch(ctx, "band_gather", fill.size() * 4 + 16, &g))) return rc;
                {
                    LaunchTimer t(ctx, "gather");
                    k_gather_scores<<<(unsigned)((fill.size() + 255) / 256), 256, 0, ctx->stream>>>(
                        dt, (uint32_t)fill.size(), scores, (int32_t *)g);
                }
                std::vector<int32_t> gs(fill.size());
                cudaError_t e = cudaMemcpyAsync(gs.data(), g, fill.size() * 4, cudaMemcpyDeviceToHost, ctx->stream);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "banded score D2H");
                {
                    HostTimer ht(ctx, "band_wait");  // the banded fill itself, seen from the host
                    if ((rc = nw_ctx_sync(ctx))) return rc;
                }
                if (band_log) {  // diagnostics: one line per banded wave
                    double sum = 0, mx = 0;
                    for (const BatchTask &t : fill) {
                        const double c = (double)band_cells_updated(t, R);
                        sum += c;
                        mx = std::max(mx, c);
                    }
                    const double ms =
                        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wave_t0).count();
                    fprintf(stderr,
                            "[nw band] round %d wave %zu pairs (%zu routed full) cells %.3g max %.3g (m %u n %u) "
                            "%.2f ms; scratch in use %.3g of %.3g B\n",
                            round, fill.size(), routed_full, sum, mx, fill.empty() ? 0u : fill[0].m,
                            fill.empty() ? 0u : fill[0].n, ms, (double)ctx->used, (double)ctx->budget);
                }
                if (by_id.empty()) by_id.assign(npairs_total, 0);
                for (size_t q = 0; q < fill.size(); ++q) by_id[fill[q].out0] = gs[q];
                hs.resize(wave.size());
                for (size_t q = 0; q < wave.size(); ++q) hs[q] = by_id[wave[q].out0];
            }
            std::vector<TraceTask> tt;
            for (size_t q = 0; q < wave.size(); ++q) {
                const BatchTask &t = wave[q];
                const uint32_t w = tw[k0 + q];
                if (!band_certifies(t.m, t.n, w, hs[q], sc, want)) {
                    next.push_back(t.out0);
                    nextw.push_back(band_next_width(t.m, t.n, w, hs[q], sc, want));
                    continue;
                }
                ctx->band_stats[1 + round] += 1;
                if (t.out0 < ctx->band_round.size()) {
                    ctx->band_round[t.out0] = (uint8_t)(round + 1);
                    ctx->band_w_cert[t.out0] = w;
                }
                if (want) {
                    const uint32_t id = t.out0;
                    tt.push_back(TraceTask{(const uint32_t *)pv + t.ptr_off, t.ncg, t.m, t.n,
                                           (uint8_t *)mv + 0, (uint64_t *)nm + tt.size(), pool + t.a_off,
                                           pool + t.b_off, cigar_pool + cigar_off[id], cigar_len + id, t.lo});
                }
            }
            if (want && !tt.empty()) {
                uint64_t mpos = 0;
                for (auto &x : tt) {
                    x.moves = (uint8_t *)mv + mpos;
                    mpos += (uint64_t)x.m + x.n + 16;
                }
                TraceTask *dtt = nullptr;
                if ((rc = upload(ctx, "band_trace_tasks", tt, &dtt))) return rc;
                if ((rc = launch_trace(ctx, R, tt.data(), dtt, (uint32_t)tt.size(), (flags & NW_CIGAR_M) ? 1u : 0u)))
                    return rc;
            }
            k0 = k;
        }
        // widen: the rejected pairs with their next widths
        if (round + 1 < kRounds) {
            pending.swap(next);
            width.swap(nextw);
        } else {
            for (uint32_t id : next) rest.push_back(id);
            pending.clear();
        }
    }
    for (uint32_t id : pending) rest.push_back(id);
    return NW_OK;
}

// One banded round with the given half-widths, banded scores as they are
// (the inspection mode NW_BAND_RAW).
static int band_raw(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                    const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, const uint32_t *w,
                    const nw_scoring &sc, int32_t *scores) {
    const Profile pf = make_profile(sc);
    constexpr int R = 8;
    std::vector<BatchTask> tasks;
    uint32_t max_n = 1;
    for (uint32_t k = 0; k < npairs; ++k) {
        BatchTask t{};
        t.a_off = a_off[k];
        t.b_off = b_off[k];
        t.m = a_len[k];
        t.n = b_len[k];
        t.out0 = k;
        t.out1 = ~0u;
        band_task(t, R, std::max<uint32_t>(w[k], 0));
        max_n = std::max(max_n, t.n);
        tasks.push_back(t);
    }
    sort_lpt(tasks);
    BatchTask *dt = nullptr;
    int rc = upload(ctx, "band_tasks", tasks, &dt);
    if (rc) return rc;
    BatchArgs ba{};
    ba.pool = pool;
    for (int c = 0; c < 4; ++c) ba.prof[c] = pf.prof[c];
    ba.gap = pf.gap;
    ba.scores = scores;
    ba.err = ctx->d_err;
    ba.tasks = dt;
    ba.ntasks = npairs;
    ba.score_cap = npairs;
    return launch_batch(ctx, R, false, ba, max_n, 1);
}

// Certified band for every pair with the given starting half-widths, then
// the full kernel for whatever no band certified.
static int band_batch(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                      const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, const uint32_t *w0,
                      const nw_scoring &sc, uint32_t flags, int32_t *scores, char *cigar_pool,
                      const uint64_t *cigar_off, uint64_t *cigar_len, BandPlanes &bp) {
    std::vector<uint32_t> ids(npairs), width(npairs), rest;
    ctx->band_round.assign(npairs, 0);
    ctx->band_w_cert.assign(npairs, 0);
    ctx->band_w_first.resize(npairs);
    for (uint32_t k = 0; k < npairs; ++k) {
        ids[k] = k;
        width[k] = std::max<uint32_t>(w0[k], 1);
        ctx->band_w_first[k] = width[k];
        const BatchTask t{a_off[k], b_off[k], a_len[k], b_len[k]};
        ctx->band_stats[7] += full_cells(t, 8);
    }
    int rc = band_rounds(ctx, pool, a_off, a_len, b_off, b_len, ids, width, sc, flags, scores, cigar_pool, cigar_off,
                         cigar_len, rest, bp);
    if (rc || rest.empty()) return rc;
    // the banded pointer words are dead now: hand their memory to the full
    // kernel's waves (it stays in the context's pool for the next call)
    free_prefix(ctx, "band_ptr");
    HostTimer ht(ctx, "band_fallback");
    ctx->band_stats[5] += rest.size();
    return batch_device_impl(ctx, pool, a_off, a_len, b_off, b_len, rest.data(), (uint32_t)rest.size(), sc, flags,
                             scores, cigar_pool, cigar_off, cigar_len);
    return NW_OK;
}

// Score-only or CIGAR batch on device buffers (the C entry point stages
// host buffers around this).
int batch_device_impl(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                      const uint64_t *b_off, const uint32_t *b_len, const uint32_t *ids, uint32_t npairs,
                      const nw_scoring &sc, uint32_t flags, int32_t *scores, char *cigar_pool,
                      const uint64_t *cigar_off, uint64_t *cigar_len) {
    const Profile pf = make_profile(sc);
    const bool want = flags & NW_CIGAR;
    int rc;
    // NW_GRAPH (score-only calls on all the caller's pairs): a repeated call
    // replays the launches captured the first time
    bool graph = (flags & NW_GRAPH) && !want && !ids;
    std::string gkey, pre = "batch";
    if (graph) {
        uint64_t h = 1469598103934665603ull;
        h = hash_bytes(a_off, (size_t)npairs * 8, h);
        h = hash_bytes(a_len, (size_t)npairs * 4, h);
        h = hash_bytes(b_off, (size_t)npairs * 8, h);
        h = hash_bytes(b_len, (size_t)npairs * 4, h);
        gkey = batch_key("batch", pool, scores, npairs, sc, flags, h);
        bool replayed = false;
        if ((rc = graph_launch(ctx, gkey, "batch_score", 1, &replayed)) || replayed) return rc;
        pre = "g" + std::to_string(++ctx->graph_seq);
    }
    std::vector<BatchTask> tasks(npairs);
    uint32_t max_n = 1;
    for (uint32_t q = 0; q < npairs; ++q) {
        const uint32_t k = ids ? ids[q] : q;
        if ((rc = check_len(ctx, sc, a_len[k], b_len[k]))) return rc;
        if (want && cigar_off[k + 1] - cigar_off[k] < nw_cigar_bound(a_len[k], b_len[k]))
            return fail(ctx, NW_ERR_ARG, "CIGAR capacity of pair %u below its bound", k);
        BatchTask t{};
        t.a_off = a_off[k];
        t.b_off = b_off[k];
        t.m = a_len[k];
        t.n = b_len[k];
        // score-only: the optimum is symmetric, so put the sequence whose
        // stripes waste fewer padded rows on the rows
        if (!want && t.m > 0 && t.n > 0) {
            const uint32_t SH = 256;
            const uint32_t wm = (t.m + SH - 1) / SH * SH - t.m, wn = (t.n + SH - 1) / SH * SH - t.n;
            if (wn * (uint64_t)t.m < wm * (uint64_t)t.n && t.m >= kMinPeriod) {
                std::swap(t.a_off, t.b_off);
                std::swap(t.m, t.n);
            }
        }
        t.out0 = k;
        t.out1 = ~0u;
        max_n = std::max(max_n, t.n);
        tasks[q] = t;
    }
    // pairs that would leave the GPU idle on one warp take the single-pair
    // kernel, and so do pairs whose pointer matrix alone exceeds half the
    // remaining budget (the single-pair path recomputes from checkpoints)
    {
        std::vector<double> wc(tasks.size()), fc(tasks.size());
        std::vector<PairCost> ps(tasks.size());
        for (size_t q = 0; q < tasks.size(); ++q) {
            wc[q] = fc[q] = (double)tasks[q].m * tasks[q].n;
            ps[q] = single_pair_cost(tasks[q].m, tasks[q].n, sc);
        }
        std::vector<size_t> strag = pick_stragglers(wc, fc, ps, ctx->sm_count);
        if (want) {
            const uint64_t room = (ctx->budget - std::min(ctx->budget, ctx->used)) / 2;
            std::vector<char> in(tasks.size(), 0);
            for (size_t q : strag) in[q] = 1;
            for (size_t q = 0; q < tasks.size(); ++q)
                if (!in[q] && ((uint64_t)tasks[q].m + 512) * ((uint64_t)tasks[q].n + 128) / 4 > room) strag.push_back(q);
        }
        if (!strag.empty()) {
            std::vector<char> routed(tasks.size(), 0);
            std::vector<BatchTask> st;
            for (size_t q : strag) {
                st.push_back(tasks[q]);
                routed[q] = 1;
            }
            if ((rc = run_stragglers(ctx, pool, st, sc, flags, scores, cigar_pool, cigar_off, cigar_len))) return rc;
            std::vector<BatchTask> keep;
            for (size_t q = 0; q < tasks.size(); ++q)
                if (!routed[q]) keep.push_back(tasks[q]);
            graph = false;  // the single-pair launches are not captured
            if (keep.empty()) return NW_OK;
            tasks.swap(keep);
            npairs = (uint32_t)tasks.size();
            max_n = 1;
            for (const auto &t : tasks) max_n = std::max(max_n, t.n);
        }
    }
    BatchArgs ba{};
    ba.pool = pool;
    for (int c = 0; c < 4; ++c) ba.prof[c] = pf.prof[c];
    ba.gap = pf.gap;
    ba.scores = scores;
    ba.err = ctx->d_err;
    // rows per lane: the padding-cost model, or the autotuner's measured
    // choice (tuned on score-only launches of the whole list)
    int R = pick_rows(tasks);
    if (!want || ctx->autotune) {
        std::vector<BatchTask> lpt = tasks;
        sort_lpt(lpt);
        BatchTask *dt = nullptr;
        if ((rc = upload(ctx, (pre + "_tasks").c_str(), lpt, &dt))) return rc;
        BatchArgs bs = ba;
        bs.tasks = dt;
        bs.ntasks = npairs;
        bs.score_cap = score_slots(lpt.data(), npairs);
        // score-only: the bit-sliced kernel (rows per lane 32) where the
        // scoring fits two bit planes
        const bool bits = !want && bits_scoring_ok(sc);
        BitsPlan bp;
        if (bits) {
            std::vector<BatchTask> bt = lpt;
            if ((rc = bits_prepare(ctx, pool, bt, sc, scores, bs.score_cap, pre, &bp))) return rc;
        }
        auto run = [&](int r) { return r == 32 ? bits_launch(ctx, bp) : launch_batch(ctx, r, false, bs, max_n, 0, pre); };
        if ((rc = tune_rows(ctx, lpt, bits ? 32 : R, run, &R, bits))) return rc;
        if (!want) {
            auto launches = [&]() -> int { return run(R); };
            if ((rc = launches())) return rc;
            if (graph)
                return capture_graph(ctx, gkey, pre, R == 32 ? "bits_score" : "batch_score", R == 32 ? 2 : 1, launches);
            return NW_OK;
        }
    }
    // CIGAR: waves whose pointer words fit half of the remaining budget.
    // (a wave always takes at least one pair; scratch() reports NW_ERR_OOM if
    // even that does not fit)
    const uint64_t wave_budget = (ctx->budget - std::min(ctx->budget, ctx->used)) / 2;
    // waves in longest-first order: pairs of similar size run together, so a
    // wave's time is not set by one long pair among many short ones; within
    // a wave, the pairs that would keep it waiting on one warp go to the
    // multi-warp kernel (same rule as for the whole batch)
    std::vector<uint32_t> order(npairs);
    std::iota(order.begin(), order.end(), 0u);  // positions in `tasks`
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        return (uint64_t)tasks[x].m * tasks[x].n > (uint64_t)tasks[y].m * tasks[y].n;
    });
    size_t k0 = 0;
    while (k0 < npairs) {
        std::vector<BatchTask> wave;
        std::vector<uint32_t> ids_w;
        uint64_t words = 0, mvbytes = 0;
        size_t k = k0;
        for (; k < npairs; ++k) {
            BatchTask t = tasks[order[k]];  // t.out0 is the caller's pair id
            const uint32_t SH = 32u * R;
            t.ncg = ptr_words_per_lane_row(std::max(t.n, 1u), R);
            const uint64_t w = (uint64_t)((t.m + SH - 1) / SH) * 32u * t.ncg;
            if (!wave.empty() && (words + w) * 4 > wave_budget) break;
            t.ptr_off = words;
            words += w;
            mvbytes += (uint64_t)t.m + t.n + 16;
            wave.push_back(t);
            ids_w.push_back(t.out0);
        }
        if (k < npairs || k0 > 0) {  // a true wave (not the whole batch): route its stragglers
            std::vector<double> wc(wave.size());
            std::vector<PairCost> ps(wave.size());
            for (size_t q = 0; q < wave.size(); ++q) {
                wc[q] = (double)wave[q].m * wave[q].n;
                ps[q] = single_pair_cost(wave[q].m, wave[q].n, sc);
            }
            const std::vector<size_t> strag = pick_stragglers(wc, wc, ps, ctx->sm_count);
            if (!strag.empty() && strag.size() < wave.size()) {
                std::vector<char> routed(wave.size(), 0);
                std::vector<BatchTask> st;
                for (size_t q : strag) {
                    st.push_back(wave[q]);
                    routed[q] = 1;
                }
                if ((rc = run_stragglers(ctx, pool, st, sc, flags, scores, cigar_pool, cigar_off, cigar_len)))
                    return rc;
                std::vector<BatchTask> keep;
                std::vector<uint32_t> keep_ids;
                for (size_t q = 0; q < wave.size(); ++q)
                    if (!routed[q]) {
                        keep.push_back(wave[q]);
                        keep_ids.push_back(ids_w[q]);
                    }
                wave.swap(keep);
                ids_w.swap(keep_ids);
            }
        }
        void *pv = nullptr, *mv = nullptr, *nm = nullptr;
        if ((rc = scratch(ctx, "batch_ptr", words * 4 + 16, &pv))) return rc;
        if ((rc = scratch(ctx, "batch_moves", mvbytes + 16, &mv))) return rc;
        if ((rc = scratch(ctx, "batch_nmoves", wave.size() * 8 + 16, &nm))) return rc;
        std::vector<TraceTask> tt(wave.size());
        uint64_t mpos = 0;
        for (size_t q = 0; q < wave.size(); ++q) {
            const BatchTask &t = wave[q];
            const uint32_t id = ids_w[q];
            tt[q] = TraceTask{(const uint32_t *)pv + t.ptr_off, t.ncg, t.m, t.n, (uint8_t *)mv + mpos,
                              (uint64_t *)nm + q, pool + t.a_off, pool + t.b_off, cigar_pool + cigar_off[id],
                              cigar_len + id, kNoBand};
            mpos += (uint64_t)t.m + t.n + 16;
        }
        // order the fill by cell count; ptr_off stays attached to each task
        std::vector<BatchTask> fill = wave;
        sort_lpt(fill);
        BatchTask *dt = nullptr;
        TraceTask *dtt = nullptr;
        if ((rc = upload(ctx, "batch_tasks", fill, &dt))) return rc;
        if ((rc = upload(ctx, "batch_trace_tasks", tt, &dtt))) return rc;
        ba.tasks = dt;
        ba.ntasks = (uint32_t)fill.size();
        ba.ptr = (uint32_t *)pv;
        ba.ptr_cap = words;
        ba.score_cap = score_slots(fill.data(), (uint32_t)fill.size());
        uint32_t wave_max_n = 1;
        for (const auto &t : wave) wave_max_n = std::max(wave_max_n, t.n);
        if ((rc = launch_batch(ctx, R, true, ba, wave_max_n))) return rc;
        if ((rc = launch_trace(ctx, R, tt.data(), dtt, (uint32_t)tt.size(), (flags & NW_CIGAR_M) ? 1u : 0u))) return rc;
        k0 = k;
    }
    return NW_OK;
}

// The CIGARs of a host-I/O batch, packed back to back (pair k's bytes at
// dst_off[k]) so that only the bytes written cross to the host.
__global__ void k_pack_cigars(const char *src, const uint64_t *src_off, const uint64_t *len, const uint64_t *dst_off,
                              uint32_t n, char *dst) {
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += (gridDim.x * blockDim.x) >> 5) {
        const char *s = src + src_off[k];
        char *d = dst + dst_off[k];
        for (uint64_t i = lane; i < len[k]; i += 32) d[i] = s[i];
    }
}

// Host-I/O staging shared by the batch entry points: copy the pool in, run
// `body` on device buffers, copy the scores out and the CIGARs' written
// bytes (packed on the device, one copy), place them at the caller's
// offsets, wait.
template <typename F>
static int with_host_io(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                        const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, uint32_t flags,
                        int32_t *scores, char *cigar_pool, const uint64_t *cigar_off, uint64_t *cigar_len, F body) {
    const bool want = flags & NW_CIGAR;
    int rc;
    uint64_t pool_bytes = 16;
    for (uint32_t k = 0; k < npairs; ++k) {
        pool_bytes = std::max<uint64_t>(pool_bytes, a_off[k] + (a_len[k] + 3) / 4);
        pool_bytes = std::max<uint64_t>(pool_bytes, b_off[k] + (b_len[k] + 3) / 4);
    }
    void *dpool = nullptr, *dsc = nullptr, *dcig = nullptr, *dlen = nullptr;
    if ((rc = to_device(ctx, pool2b, pool_bytes, "hio_pool", &dpool))) return rc;
    if ((rc = scratch(ctx, "hio_scores", (size_t)npairs * 4, &dsc))) return rc;
    if (want) {
        if ((rc = scratch(ctx, "hio_cigar", cigar_off[npairs] + 16, &dcig))) return rc;
        if ((rc = scratch(ctx, "hio_cigar_len", (size_t)npairs * 8, &dlen))) return rc;
    }
    rc = body((const uint8_t *)dpool, (int32_t *)dsc, (char *)dcig, (uint64_t *)dlen);
    if (rc) return rc;
    cudaMemcpyAsync(scores, dsc, (size_t)npairs * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (!want) return nw_ctx_sync(ctx);
    cudaMemcpyAsync(cigar_len, dlen, (size_t)npairs * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if ((rc = nw_ctx_sync(ctx))) return rc;
    std::vector<uint64_t> packed(npairs + 1, 0);
    for (uint32_t k = 0; k < npairs; ++k) {
        if (cigar_len[k] > cigar_off[k + 1] - cigar_off[k]) return fail(ctx, NW_ERR_CIGAR_TRUNC, "CIGAR %u", k);
        packed[k + 1] = packed[k] + cigar_len[k];
    }
    void *dsrc = nullptr, *ddst = nullptr, *dpk = nullptr;
    if ((rc = to_device(ctx, cigar_off, (size_t)npairs * 8, "hio_cigar_src", &dsrc))) return rc;
    if ((rc = to_device(ctx, packed.data(), (size_t)npairs * 8, "hio_cigar_dst", &ddst))) return rc;
    if ((rc = scratch(ctx, "hio_cigar_packed", packed[npairs] + 16, &dpk))) return rc;
    {
        LaunchTimer t(ctx, "pack_cigars");
        const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((npairs + 7) / 8, (uint32_t)ctx->sm_count * 8));
        k_pack_cigars<<<blocks, 256, 0, ctx->stream>>>((const char *)dcig, (const uint64_t *)dsrc,
                                                       (const uint64_t *)dlen, (const uint64_t *)ddst, npairs,
                                                       (char *)dpk);
    }
    void *hv = nullptr;  // the packed bytes land in pinned staging (one DMA, no zero fill)
    if ((rc = pinned_host(ctx, packed[npairs] + 16, &hv))) return rc;
    const char *host = (const char *)hv;
    if (packed[npairs]) cudaMemcpyAsync(hv, dpk, packed[npairs], cudaMemcpyDeviceToHost, ctx->stream);
    if ((rc = nw_ctx_sync(ctx))) return rc;
    for (uint32_t k = 0; k < npairs; ++k) {
        memcpy(cigar_pool + cigar_off[k], host + packed[k], cigar_len[k]);
        if (cigar_off[k] + cigar_len[k] < cigar_off[k + 1]) cigar_pool[cigar_off[k] + cigar_len[k]] = '\0';
    }
    return NW_OK;
}

static int check_batch_args(nw_ctx *ctx, const nw_scoring &sc, const uint8_t *pool2b, const uint64_t *a_off,
                            const uint32_t *a_len, const uint64_t *b_off, const uint32_t *b_len, uint32_t flags,
                            int32_t *scores, char *cigar_pool, const uint64_t *cigar_off, uint64_t *cigar_len) {
    int rc = check_common(ctx, sc);
    if (rc) return rc;
    if (!a_off || !a_len || !b_off || !b_len || !scores || !pool2b) return fail(ctx, NW_ERR_ARG, "null argument");
    if ((flags & NW_CIGAR) && (!cigar_pool || !cigar_off || !cigar_len))
        return fail(ctx, NW_ERR_ARG, "CIGAR buffers are null");
    return NW_OK;
}

int learned_band_widths(nw_ctx *ctx, const uint8_t *pool, const uint64_t *a_off, const uint32_t *a_len,
                        const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, std::vector<uint32_t> &w,
                        const std::function<int()> &overlap);

extern "C" int nw_align_batch(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                              const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, nw_scoring sc,
                              uint32_t flags, int32_t *scores, char *cigar_pool, const uint64_t *cigar_off,
                              uint64_t *cigar_len) {
    if (!ctx) return NW_ERR_ARG;
    if (npairs == 0) return check_common(ctx, sc);
    int rc = check_batch_args(ctx, sc, pool2b, a_off, a_len, b_off, b_len, flags, scores, cigar_pool, cigar_off,
                              cigar_len);
    if (rc) return rc;
    if ((flags & NW_GRAPH) && (flags & NW_HOST_IO)) return fail(ctx, NW_ERR_ARG, "NW_GRAPH needs device buffers");
    if ((flags & NW_LEARNED_BAND) && (rc = check_band_scoring(ctx, sc))) return rc;
    auto body = [&](const uint8_t *pool, int32_t *sc_out, char *cig, uint64_t *clen) -> int {
        const uint32_t fl = flags & ~NW_HOST_IO;
        if (!(flags & NW_LEARNED_BAND))
            return batch_device_impl(ctx, pool, a_off, a_len, b_off, b_len, nullptr, npairs, sc, fl, sc_out, cig,
                                     cigar_off, clen);
        std::vector<uint32_t> w;
        BandPlanes bp;
        int r;
        {
            // the table of the window kernel's planar copy is built on the
            // host while the feature and network kernels run (the paper's
            // scoring only)
            HostTimer ht(ctx, "band_widths");
            const bool bits = sc.match - 2 * sc.gap == 3 && sc.mismatch - 2 * sc.gap == 1 && !getenv("NW_BAND_SCALAR");
            std::vector<uint32_t> all(npairs);
            for (uint32_t k = 0; k < npairs; ++k) all[k] = k;
            r = learned_band_widths(ctx, pool, a_off, a_len, b_off, b_len, npairs, w, [&]() -> int {
                if (bits) add_band_planes(ctx, a_off, a_len, b_off, b_len, all, bp);
                return NW_OK;
            });
        }
        if (r) return r;
        return band_batch(ctx, pool, a_off, a_len, b_off, b_len, npairs, w.data(), sc, fl, sc_out, cig, cigar_off,
                          clen, bp);
    };
    if (!(flags & NW_HOST_IO)) return body(pool2b, scores, cigar_pool, cigar_len);
    return with_host_io(ctx, pool2b, a_off, a_len, b_off, b_len, npairs, flags, scores, cigar_pool, cigar_off,
                        cigar_len, body);
}

extern "C" int nw_align_batch_banded(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off,
                                     const uint32_t *a_len, const uint64_t *b_off, const uint32_t *b_len,
                                     uint32_t npairs, const uint32_t *band_w, nw_scoring sc, uint32_t flags,
                                     int32_t *scores, char *cigar_pool, const uint64_t *cigar_off,
                                     uint64_t *cigar_len) {
    if (!ctx) return NW_ERR_ARG;
    if (npairs == 0) return check_common(ctx, sc);
    int rc = check_batch_args(ctx, sc, pool2b, a_off, a_len, b_off, b_len, flags, scores, cigar_pool, cigar_off,
                              cigar_len);
    if (rc) return rc;
    if (!band_w) return fail(ctx, NW_ERR_ARG, "band widths are null");
    if ((rc = check_band_scoring(ctx, sc))) return rc;
    for (uint32_t k = 0; k < npairs; ++k)
        if ((rc = check_len(ctx, sc, a_len[k], b_len[k]))) return rc;
    if ((flags & NW_BAND_RAW) && (flags & NW_CIGAR)) return fail(ctx, NW_ERR_ARG, "NW_BAND_RAW is score only");
    auto body = [&](const uint8_t *pool, int32_t *sc_out, char *cig, uint64_t *clen) -> int {
        if (flags & NW_BAND_RAW) return band_raw(ctx, pool, a_off, a_len, b_off, b_len, npairs, band_w, sc, sc_out);
        BandPlanes bp;
        return band_batch(ctx, pool, a_off, a_len, b_off, b_len, npairs, band_w, sc, flags & ~NW_HOST_IO, sc_out, cig,
                          cigar_off, clen, bp);
    };
    if (!(flags & NW_HOST_IO)) return body(pool2b, scores, cigar_pool, cigar_len);
    return with_host_io(ctx, pool2b, a_off, a_len, b_off, b_len, npairs, flags, scores, cigar_pool, cigar_off,
                        cigar_len, body);
}

extern "C" int64_t nw_route_stragglers(const double *warp_cells, const double *full_cells, uint32_t n,
                                       uint32_t *out) {
    if (n && (!warp_cells || !full_cells || !out)) return -NW_ERR_ARG;
    const std::vector<size_t> r = pick_stragglers(std::vector<double>(warp_cells, warp_cells + n),
                                                  std::vector<double>(full_cells, full_cells + n), {}, 152);
    for (size_t k = 0; k < r.size(); ++k) out[k] = (uint32_t)r[k];
    return (int64_t)r.size();
}

extern "C" int nw_shard_pairs(const uint32_t *a_len, const uint32_t *b_len, uint32_t npairs, uint32_t nranks,
                              uint32_t *rank_of, uint64_t *load) {
    if (nranks == 0 || (npairs && (!a_len || !b_len || !rank_of))) return NW_ERR_ARG;
    // longest processing time first: pairs by cells, largest first (index
    // order among equals), each to the least loaded rank (lowest on ties)
    std::vector<uint32_t> order(npairs);
    std::iota(order.begin(), order.end(), 0u);
    auto cells = [&](uint32_t k) { return (uint64_t)a_len[k] * b_len[k]; };
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return cells(x) > cells(y); });
    std::vector<uint64_t> ld(nranks, 0);
    for (uint32_t k : order) {
        uint32_t best = 0;
        for (uint32_t r = 1; r < nranks; ++r)
            if (ld[r] < ld[best]) best = r;
        rank_of[k] = best;
        ld[best] += cells(k);
    }
    if (load)
        for (uint32_t r = 0; r < nranks; ++r) load[r] = ld[r];
    return NW_OK;
}

extern "C" int nw_ctx_band_stats(nw_ctx *ctx, uint64_t *out, int cap) {
    if (!ctx) return -NW_ERR_ARG;
    for (int k = 0; k < cap && k < 8; ++k) out[k] = ctx->band_stats[k];
    return 8;
}

extern "C" int64_t nw_ctx_band_outcome(nw_ctx *ctx, uint8_t *round, uint32_t *first_width, uint32_t *cert_width,
                                       uint64_t cap) {
    if (!ctx) return -NW_ERR_ARG;
    const uint64_t n = ctx->band_round.size();
    for (uint64_t k = 0; k < n && k < cap; ++k) {
        if (round) round[k] = ctx->band_round[k];
        if (first_width) first_width[k] = ctx->band_w_first[k];
        if (cert_width) cert_width[k] = ctx->band_w_cert[k];
    }
    return (int64_t)n;
}

extern "C" int nw_score_all_pairs(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *off, const uint32_t *len,
                                  uint32_t nseq, nw_scoring sc, uint32_t flags, int32_t *out) {
    int rc = check_common(ctx, sc);
    if (rc) return rc;
    if (nseq == 0) return NW_OK;
    if (!off || !len || !out || !pool2b) return fail(ctx, NW_ERR_ARG, "null argument");
    if (nseq > 65535) return fail(ctx, NW_ERR_ARG, "at most 65535 sequences");
    for (uint32_t i = 0; i < nseq; ++i)
        if ((rc = check_len(ctx, sc, len[i], len[i]))) return rc;
    const bool graph = flags & NW_GRAPH;
    const uint8_t *pool = pool2b;
    int32_t *dout = out;
    if (flags & NW_HOST_IO) {
        // host buffers: the pool goes to a device slot first (also before a
        // graph replay, which reads that slot), the matrix comes back at the end
        uint64_t pool_bytes = 16;
        for (uint32_t i = 0; i < nseq; ++i) pool_bytes = std::max<uint64_t>(pool_bytes, off[i] + (len[i] + 3) / 4);
        void *dp = nullptr, *dq = nullptr;
        if ((rc = to_device(ctx, pool2b, pool_bytes, "hio_pool", &dp))) return rc;
        if ((rc = scratch(ctx, "hio_matrix", (size_t)nseq * nseq * 4, &dq))) return rc;
        pool = (const uint8_t *)dp;
        dout = (int32_t *)dq;
    }
    auto copy_back = [&]() -> int {
        if (!(flags & NW_HOST_IO)) return NW_OK;
        cudaError_t e = cudaMemcpyAsync(out, dout, (size_t)nseq * nseq * 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "matrix D2H");
        return nw_ctx_sync(ctx);
    };
    std::string gkey, pre = "batch";
    if (graph) {
        // a repeated call replays its captured launches (keyed by the device
        // buffers they read and write)
        const uint64_t h = hash_bytes(len, (size_t)nseq * 4, hash_bytes(off, (size_t)nseq * 8, 1469598103934665603ull));
        gkey = batch_key("allpairs", pool, dout, nseq, sc, flags, h);
        bool replayed = false;
        if ((rc = graph_launch(ctx, gkey, "batch_score", 2, &replayed))) return rc;
        if (replayed) return copy_back();
        pre = "g" + std::to_string(++ctx->graph_seq);
    }
    // n(n-1)/2 pairs (Eq. 2), each written to both triangle entries
    std::vector<BatchTask> tasks;
    tasks.reserve((size_t)nseq * (nseq - 1) / 2);
    uint32_t max_n = 1;
    for (uint32_t i = 0; i < nseq; ++i)
        for (uint32_t j = i + 1; j < nseq; ++j) {
            BatchTask t{};
            // rows: the sequence whose 256-row stripes waste fewer padded rows
            const uint32_t SH = 256;
            const uint32_t wi = (len[i] + SH - 1) / SH * SH - len[i], wj = (len[j] + SH - 1) / SH * SH - len[j];
            const bool rows_i = (uint64_t)wi * len[j] <= (uint64_t)wj * len[i] || len[j] < kMinPeriod;
            const uint32_t r = rows_i ? i : j, c = rows_i ? j : i;
            t.a_off = off[r];
            t.m = len[r];
            t.b_off = off[c];
            t.n = len[c];
            t.out0 = i * nseq + j;
            t.out1 = j * nseq + i;
            max_n = std::max(max_n, t.n);
            tasks.push_back(t);
        }
    sort_lpt(tasks);
    const Profile pf = make_profile(sc);
    BatchArgs ba{};
    ba.pool = pool;
    for (int c = 0; c < 4; ++c) ba.prof[c] = pf.prof[c];
    ba.gap = pf.gap;
    ba.scores = dout;
    ba.err = ctx->d_err;
    ba.ntasks = (uint32_t)tasks.size();
    ba.score_cap = nseq * nseq;
    std::vector<uint32_t> lens(len, len + nseq);
    uint32_t *dlen = nullptr;
    if ((rc = upload(ctx, (pre + "_len").c_str(), lens, &dlen))) return rc;
    // the bit-sliced kernel where the scoring fits two bit planes (rows per
    // lane 32), else -- or as the autotuner finds -- the scalar batch kernel
    const bool bits = bits_scoring_ok(sc);
    BitsPlan bp;
    if (bits) {
        std::vector<BatchTask> bt = tasks;
        if ((rc = bits_prepare(ctx, pool, bt, sc, dout, nseq * nseq, pre, &bp))) return rc;
    }
    BatchTask *dt = nullptr;
    if ((rc = upload(ctx, (pre + "_tasks").c_str(), tasks, &dt))) return rc;
    ba.tasks = dt;
    auto run = [&](int r) { return r == 32 ? bits_launch(ctx, bp) : launch_batch(ctx, r, false, ba, max_n, 0, pre); };
    int R = 16;
    if ((rc = tune_rows(ctx, tasks, bits ? 32 : pick_rows(tasks), run, &R, bits))) return rc;
    auto launches = [&]() -> int {
        int r = run(R);
        if (r) return r;
        {
            LaunchTimer t(ctx, "diag");
            k_diag<<<(nseq + 255) / 256, 256, 0, ctx->stream>>>(dlen, nseq, sc.match, dout);
        }
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? NW_OK : cuda_fail(ctx, e, "all-pairs launch");
    };
    if ((rc = launches())) return rc;
    if (graph && (rc = capture_graph(ctx, gkey, pre, R == 32 ? "bits_score" : "batch_score", R == 32 ? 3 : 2,
                                     launches)))
        return rc;
    return copy_back();
}
