// Internal declarations shared by the libnw translation units.
//
// Score domain used by every kernel.  With W(i,j) = H(i,j) - gap*(i+j) the
// recurrence of Sec. 2.3 becomes
//     W(i,j) = max(W(i-1,j-1) + s'(A_i,B_j), W(i-1,j), W(i,j-1)),
//     s' = s - 2*gap,  W(i,0) = W(0,j) = 0,  H(m,n) = W(m,n) + gap*(m+n),
// because a vertical or horizontal step adds exactly gap to H and one to i+j.
// The gap term disappears from the inner loop: one cell costs a byte-permute
// (s'), one DPX add-max and one max.  W is never negative (the all-gap path
// gives W = 0) and is bounded by max(s',0)*min(i,j).  Ties keep their meaning:
// H == H(i-1,j-1)+s  <=>  W == W(i-1,j-1)+s',  H == H(i-1,j)+gap  <=>  W == W(i-1,j).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/nw.h"

namespace nw {

constexpr unsigned kFull = 0xffffffffu;

// Bounds of every spin-wait on a flag another warp or CTA raises: two seconds
// of wall time (%globaltimer, ns) or 2^24 polls, whichever comes first.
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr uint64_t kSpinNanos = 2000000000ull;

// Device error word layout: [0] = first nw_status raised, [1] = detail.
__device__ __forceinline__ void raise_error(uint32_t *err, uint32_t code, uint32_t detail) {
    if (atomicCAS(err, 0u, code) == 0u) err[1] = detail;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until *flag >= target.  Returns false (after raising NW_ERR_TIMEOUT)
// when a bound is reached or another thread already raised an error, so the
// caller can leave instead of hanging.
__device__ __forceinline__ bool wait_geq(const uint32_t *flag, uint32_t target, uint32_t *err, uint32_t where) {
    if (ld_acquire(flag) >= target) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t spins = 1;; ++spins) {
        if (ld_acquire(flag) >= target) return true;
        if ((spins & 63u) == 0) {
            if (*(volatile uint32_t *)err != 0u) return false;
            if (spins >= kSpinLimit || global_ns() - t0 > kSpinNanos) {
                raise_error(err, NW_ERR_TIMEOUT, where);
                return false;
            }
            __nanosleep(64);
        }
    }
}

// Checked build (compiled with -DNW_CHECKS): the kernels' global stores go
// through in_range(), which compares the index with the buffer's capacity;
// out of range it records NW_ERR_BOUNDS in the error word (detail: the
// store site in the top 8 bits, the low 24 bits of the index) and the store
// is skipped.  In the normal build in_range() is constant true and costs
// nothing.
#ifdef NW_CHECKS
constexpr bool kChecks = true;
#else
constexpr bool kChecks = false;
#endif
enum CheckSite : uint32_t {
    kSiteBatchPtr = 1, kSiteBatchRing, kSiteBatchScore, kSiteLocalPtr, kSiteLocalRing, kSiteLocalOut,
    kSiteLocalMoves, kSiteAffPtr, kSiteAffRing, kSiteAffScore, kSiteAffMoves, kSiteMsaRow, kSiteMsaSlot, kSiteBandBitsPtr
};
__device__ __forceinline__ bool in_range(uint64_t idx, uint64_t cap, uint32_t *err, uint32_t site) {
    if constexpr (kChecks) {
        if (idx >= cap) {
            raise_error(err, NW_ERR_BOUNDS, (site << 24) | (uint32_t)(idx & 0xffffffu));
            return false;
        }
    }
    return true;
}

// Byte permute: output byte 0 = byte (sel & 7) of {hi:lo}, etc. (PTX prmt).
__device__ __forceinline__ uint32_t prmt(uint32_t lo, uint32_t hi, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(lo), "r"(hi), "r"(sel));
    return d;
}

// Selector that reads byte `code` (0..3) of a row profile and sign-extends
// it to 32 bits: nibble 0 picks the byte, nibbles 1..3 replicate its sign.
__device__ __forceinline__ uint32_t sext_selector(uint32_t code) { return code * 0x1111u + 0x8880u; }

// Pointer words (the fill kernels write them, the traceback reads them).
// Each cell gets two bits: L = its diagonal candidate is below the maximum,
// H = its horizontal candidate is above the vertical one.  The Sec. 2.4 walk
// with priority diagonal > vertical > horizontal reads: !L -> diagonal, else
// !H -> vertical (consumes a base of A: 'I'), else horizontal ('D').  A word
// holds R rows x 16/R columns of one lane; the cell in row r, column c of the
// word has index o = c*R + r, its L bit at 31 - o and its H bit at 15 - o.
// The fill appends sign bits -- of d + s' - max(u, l) for L and of u - l for
// H -- cells in index order, one funnel shift each, into two registers, and
// joins their low halves with one byte permute.
__device__ __forceinline__ uint32_t ptr_append(uint32_t acc, int32_t diff) {
    return __funnelshift_l((uint32_t)diff, acc, 1);  // (acc << 1) | sign bit of diff
}
__device__ __forceinline__ uint32_t ptr_word(uint32_t accL, uint32_t accH) { return __byte_perm(accH, accL, 0x5410); }
// Move of cell o of a word: 0 diagonal, 1 vertical, 2 horizontal.
__device__ __forceinline__ uint32_t ptr_move(uint32_t word, uint32_t o) {
    const uint32_t L = (word >> (31u - o)) & 1u, H = (word >> (15u - o)) & 1u;
    return L ? (H ? 2u : 1u) : 0u;
}

// 2-bit code of base k of a packed sequence.
__device__ __forceinline__ uint32_t base_at(const uint8_t *s2b, uint64_t k) {
    return (s2b[k >> 2] >> ((k & 3) * 2)) & 3u;
}

// Scoring handed to kernels: prof[c] is the row profile of a query base c,
// byte d of prof[c] = s'(c, d) as int8.
struct Profile {
    uint32_t prof[4];
    int32_t gap;
};

Profile make_profile(const nw_scoring &sc);

// ------------------------------------------------------------------ context
struct KernelStat {
    uint64_t launches = 0;
    double ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<uint32_t> pending_count;  // kernels per pending pair (a graph replay holds several)
};

// A CUDA graph of a repeated call: its instantiated executable, the prefix
// of the scratch slots it owns (never shared with other calls, so its baked
// pointers stay valid), the kernel-stat name and kernel count of a replay.
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::string prefix;
    const char *label = "";
    uint32_t kernels = 0;
    uint64_t last_use = 0;
};

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
};

}  // namespace nw

struct nw_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint64_t budget = 0;
    uint64_t used = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    uint32_t *d_err = nullptr;  // 2 words
    std::map<std::string, nw::Buf> bufs;
    std::string msg;
    bool profiling = false;
    std::map<std::string, nw::KernelStat> stats;
    std::vector<cudaEvent_t> event_pool;
    // certified-band statistics: [0] pairs tried banded, [1..4] accepted in
    // round 0..3, [5] sent to the full kernel, [6] banded cells computed,
    // [7] full-grid cells of all pairs
    uint64_t band_stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // per pair of the last certified-band call: the round that certified it
    // (1..3, 0 = the full kernel), its first and its certified half-width
    std::vector<uint8_t> band_round;
    std::vector<uint32_t> band_w_first, band_w_cert;
    // learned band model (device parameters, see nw_mlp.cu)
    void *band_model = nullptr;
    // host staging for NW_HOST_IO (pinned, grown on demand)
    void *pinned = nullptr;
    size_t pinned_cap = 0;
    // autotuning: when on, the first call of a workload signature times the
    // candidate shapes and keeps the fastest (key -> packed choice)
    bool autotune = false;
    std::map<std::string, uint32_t> tuning;
    // CUDA graphs of repeated calls (NW_GRAPH), at most kMaxGraphs, LRU
    std::map<std::string, nw::GraphEntry> graphs;
    uint64_t graph_seq = 0, graph_replays = 0, graph_captures = 0;
    bool capturing = false;            // LaunchTimer records nothing while capturing
    cudaStream_t capture_stream = nullptr;
    // private stream-ordered pool of the scratch slots: freed slots stay
    // reserved in it (release threshold: never), so regrowing is cheap
    cudaMemPool_t mempool = nullptr;
    uint32_t test_hook = 0;            // NW_TEST_DROP_PROGRESS (one use)
    // ring of the bit-sliced single-pair fill: its buffer and the tag of its
    // last launch (entries carry the tag of the launch that wrote them)
    void *bits_ring = nullptr;
    uint32_t bits_epoch = 0;
};

namespace nw {

// Set ctx->msg and return code.
int fail(nw_ctx *ctx, int code, const char *fmt, ...);
int cuda_fail(nw_ctx *ctx, cudaError_t e, const char *what);

// Named scratch buffer of at least `bytes`, reused across calls; grows
// (stream-ordered) under the context budget.  Returns NW_OK or NW_ERR_OOM /
// NW_ERR_CUDA.
int scratch(nw_ctx *ctx, const char *name, size_t bytes, void **out);
// Bytes the scratch slot `name` may still grow to under the budget.
inline uint64_t scratch_headroom(nw_ctx *ctx, const char *name) {
    const auto it = ctx->bufs.find(name);
    const uint64_t mine = it == ctx->bufs.end() ? 0 : it->second.cap;
    const uint64_t others = ctx->used - mine;
    return ctx->budget > others ? ctx->budget - others : 0;
}

// Validate scoring and sizes shared by all entry points.
int check_scoring(nw_ctx *ctx, const nw_scoring &sc);

// Launch bracket for per-kernel timing.
struct LaunchTimer {
    nw_ctx *ctx;
    const char *name;
    uint32_t count;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LaunchTimer(nw_ctx *c, const char *n, uint32_t kernels = 1);
    ~LaunchTimer();
};

// Host-side section timer: with profiling on, the section's wall time (the
// host work and any waits in it) is added to the stat "host:<name>".
struct HostTimer {
    nw_ctx *ctx;
    const char *name;
    double t0;
    bool done = false;
    HostTimer(nw_ctx *c, const char *n);
    ~HostTimer() { stop(); }
    void stop();  // ends the section early (once)
};

// Autotuning keys and the graph cache (nw_runtime.cu).
constexpr size_t kMaxGraphs = 8;
bool tuned(nw_ctx *ctx, const std::string &key, uint32_t *choice);
void set_tuned(nw_ctx *ctx, const std::string &key, uint32_t choice);
std::string size_bucket(uint64_t v);  // "2^k" bucket of a size
// Runs `launches` once normally, then captures it into a graph stored under
// `key` (scratch slots named from the returned prefix); replays if present.
int graph_launch(nw_ctx *ctx, const std::string &key, const char *label, uint32_t kernels, bool *replayed);
int graph_store(nw_ctx *ctx, const std::string &key, const std::string &prefix, const char *label,
                uint32_t kernels, cudaGraph_t g);
uint64_t hash_bytes(const void *p, size_t n, uint64_t h);
void free_prefix(nw_ctx *ctx, const std::string &prefix);

// Capture `launches` (a callable returning a status; it must only enqueue
// work: its scratch slots already exist from an uncaptured run) into a graph
// stored under `key`.  The capture runs on a private stream (the caller's
// may be the legacy default stream, which cannot be captured); LaunchTimer
// records nothing meanwhile.
template <typename F>
int capture_graph(nw_ctx *ctx, const std::string &key, const std::string &prefix, const char *label,
                  uint32_t kernels, F launches) {
    if (!ctx->capture_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "capture stream");
    }
    cudaStream_t saved = ctx->stream;
    ctx->stream = ctx->capture_stream;
    ctx->capturing = true;
    cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? launches() : NW_OK;
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->capture_stream, &g) : e;
    ctx->stream = saved;
    ctx->capturing = false;
    if (rc || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : cuda_fail(ctx, e2, "graph capture");
    }
    return graph_store(ctx, key, prefix, label, kernels, g);
}

// Copy helpers for NW_HOST_IO.
int to_device(nw_ctx *ctx, const void *host, size_t bytes, const char *slot, void **dev);
// Pinned host staging of at least `bytes` owned by the context (grown on
// demand, kept until nw_ctx_destroy); one user at a time per context.
int pinned_host(nw_ctx *ctx, size_t bytes, void **out);

}  // namespace nw

// Entry points implemented in the other translation units (C++ linkage).
namespace nw {
// Pointer-tile geometry shared by the fill kernels and the traceback: the
// walk stages 8 lanes x 32 words of one stripe at a time, so every lane row
// of pointer words is padded to a multiple of 32 words.
constexpr uint32_t kTileLanes = 8, kTileWords = 32;
inline uint32_t ptr_words_per_lane_row(uint32_t n, int R) {
    const uint32_t cpw = 16u / (uint32_t)R;
    return (((n + cpw - 1) / cpw + kTileWords - 1) / kTileWords) * kTileWords;
}

// One pair of a batched launch (nw_batch_kernel.cuh, nw_bits.cu).
struct BatchTask {
    uint64_t a_off, b_off;  // byte offsets in the pool
    uint32_t m, n;          // rows (A) and columns (B)
    uint32_t out0, out1;    // score destinations (out1 == ~0u: none)
    uint64_t ptr_off;       // word offset of the pair's pointer words
    uint32_t ncg;           // pointer words per lane row
    uint32_t period;        // steps per stripe (banded: fixed band width)
    int32_t lo, hi;         // banded: diagonals j - i kept, [lo, hi]
};

// One traceback + CIGAR job (see nw_trace.cu).
struct TraceTask {
    const uint32_t *ptr;   // pointer words of the pair
    uint32_t ncg;          // words per lane row
    uint32_t m, n;
    uint8_t *moves;        // scratch, m+n bytes (reversed move codes)
    uint64_t *nmoves;      // scratch, 1 word
    const uint8_t *a, *b;  // packed sequences
    char *cigar;           // output
    uint64_t *cigar_len;   // output
    int32_t band_lo;       // banded layout: stripe s keeps columns from max(0, s*32R + band_lo);
                           // kNoBand for the full layout
    uint32_t s_lo;         // first stripe whose words `ptr` holds (0: all of them)
    uint32_t *state;       // null: walk from (m, n) to the end; else a walk resumed and
                           // paused in device memory: {i, j, k lo, k hi, done}
    const uint32_t *origin;  // null: the moves start at (0, 0); else at (origin[0], origin[1])
                             // (a local alignment's start cell, read by the CIGAR assembly)
};
constexpr int32_t kNoBand = INT32_MIN;
// Traceback + CIGAR for `ntasks` tasks: `host` describes them on the host
// (always), `dev` is the same array in device memory (null: one task,
// passed by value).  Pairs of kParMinStripes stripes or more walk their
// stripes in parallel (see nw_trace.cu).
int launch_trace(nw_ctx *ctx, int R, const TraceTask *host, const TraceTask *dev, uint32_t ntasks, uint32_t mflag);
// The same on the bit-sliced single-pair records (ptr: (L, Hb) word pairs,
// [warp][step pair][lane] with ncg step pairs per warp; stripes of 31 rows
// from the top, see nw_bits_pair.cu).
int launch_trace_bits(nw_ctx *ctx, const TraceTask *host, const TraceTask *dev, uint32_t ntasks, uint32_t mflag);
// The two halves of launch_trace: the walk (resumable through `state`) and
// the CIGAR assembly from the finished move list.
int launch_traceback(nw_ctx *ctx, int R, const TraceTask &one, const TraceTask *many, uint32_t ntasks);
int launch_finish(nw_ctx *ctx, const TraceTask &one, const TraceTask *many, uint32_t ntasks, uint32_t mflag);
int align_single(nw_ctx *ctx, const uint8_t *a2b, uint64_t m, const uint8_t *b2b, uint64_t n,
                 const nw_scoring &sc, uint32_t flags, int32_t *score, char *cigar, uint64_t cigar_cap,
                 uint64_t *cigar_len);
cudaError_t fill_score_with_scratch(const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n,
                                    const nw_scoring &sc, int32_t *score, uint32_t *bnd, uint32_t *progress,
                                    uint32_t *err, cudaStream_t stream, int sm_count);
// Single-pair fill (nw_pair.cu).  Stripes of 32*R rows, `nw` of them per
// CTA ("group"); the bottom W row of every group but the last is kept in
// `bnd` (the checkpoints of the recompute traceback).
struct PairFill {
    int R = 4, C = 4, nw = 4;      // rows per lane, columns per step, warps per CTA
    const uint32_t *sel = nullptr; // column selector table (null: built here)
    bool ptr = false;              // write 2-bit pointers
    uint32_t *ptr_words = nullptr; // pointer words of stripes [cs_lo*nw, ...)
    uint32_t ncg = 0;              // pointer words per lane row
    int32_t *score = nullptr;      // null: no score
    uint32_t *bnd = nullptr;       // group rows (null: scratch)
    uint32_t *progress = nullptr;  // per-group progress words (null: scratch; zeroed unless recompute)
    uint32_t cs_lo = 0, cs_hi = 0xffffffffu;  // groups to run
    const uint32_t *ncols = nullptr;          // device word: columns needed (null: all)
    bool recompute = false;        // groups start from kept checkpoints, write none
    bool keep_rows = false;        // every group's bottom row goes to `bnd` (the checkpoints)
};
uint32_t pair_bstride(uint32_t n);
int launch_pair_fill(nw_ctx *ctx, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n, const Profile &pf,
                     const PairFill &f);
void free_band_model(nw_ctx *ctx);
}
