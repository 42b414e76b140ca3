/*
 * nw.h -- C ABI of libnw, a GB300 (sm_103a) Needleman-Wunsch library.
 *
 * What it computes (the paper's Sec. 2): global alignment of two DNA
 * sequences with a linear gap penalty.  The score grid has (m+1) x (n+1)
 * cells (Sec. 2.1, row 0 / column 0 are the empty label cells), starts from
 * H(0,0)=0, H(i,0)=i*gap, H(0,j)=j*gap (Sec. 2.2) and is filled with
 *     H(i,j) = max(H(i-1,j-1) + s(A_i,B_j), H(i-1,j) + gap, H(i,j-1) + gap)
 * (Sec. 2.3, Eq. 1 read as standard NW; s = match or mismatch).  The
 * alignment is the backtrack of Sec. 2.4 from (m,n) with the single path
 * chosen by the priority diagonal > vertical > horizontal (the order of the
 * direction codes 1/2/3 of Sec. 3.1).
 *
 * Conventions used by every entry point
 *   - A is the query (rows, length m), B the reference (columns, length n).
 *   - Sequences are 2-bit packed: A=0, C=1, G=2, T=3; base k sits at bits
 *     2*(k%4) .. 2*(k%4)+1 of byte k/4 (least significant first); a sequence
 *     of L bases takes ceil(L/4) bytes; unused high bits of the last byte are
 *     ignored.
 *   - CIGAR ops: '=' match, 'X' mismatch, 'I' base of A alone (vertical move),
 *     'D' base of B alone (horizontal move); run-length encoded ("12=1X3I"),
 *     NUL-terminated.  NW_CIGAR_M merges '='/'X' into 'M'.  A CIGAR never
 *     needs more than nw_cigar_bound(m, n) bytes including the NUL.
 *   - Zero-length sequences are valid.  m and n must be below 2^30.
 *   - Scoring: gap <= 0, mismatch <= match, every value in [-40, 40]; the
 *     product max(match - 2*gap, 0) * min(m,n) must stay below 2^29.  The
 *     certified band (NW_LEARNED_BAND, nw_align_batch_banded, a server made
 *     with NW_LEARNED_BAND) also needs match >= 2*gap: its exit bound
 *     assumes that a path with fewer gap moves scores higher (NW_ERR_ARG
 *     otherwise).
 *   - Memory: without NW_HOST_IO every sequence/output pointer is a device
 *     pointer on the context's device and the call is asynchronous on the
 *     context's stream (stream-ordered; call nw_ctx_sync to wait and collect
 *     device-side errors).  With NW_HOST_IO they are host pointers: the call
 *     copies inputs in, runs, copies results out and waits.  Per-pair and
 *     per-sequence metadata arrays (offsets, lengths, CIGAR offsets) are
 *     always host arrays.
 *   - Ownership: the caller owns every buffer it passes; the library never
 *     frees or retains them after the call returns (device-side work may
 *     still read them until the stream reaches that point).  Scratch memory
 *     comes from the context's pool, capped by its budget (NW_ERR_OOM beyond).
 *   - Errors: every call returns an nw_status; nw_strerror gives a short
 *     text and nw_ctx_last_message the detail of the last failure on that
 *     context.  Calls on one context must not be made from two host threads
 *     at once.
 */
#ifndef NW_H_
#define NW_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NW_OK = 0,
    NW_ERR_ARG = 1,           /* bad argument (size, scoring, null pointer)  */
    NW_ERR_BAD_BASE = 2,      /* a character outside ACGT/acgt               */
    NW_ERR_OOM = 3,           /* scratch would exceed the context budget     */
    NW_ERR_CIGAR_TRUNC = 4,   /* CIGAR capacity too small; length reported   */
    NW_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up          */
    NW_ERR_CUDA = 6,          /* a CUDA runtime call failed                   */
    NW_ERR_UNSUPPORTED = 7,   /* valid request this build cannot serve        */
    NW_ERR_BOUNDS = 8         /* checked build (NW_CHECKS): a kernel index fell
                                 outside its buffer; the store was skipped    */
} nw_status;

/* Flags (bitwise OR). */
#define NW_SCORE_ONLY   0u
#define NW_CIGAR        1u    /* also produce the alignment                  */
#define NW_LEARNED_BAND 2u    /* batch: certified learned band first          */
#define NW_HOST_IO      4u    /* sequence inputs and outputs are host memory  */
#define NW_CIGAR_M      8u    /* write 'M' for both '=' and 'X'               */
#define NW_BAND_RAW     16u   /* nw_align_batch_banded: one banded round, the
                                 banded score itself, no certificate or
                                 fallback (score only; for inspection)      */
#define NW_GRAPH        64u   /* nw_score_all_pairs / score-only nw_align_batch
                                 on device buffers (nw_score_all_pairs also
                                 with NW_HOST_IO: the pool is copied to the
                                 context's device slot first): capture the
                                 launches into a CUDA graph kept on the
                                 context, keyed by every pointer, size and host
                                 metadata of the call; a repeated call replays
                                 it (see below)                             */
#define NW_RECOMPUTE    32u   /* nw_align with NW_CIGAR: take the stripe-
                                 checkpoint recompute path even when the
                                 pointer matrix fits (see nw_align)         */

typedef struct {
    int32_t match;      /* score of a diagonal step with equal bases (Sec. 2.3: +1)   */
    int32_t mismatch;   /* score of a diagonal step with unequal bases (Sec. 2.3: -1) */
    int32_t gap;        /* score of a vertical or horizontal step (Sec. 2.3: -1)      */
} nw_scoring;

/* Affine gap scores (not in the paper): a run of k gap moves of one kind
 * scores gap_open + k * gap_extend. */
typedef struct {
    int32_t match;
    int32_t mismatch;
    int32_t gap_open;     /* <= 0 */
    int32_t gap_extend;   /* <= 0 */
} nw_affine_scoring;

typedef struct nw_ctx nw_ctx;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` that launches on `stream` (a
 * cudaStream_t; NULL = the legacy default stream) and keeps at most
 * `mem_budget` bytes of scratch (0 = 90% of the device's free memory).
 * Returns NULL on failure.  Not in the paper: the host-side state the
 * library needs around its kernels. */
nw_ctx *nw_ctx_create(int device, void *stream, uint64_t mem_budget);
void nw_ctx_destroy(nw_ctx *ctx);
/* Change the stream later calls launch on. */
int nw_ctx_set_stream(nw_ctx *ctx, void *stream);
/* Wait for the context's stream and return the first device-side error
 * raised since the previous sync (NW_ERR_TIMEOUT, NW_ERR_BAD_BASE), else the
 * CUDA status mapped to NW_ERR_CUDA, else NW_OK.  Clears the device error. */
int nw_ctx_sync(nw_ctx *ctx);
/* Detail of the last failure on this context ("" if none).  Owned by ctx. */
const char *nw_ctx_last_message(const nw_ctx *ctx);
const char *nw_strerror(int status);

/* Per-kernel timing: when on, every launch is bracketed by CUDA events on
 * the context's stream; nw_ctx_kernel_stats reports, per kernel name, the
 * launch count and the summed device time in ms (summed after a sync). It
 * returns how many kernel names exist (fills at most `cap` of them). */
int nw_ctx_set_profiling(nw_ctx *ctx, int on);
int nw_ctx_kernel_stats(nw_ctx *ctx, const char **names, uint64_t *launches, double *total_ms, int cap);
int nw_ctx_reset_stats(nw_ctx *ctx);

/* ---------------------------------------------------- autotuning, graphs */

/* Autotuning (off by default; not in the paper).  When on, the first call
 * of a workload signature -- a batch's mean lengths and pair count, or a
 * single pair's lengths, each bucketed by powers of two -- runs the fill with
 * every candidate shape (rows per lane of the batched kernel: 4, 8, 16; rows
 * x columns x warps of the single-pair kernel), times each with CUDA events
 * and keeps the fastest for later calls of that signature.  The timed runs
 * compute the real result, so the first call only costs more time. */
int nw_ctx_set_autotune(nw_ctx *ctx, int on);
/* The tuning table as text, one "key value" line per entry: written into
 * buf[0..cap) NUL-terminated (truncated if short); returns the full length
 * without the NUL, or -NW_ERR_ARG.  Values: rows per lane for batch_rows
 * keys, R*100 + C*10 + warps for pair_shape keys. */
int64_t nw_ctx_tuning(nw_ctx *ctx, char *buf, uint64_t cap);
/* Adds or replaces entries from text in the same format (e.g. a table
 * saved by an earlier process).  NW_ERR_ARG on a malformed line (nothing
 * is changed then).  A value that is not a valid shape makes the calls of
 * that signature fail with NW_ERR_ARG. */
int nw_ctx_set_tuning(nw_ctx *ctx, const char *text);
/* Failure-path test hook (not in the paper).  NW_TEST_DROP_PROGRESS makes
 * the next single-pair fill on this context run with row-group progress
 * counters that nothing releases: every wait on them gives up after its
 * time limit (2 s), the kernel returns, and the call reports NW_ERR_TIMEOUT;
 * the context stays usable.  The hook clears itself after one use.  It
 * exists so that tests can exercise the bounded waits without a GPU fault. */
#define NW_TEST_DROP_PROGRESS 1u
int nw_ctx_set_test_hook(nw_ctx *ctx, uint32_t hook);

/* NW_GRAPH cache: out[0] graphs held (at most 8, least recently used
 * evicted with the scratch they own), out[1] captures, out[2] replays.
 * Returns 3.  A replay re-reads the sequence pool and writes the same output
 * buffer as the captured call; it is valid as long as those buffers (and the
 * host metadata, which is part of the key) are the caller's current ones. */
int nw_ctx_graph_stats(nw_ctx *ctx, uint64_t *out, int cap);

/* ---------------------------------------------------------------- packing */

/* Host: pack `len` ASCII bases (ACGT, either case) into 2-bit codes.
 * out2b must hold ceil(len/4) bytes.  NW_ERR_BAD_BASE on any other
 * character (out2b is then unspecified).  The paper stores one char per
 * base (Sec. 3.1 listing); this is the 2-bit layout described above. */
int nw_pack(const char *ascii, uint64_t len, uint8_t *out2b);

/* Host: the same layout from base codes (one byte per base, 0..3 = A, C,
 * G, T) instead of ASCII; NW_ERR_BAD_BASE on a code above 3. */
int nw_pack_codes(const uint8_t *codes, uint64_t len, uint8_t *out2b);
/* Host: pack `count` code sequences into one pool: sequence k is
 * codes[code_off[k] .. code_off[k]+len[k]) and goes to pool + pool_off[k]
 * (ceil(len[k]/4) bytes; the caller lays out pool_off, e.g. 16-byte
 * aligned).  Stops at the first bad code (NW_ERR_BAD_BASE). */
int nw_pack_pool(const uint8_t *codes, const uint64_t *code_off, const uint32_t *len, uint32_t count, uint8_t *pool,
                 const uint64_t *pool_off);

/* Device: the same packing by a GPU kernel (device pointers, asynchronous).
 * A bad character is reported by the next nw_ctx_sync as NW_ERR_BAD_BASE. */
int nw_pack_device(nw_ctx *ctx, const char *ascii, uint64_t len, uint8_t *out2b);

/* Worst-case CIGAR size in bytes, NUL included: 2*(m+n)+1. */
uint64_t nw_cigar_bound(uint64_t m, uint64_t n);

/* The certificate of the banded rounds (no GPU needed): an upper bound on
 * the score of any path of an m x n grid that leaves the band of half-width
 * w around the diagonals [min(0,n-m), max(0,n-m)].  Such a path reaches
 * diagonal max(0,n-m)+w+1 or min(0,n-m)-w-1, so it has at least G gap moves
 * (the fewer of the two sides' minimum counts that fit the grid), hence at
 * most k = floor((m+n-G)/2) diagonal moves worth at most `match` each:
 * *bound = match*k + gap*(m+n-2k), the larger over the two sides.  Returns 1
 * with *bound set, 0 when no path can leave the band (*bound = 0), or
 * -NW_ERR_ARG (sizes >= 2^31, gap > 0, match < 0, null bound).  A banded
 * score above the bound equals the full score, and its alignment is the
 * full alignment. */
int nw_band_exit_bound(uint64_t m, uint64_t n, uint64_t w, nw_scoring sc, int64_t *bound);
/* The certificate the banded rounds apply (no GPU needed): 1 when a banded
 * score of half-width w proves the full result -- the score when
 * banded_score >= the exit bound, the alignment (want_cigar != 0) only when
 * banded_score > the bound, always when no path can leave the band -- else
 * 0; -NW_ERR_ARG as nw_band_exit_bound. */
int nw_band_certifies(uint64_t m, uint64_t n, uint64_t w, int32_t banded_score, nw_scoring sc, uint32_t want_cigar);
/* The half-width the next banded round uses after banded_score failed at w:
 * the larger of 2w and the smallest w' > w at which banded_score itself
 * would certify (a wider band scores no less, so the round at w' certifies);
 * at most max(2w, max(m,n)+1).  -NW_ERR_ARG for sizes >= 2^31, w >= 2^30, gap
 * > 0 or match < 0. */
int64_t nw_band_next_width(uint64_t m, uint64_t n, uint64_t w, int32_t banded_score, nw_scoring sc,
                           uint32_t want_cigar);

/* -------------------------------------------------------------- alignment */

/* One pair (Sec. 2.2-2.4).  Writes the score H(m,n) to *score; with
 * NW_CIGAR also the CIGAR (NUL-terminated) into cigar[0..cigar_cap) and its
 * length without the NUL into *cigar_len.  With device outputs cigar_cap
 * must be at least nw_cigar_bound(m,n); with NW_HOST_IO a smaller buffer
 * returns NW_ERR_CIGAR_TRUNC with the needed length in *cigar_len.
 *
 * Memory.  The CIGAR normally comes from a full matrix of 2-bit pointers,
 * about m*n/4 bytes of scratch.  When that does not fit the context budget
 * (or with NW_RECOMPUTE) the call switches to stripe-checkpoint recompute:
 * a score-only fill keeps one W row per 32*R*4 rows (R = 8 rows per lane
 * from m >= 2048, else 4; about 4*(n+128) bytes per kept row), then the
 * pointers are filled again wave by wave from the bottom, each wave as many
 * row groups as the remaining budget holds, and the traceback walks each
 * wave before the next is computed.  Same result, at most twice the fill
 * work; NW_ERR_OOM only if one group of 32*R*4 rows of pointers does not
 * fit.  Sec. 2 keeps the whole matrix; this path is not in the paper. */
int nw_align(nw_ctx *ctx, const uint8_t *a2b, uint64_t m, const uint8_t *b2b, uint64_t n,
             nw_scoring sc, uint32_t flags, int32_t *score,
             char *cigar, uint64_t cigar_cap, uint64_t *cigar_len);

/* Score of one pair without allocating anything.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory
 * when they align -- a server that reserved all device memory for its own
 * pool up front, a plug-in inside a runtime that owns the allocator, or a
 * latency-critical path where cudaMalloc/cudaFree would synchronize the
 * device.  No context is needed: the fill's scratch lives in a 12 MiB
 * static device array that every GPU loading the library reserves until
 * the process exits.  a2b, b2b and score are device pointers on the current
 * device; the kernel runs on `stream` (a cudaStream_t, NULL = legacy
 * default) and the call waits for that stream (cudaStreamSynchronize)
 * before returning, so a device-side timeout comes back as NW_ERR_TIMEOUT;
 * because it waits for its stream, it may not be called while that stream
 * (or the legacy default stream) is being captured into a CUDA graph.  The
 * first call on each device looks up the array's device address with that
 * device current and keeps it for later calls; a cudaDeviceReset while the
 * library is loaded is not supported, since the kept address would be
 * stale.
 * Sizes: ceil(m/512) <= 4096 and (ceil(m/512)-1) * 32*ceil((n+1)/32) <=
 * 3,141,568 words (for example m = n = 32,768 fits); larger inputs return
 * NW_ERR_ARG.  Calls share the array, so calls that overlap on the GPU
 * (two host threads, or two streams) race; serialize them.  Same scoring
 * and length rules as nw_align; score only. */
int nw_align_score_noalloc(const uint8_t *a2b, uint64_t m, const uint8_t *b2b, uint64_t n, nw_scoring sc,
                           int32_t *score, void *stream);

/* Many independent pairs in one call (the paper's Sec. 3.2 pairwise stage,
 * batched on one device instead of split over MPI ranks).  Pair k aligns the
 * sequence at byte offset a_off[k] of `pool2b` (a_len[k] bases) against the
 * one at b_off[k] (b_len[k] bases).  scores[k] receives the score.  With
 * NW_CIGAR, pair k's CIGAR goes to cigar_pool + cigar_off[k] with capacity
 * cigar_off[k+1] - cigar_off[k] (which must be >= nw_cigar_bound of the pair)
 * and its length to cigar_len[k].  a_off, a_len, b_off, b_len and cigar_off
 * (npairs+1 entries) are host arrays; pool2b, scores, cigar_pool, cigar_len
 * are device memory unless NW_HOST_IO.  With NW_LEARNED_BAND each pair is
 * first run in a band whose half-width a trained model predicts (see
 * nw_band_model_load); a banded result is kept only when a certificate
 * proves it equals the full alignment, else the band is widened and finally
 * the full grid is used -- results are exact either way. */
int nw_align_batch(nw_ctx *ctx, const uint8_t *pool2b,
                   const uint64_t *a_off, const uint32_t *a_len,
                   const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs,
                   nw_scoring sc, uint32_t flags, int32_t *scores,
                   char *cigar_pool, const uint64_t *cigar_off, uint64_t *cigar_len);

/* Local alignment of many pairs (Smith-Waterman; not in the paper, which
 * aligns globally): the grid of Sec. 2.3 with a floor of 0,
 *     H(i,0) = H(0,j) = 0,
 *     H(i,j) = max(0, H(i-1,j-1) + s(A_i,B_j), H(i-1,j) + gap, H(i,j-1) + gap),
 * so the best alignment of any substring of A with any substring of B.
 * scores[k] = the largest H(i,j) of pair k.  The alignment ends at the
 * first cell in row-major order (smallest i, then smallest j) holding that
 * value and is walked back with the priority diagonal > vertical >
 * horizontal of nw_align until the first cell whose H is 0, its start; a
 * score of 0 is the empty alignment at (0,0).  ends (4 entries per pair,
 * may be NULL without NW_CIGAR): i_start, j_start, i_end, j_end -- the
 * alignment covers A[i_start .. i_end) and B[j_start .. j_end), 0-based;
 * without NW_CIGAR the start is not computed and reads 0xFFFFFFFF.  With
 * NW_CIGAR (ends then required) pair k's CIGAR of the aligned part goes to
 * cigar_pool + cigar_off[k] as in nw_align_batch (capacity at least
 * nw_cigar_bound).  Pool, scores, ends and CIGAR buffers are device memory
 * unless NW_HOST_IO; metadata arrays are host arrays.  Scoring as nw_align,
 * with max(match, 0) * min(m, n) below 2^29; a pair whose one-warp sweep
 * would exceed 2^31 stripe steps (about m*n/256 >= 2^31) is
 * NW_ERR_UNSUPPORTED. */
int nw_local_align_batch(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                         const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, nw_scoring sc,
                         uint32_t flags, int32_t *scores, uint32_t *ends, char *cigar_pool,
                         const uint64_t *cigar_off, uint64_t *cigar_len);

/* Global alignment of many pairs with affine gaps (Gotoh; not in the paper,
 * whose gap penalty is linear, though the center-star method it cites uses
 * affine gaps).  A run of k gap moves of one kind scores go + k*ge:
 *     E(i,j) = max(E(i,j-1) + ge, H(i,j-1) + go + ge)     (ends with 'D')
 *     F(i,j) = max(F(i-1,j) + ge, H(i-1,j) + go + ge)     (ends with 'I')
 *     H(i,j) = max(H(i-1,j-1) + s(A_i,B_j), E(i,j), F(i,j))
 * from H(0,0) = 0, H(0,j) = go + j*ge, H(i,0) = go + i*ge.  scores[k] =
 * H(m,n).  With NW_CIGAR the alignment is walked back from (m,n): in state
 * H the diagonal when it gives H, else the vertical gap when F gives H,
 * else the horizontal gap; in a gap the walk extends only when extending is
 * strictly better than opening (a tie closes the gap); on row 0 / column 0
 * only horizontal / vertical moves remain.  With gap_open = 0 the result
 * equals nw_align_batch with gap = gap_extend, move for move.  Memory and
 * arguments as nw_align_batch (NW_HOST_IO, NW_CIGAR, NW_CIGAR_M; pointer
 * words take 0.5 byte per cell).  Scores in [-40, 40], both gap scores <=
 * 0, mismatch <= match, max(match - 2*gap_extend, 0) * min(m,n) below 2^29;
 * a pair whose one-warp sweep would exceed 2^31 stripe steps is
 * NW_ERR_UNSUPPORTED. */
int nw_affine_align_batch(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                          const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, nw_affine_scoring sc,
                          uint32_t flags, int32_t *scores, char *cigar_pool, const uint64_t *cigar_off,
                          uint64_t *cigar_len);

/* Partition of a pair list over `nranks` ranks (no GPU needed): the
 * paper's Sec. 3.2 divides the alignments over MPI ranks and gathers the
 * results; here each rank of a multi-GPU job aligns its share with
 * nw_align_batch and the results are gathered.  Longest processing time
 * first: pairs sorted by cells a_len*b_len, largest first (index order
 * among equals), each given to the rank with the fewest cells so far (the
 * lowest rank on ties); so the largest load is at most the mean load plus
 * the largest pair.  rank_of[k] receives pair k's rank; load (optional,
 * nranks entries) each rank's cells.  NW_ERR_ARG for nranks = 0 or null
 * arrays. */
int nw_shard_pairs(const uint32_t *a_len, const uint32_t *b_len, uint32_t npairs, uint32_t nranks, uint32_t *rank_of,
                   uint64_t *load);

/* The certified band with explicit starting half-widths (host array
 * band_w, one per pair): each pair is first aligned in the band of diagonals
 * d = j - i in [min(0,n-m) - w, max(0,n-m) + w].  The banded score S_b is
 * kept only when a certificate proves it is the full-grid score: every path
 * that leaves the band makes at least G gap moves (G from the band
 * geometry), so it scores at most U0 = match*floor((m+n-G)/2) + gap*(m+n-2*
 * floor((m+n-G)/2)); S_b >= U0 certifies the score and S_b > U0 also the
 * alignment (no out-of-band path can tie).  Rejected pairs retry at 2w and
 * 4w, then go to the full kernel, so results always equal nw_align_batch.
 * Needs match >= 0.  Arguments otherwise as nw_align_batch.  Not in the
 * paper. */
int nw_align_batch_banded(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                          const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, const uint32_t *band_w,
                          nw_scoring sc, uint32_t flags, int32_t *scores, char *cigar_pool, const uint64_t *cigar_off,
                          uint64_t *cigar_len);
/* Counters of the certified band since the context was created: [0] pairs
 * tried in a band, [1..3] certified in round 1..3, [4] unused, [5] sent to
 * the full kernel, [6] cells the banded kernels computed, [7] full-grid
 * cells of every pair handed to the banded path.  Returns 8 (fills at most
 * `cap`). */
int nw_ctx_band_stats(nw_ctx *ctx, uint64_t *out, int cap);

/* Per-pair outcome of the last certified-band call on this context
 * (nw_align_batch with NW_LEARNED_BAND, or nw_align_batch_banded), for
 * inspection: round[k] = the banded round (1..3) whose certificate accepted
 * pair k, or 0 when it went to the full kernel; first_width[k] = the
 * half-width of its first round; cert_width[k] = the half-width that
 * certified it (0 for the full kernel).  Any output may be NULL; at most
 * `cap` entries are written.  Returns the number of pairs of that call
 * (0 before any), or -NW_ERR_ARG.  Not in the paper. */
int64_t nw_ctx_band_outcome(nw_ctx *ctx, uint8_t *round, uint32_t *first_width, uint32_t *cert_width,
                            uint64_t cap);

/* ------------------------------------------------------------ learned band
 * Not in the paper.  A pair's features (65 floats): a 64-bin histogram of
 * exact 4-mer hits around the pair's expected diagonal (256 anchors in A,
 * hits within +-max(m,n)/8 of the anchor's expected column, bins over that
 * window, log1p(count)/log1p(anchors)) and (n-m)/max(m,n).  The model is a
 * 65-128-128-1 ReLU network with BF16 weights and activations and FP32
 * accumulation whose output is log of the band half-width; with
 * NW_LEARNED_BAND, nw_align_batch runs the certified band from
 * ceil(0.75 * exp(output)) (at least 8), or from 64 without a model; a pair
 * whose round fails the certificate is banded again at the smallest width
 * whose exit bound lies below the failed banded score (which then
 * certifies: a wider band scores no less), at least twice the last one. */

/* Features of npairs pairs into feat (device, npairs x 65 floats, row per
 * pair); pool2b device, metadata host arrays; B <= 200,000 bases. */
int nw_band_features(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                     const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, float *feat);
/* Number of model parameters (FP32 masters, flat: W1[128][65], b1[128],
 * W2[128][128], b2[128], W3[128], b3). */
uint64_t nw_band_model_size(void);
/* Fresh parameters (uniform He initialisation from a counter-based
 * SplitMix64 stream keyed by seed), Adam state cleared. */
int nw_band_model_init(nw_ctx *ctx, uint64_t seed);
/* Copy parameters in / out (host arrays of nw_band_model_size() floats). */
int nw_band_model_set(nw_ctx *ctx, const float *params, uint64_t count);
int nw_band_model_get(nw_ctx *ctx, float *params, uint64_t count);
/* Save the parameters to a file / load them from one (then as
 * nw_band_model_set: optimizer state cleared).  Format: "NWBAND01", the
 * parameter count (little-endian uint64), the FP32 parameters.  A file of
 * another format or size is NW_ERR_ARG. */
int nw_band_model_save(nw_ctx *ctx, const char *path);
int nw_band_model_load(nw_ctx *ctx, const char *path);
/* The straggler rule of the batched paths (no GPU needed): given each
 * pair's cost on one warp (warp_cells: cells, scaled for slower kernels) and
 * its full grid (full_cells), the pairs to run on the multi-warp single-pair
 * kernel instead.  With the pairs sorted by one-warp cost, routing the
 * first k costs the sum of their single-pair times plus the larger of the
 * rest's batch time and the (k+1)-th pair's one-warp time; the k with the
 * lowest estimate is taken (pairs under 1e7 full cells are never routed).
 * Here a single-pair time is full_cells / 2e11 s + 1 ms (the scalar
 * single-pair kernel); inside the batched paths, pairs whose scoring the
 * bit-sliced single-pair kernel takes are costed by its chain instead,
 * (m + n + m/31) x 40 ns + 0.3 ms.
 * Writes the indices, costliest first, to out (n entries of room) and
 * returns how many, or -NW_ERR_ARG. */
int64_t nw_route_stragglers(const double *warp_cells, const double *full_cells, uint32_t n, uint32_t *out);
/* The first banded round's half-width for a pair whose network output is y
 * (= log of the predicted half-width): ceil(0.75 * e^y), clamped to
 * [8, max(m, n)]; no GPU needed.  0 for sizes >= 2^31. */
uint32_t nw_band_start_width(float y, uint64_t m, uint64_t n);
/* Drop the context's model and its optimizer state (NW_LEARNED_BAND then
 * starts every pair at half-width 64, as on a context that never had one). */
int nw_band_model_clear(nw_ctx *ctx);
/* Network outputs for n feature rows (device in, device out). */
int nw_band_model_forward(nw_ctx *ctx, const float *feat, uint32_t n, float *out);
/* Gradient of 0.5*mean((y - target)^2) w.r.t. the parameters (device
 * arrays: grad has nw_band_model_size() floats, loss one float). */
int nw_band_model_grad(nw_ctx *ctx, const float *feat, const float *target, uint32_t n, float *grad, float *loss);
/* One Adam step (lr; beta 0.9/0.999, eps 1e-8) on that loss. */
int nw_band_model_train_step(nw_ctx *ctx, const float *feat, const float *target, uint32_t n, float lr, float *loss);

/* All-vs-all scores of `nseq` sequences (the scoring-matrix stage of the
 * paper's center-star alignment, Sec. 3.2; Eq. 2 gives its n(n-1)/2 pairs).
 * Sequence k starts at byte offset off[k] of pool2b and has len[k] bases
 * (host arrays).  out receives the full nseq x nseq int32 matrix,
 * row-major: out[i*nseq+j] = score(seq i as A, seq j as B), symmetric, with
 * out[i*nseq+i] = len[i]*match. */
int nw_score_all_pairs(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *off, const uint32_t *len,
                       uint32_t nseq, nw_scoring sc, uint32_t flags, int32_t *out);

/* Center-star multiple alignment of `nseq` sequences (the paper's Sec.
 * 3.2): the scoring matrix of all n(n-1)/2 pairs (Eq. 2, as
 * nw_score_all_pairs), the center = the sequence most similar to the rest
 * (the largest sum of its scores against the other sequences; the diagonal
 * is left out; the lowest index on ties), every sequence k aligned as the
 * query against the center as the reference (as nw_align_batch with
 * NW_CIGAR), then the pairwise alignments merged with the aligned center as
 * the reference.  In the merge, G[p] = the most 'I' ops any alignment
 * places before center base p (p = 0..len[center]; the last slot follows
 * the last base); center base p lands in column p + G[0] + ... + G[p]; the
 * I-bases of a row fill their slot from the left; 'D' leaves '-'.
 * Inputs: pool2b, off, len as nw_score_all_pairs.  Outputs: *center (host);
 * row_sums (nseq int64, may be NULL); scores (nseq int32: sequence k against
 * the center); the CIGARs at cigar_pool + cigar_off[k] (cigar_off has
 * nseq+1 entries, each capacity >= nw_cigar_bound(len[k], len[center]) --
 * 2*(len[k] + max len) + 1 always suffices) with lengths cigar_len[k]; the
 * merged rows (bytes 'A','C','G','T','-') at msa + k*msa_ld, NUL-terminated
 * when msa_ld exceeds the column count, written to *msa_cols (host).  msa
 * may be NULL (only the column count is returned; nw_msa_merge writes the
 * rows later from the CIGARs); msa_ld below the column count returns
 * NW_ERR_CIGAR_TRUNC with every other output written.  Buffers are device
 * memory on the context's device unless NW_HOST_IO; NW_GRAPH applies to the
 * scoring stage (with NW_HOST_IO too: it runs on the copied pool);
 * NW_CIGAR_M is passed to the alignments.  Synchronises the
 * context's stream (the center and the column count come to the host).
 * 1..65535 sequences. */
int nw_center_star(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *off, const uint32_t *len, uint32_t nseq,
                   nw_scoring sc, uint32_t flags, uint32_t *center, int64_t *row_sums, int32_t *scores,
                   char *cigar_pool, const uint64_t *cigar_off, uint64_t *cigar_len, char *msa, uint64_t msa_ld,
                   uint64_t *msa_cols);
/* The merge step of nw_center_star alone, from given alignments of every
 * sequence k (query) against sequence `center` (reference): CIGAR k at
 * cigar_pool + cigar_off[k] (nseq entries, host array), cigar_len[k] bytes.
 * Each CIGAR must consume exactly len[k] bases of sequence k and
 * len[center] of the center (NW_ERR_ARG from the next sync otherwise, and
 * no row is written).  Writes *msa_cols and, unless msa is NULL, the rows as
 * above (NW_ERR_CIGAR_TRUNC when msa_ld is below the column count).
 * Device buffers unless NW_HOST_IO.  Synchronises the context's stream. */
int nw_msa_merge(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *off, const uint32_t *len, uint32_t nseq,
                 uint32_t center, uint32_t flags, const char *cigar_pool, const uint64_t *cigar_off,
                 const uint64_t *cigar_len, char *msa, uint64_t msa_ld, uint64_t *msa_cols);

/* ---------------------------------------------------------------- serving
 * Not in the paper (its Sec. 3.2 splits a fixed set of alignments over MPI
 * ranks): a continuous-batching server on one GPU.  The queue is device
 * memory: submitting copies a request's 2-bit sequences into a device arena
 * (`queue_bytes`) and its descriptor into a device ring (`queue_slots`
 * slots, a power of two); one device word holds how many requests were
 * admitted and how many traceback bytes are reserved in flight.  `workers`
 * threads each own a context and stream; each repeatedly runs the device
 * admission kernel, which admits the oldest waiting requests into a batch
 * of at most `max_batch` pairs while the reserved bytes stay within
 * `trace_budget` (a CIGAR request reserves ceil((m+1)(n+1)/4) rounded up to
 * 256 bytes, a score-only request nothing; a request alone on an idle
 * server is always admitted) and claims them atomically.  Batches run from
 * the arena through nw_align_batch (with NW_LEARNED_BAND if given in
 * `flags` and the creating context holds a model, which every worker
 * copies); batches of different workers overlap on the GPU; a finished
 * batch returns its reservation on the device.  Results equal those of
 * nw_align on the same pair.  Submit, poll, drain and the state queries
 * may be called from several host threads at once. */
typedef struct nw_server nw_server;
typedef struct {
    uint64_t ticket;     /* from nw_server_submit                          */
    int32_t status;      /* nw_status of this request                      */
    int32_t score;
    uint64_t cigar_len;  /* 0 for score-only requests                      */
    uint64_t cigar_off;  /* offset of its NUL-terminated CIGAR in cigar_buf */
    double latency_s;    /* completion minus submission (host clock)       */
} nw_completion;

/* NULL on failure (bad sizes: workers 1..16, max_batch 1..2^20,
 * queue_bytes >= 4096, queue_slots a power of two in 2..2^30; or device
 * memory).  The context must outlive the server.  The arena and the ring
 * are allocated on the context's device outside its scratch budget
 * (queue_bytes + 40 * queue_slots bytes).  Each worker's context gets a
 * scratch budget of 1/(workers+1) of what is available at creation: the
 * creating context's unused budget, capped at 90 % of the device's free
 * memory. */
nw_server *nw_server_create_ex(nw_ctx *ctx, uint32_t workers, uint32_t max_batch, uint64_t trace_budget,
                               uint64_t queue_bytes, uint32_t queue_slots, nw_scoring sc, uint32_t flags);
/* nw_server_create_ex with a 1 GiB arena and 2^20 slots. */
nw_server *nw_server_create(nw_ctx *ctx, uint32_t workers, uint32_t max_batch, uint64_t trace_budget, nw_scoring sc,
                            uint32_t flags);
/* Queue one request; sequences are host 2-bit arrays, copied to the
 * device before return.  *ticket identifies its completion.  While the
 * arena or the ring is full of unfinished requests the call waits for
 * completions (NW_ERR_TIMEOUT after 60 s); a request larger than the arena
 * is NW_ERR_ARG. */
int nw_server_submit(nw_server *srv, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n,
                     uint32_t want_cigar, uint64_t *ticket);
/* Queue `count` requests at once from a host pool (same layout as
 * nw_align_batch); want_cigar[k] != 0 asks for pair k's CIGAR; tickets
 * (optional) receives their tickets in order. */
int nw_server_submit_many(nw_server *srv, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                          const uint64_t *b_off, const uint32_t *b_len, const uint8_t *want_cigar, uint32_t count,
                          uint64_t *tickets);
/* Move up to `cap` finished requests (oldest first) into out; their CIGARs
 * go to cigar_buf, NUL-terminated (stops early when cigar_cap would
 * overflow).  When the oldest one's CIGAR alone does not fit, nothing moves,
 * *cigar_used receives the bytes it needs (with the NUL) and the call
 * returns NW_ERR_CIGAR_TRUNC. */
int nw_server_poll(nw_server *srv, nw_completion *out, uint32_t cap, uint32_t *count, char *cigar_buf,
                   uint64_t cigar_cap, uint64_t *cigar_used);
/* The status text and context message of the last batch that failed, with
 * its request count ("" while none has), copied NUL-terminated into buf
 * (cap bytes; truncated to fit).  Returns the full length without the NUL,
 * or -NW_ERR_ARG.  Every request of a failed batch completes with that
 * batch's status. */
int64_t nw_server_last_message(nw_server *srv, char *buf, uint64_t cap);
/* Wait until nothing is queued or running (NW_ERR_TIMEOUT after timeout_s). */
int nw_server_drain(nw_server *srv, double timeout_s);
/* [0] submitted, [1] completed, [2] waiting, [3] running, [4] full-grid
 * cells completed, [5] traceback bytes reserved, [6] batches, [7] budget. */
int nw_server_stats(nw_server *srv, uint64_t *out, int cap);
/* Read the device queue word: requests admitted so far and traceback bytes
 * reserved in flight (synchronises with the intake stream). */
int nw_server_queue_state(nw_server *srv, uint64_t *admitted, uint64_t *reserved_bytes);
/* Finish queued work, stop the workers, free everything.  No other call on
 * this server may be in progress or made afterwards. */
void nw_server_destroy(nw_server *srv);

/* ------------------------------------------------------------ measurement */

/* Integer-pipe peak microbenchmark used as the roofline denominator: every
 * SM runs independent dependency chains of one kind of work for `iters`
 * iterations; *gops receives the measured rate in 1e9 units per second,
 * where a unit is one lane-instruction for kinds 0-4, 8-10 and one
 * score-only cell for kinds 5-7 and 11.  kind: 0 = add-then-max
 * (__viaddmax_s32), 1 = 3-input max (__vimax3_s32), 2 = 2-input max,
 * 3 = 3-input add, 4 = byte permute (prmt), 5 = cell as prmt + add-max +
 * max, 6 = cell as prmt + add + 3-input max, 7 = cell as prmt + add + max +
 * max, 8 = 3-input logic op, 9 = integer multiply-add, 10 = funnel shift,
 * 11 = one anti-diagonal step of the bit-sliced difference update (32
 * cells).  Not in the paper. */
int nw_peak_int(nw_ctx *ctx, int kind, uint64_t iters, double *gops);

#ifdef __cplusplus
}
#endif

#endif /* NW_H_ */
