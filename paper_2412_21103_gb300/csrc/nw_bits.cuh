// Bit-sliced fills (nw_bits.cu: score-only batches; nw_bits_band.cu: the
// certified band with pointers): shared declarations and device helpers.
#pragma once

#include <string>
#include <vector>

#include "nw_internal.cuh"

namespace nw {

constexpr int64_t kPlanePad = 64;  // bases of padding in front of base 0 of the planar pool
constexpr int kBitsWarps = 8;      // warps per CTA

// Three-input logic operation with the truth table LUT (PTX lop3).
template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}
// Truth tables from the canonical inputs a = 0xF0, b = 0xCC, c = 0xAA.
constexpr uint32_t kA = 0xF0, kB = 0xCC, kC = 0xAA;
constexpr uint32_t lut(uint32_t v) { return v & 0xFFu; }
constexpr uint32_t kLutXorOrNotC = lut((kA ^ kB) | ~kC);     // (a ^ b) | ~c
constexpr uint32_t kLutEq = lut(~(kA ^ kB) & ~kC);           // ~(a ^ b) & ~c
constexpr uint32_t kLutAndOrNot = lut(kA & (kB | ~kC));      // a & (b | ~c)
constexpr uint32_t kLutCOrNor = lut(kC | (~kA & ~kB));       // c | ~(a | b)
constexpr uint32_t kLutOrAnd = lut(kA | (kB & kC));          // a | (b & c)
constexpr uint32_t kLutOr3 = lut(kA | kB | kC);              // a | b | c
constexpr uint32_t kLutXor3 = lut(kA ^ kB ^ kC);             // a ^ b ^ c
constexpr uint32_t kLutAndNot = lut(kA & ~kB);               // a & ~b
constexpr uint32_t kLutXorAnd = lut((kA ^ kB) & kC);         // (a ^ b) & c
constexpr uint32_t kLutSel = lut((kA & kB) | (~kA & kC));    // a ? b : c
constexpr uint32_t kLutAndNotOr = lut(kA & (~kB | kC));      // a & (~b | c)

// 32 bits of a planar sequence plane starting at global base index g.
__device__ __forceinline__ uint32_t plane_window(const uint32_t *pl, int64_t g) {
    const uint64_t x = (uint64_t)(g + kPlanePad);
    return __funnelshift_r(__ldg(pl + (x >> 5)), __ldg(pl + (x >> 5) + 1), (uint32_t)x & 31u);
}

// The two planes of s' for a general scoring with 0 <= s'x <= s'm <= 3:
// bit k of s'(match) / s'(mismatch) as all-ones or zero words.
struct BitsScoring {
    uint32_t M1, M0, X1, X0;
};

struct BitsJob {
    uint32_t t0, cnt;  // tasks [t0, t0 + cnt), cnt <= 32, one per lane
    uint32_t S, C;     // stripes, chunks per stripe (the job's largest)
};

struct BitsArgs {
    const uint32_t *pl0, *pl1;  // planar sequences: bit k of global base g at word (g+64)>>5, bit (g+64)&31
    const BatchTask *tasks;     // a_off / b_off: the sequences' slots (global base indices)
    const BitsJob *jobs;
    uint32_t njobs;
    uint32_t *counter;
    uint2 *rows;          // per warp: rows_chunks x 32 lanes of (plane 0, plane 1) words
    uint32_t rows_chunks;
    int32_t *scores;
    uint32_t score_cap;
    int32_t gap;
    BitsScoring g;
    uint32_t *err;
};

// Planar copy of the sequences a launch reads.  Each distinct sequence
// (pool byte offset, length) gets a slot of whole 32-base words, two words
// apart; a kernel addresses base i of the sequence as global base index
// slot + i.  Only the launch's own sequences are copied, wherever they lie
// in the pool.
struct PlaneSeg {
    uint64_t src;      // pool byte offset of the sequence (its device address when the pool is null)
    uint32_t nbytes;   // its packed bytes
    uint32_t dst;      // first word of its slot
};
class PlaneSet {
  public:
    // Room for n sequences without regrowing.
    void reserve(size_t n);
    // Slot (global base index of base 0) of the sequence at pool byte `off`
    // with `len` bases, added on first use.
    int64_t add(uint64_t off, uint32_t len);
    // Enqueues the copy (one H2D table, one kernel); pl0 / pl1 receive the
    // two planes, max_base the largest base index a 32-bit window may start at.
    // With a null pool the offsets given to add() are device addresses.
    int launch(nw_ctx *ctx, const uint8_t *pool, const std::string &prefix);
    // Uploads the segment table and sizes the planes without copying (the
    // copy can then be enqueued, also into a graph, by enqueue()).
    int prepare(nw_ctx *ctx, const std::string &prefix);
    int enqueue(nw_ctx *ctx, const uint8_t *pool) const;
    const uint32_t *pl0 = nullptr, *pl1 = nullptr;
    int64_t max_base = 0;

  private:
    // open addressing (linear probing, at most half full): one table of
    // entries instead of a node per sequence
    struct Entry {
        uint64_t off;
        uint32_t len, used;
        int64_t slot;
    };
    std::vector<Entry> table_;
    size_t count_ = 0;
    void rehash(size_t size);
    std::vector<PlaneSeg> segs_;
    uint64_t words_ = 2;  // kPlanePad bases in front of the first slot
    PlaneSeg *dsegs_ = nullptr;
    uint32_t *planes_ = nullptr;
};

// Everything a launch needs, prepared (sorted, uploaded, scratch sized)
// ahead of the launch so that the launch itself only enqueues kernels.
struct BitsPlan {
    BitsArgs ba{};
    uint32_t blocks = 0;
    const uint8_t *pool = nullptr;
    PlaneSet planes;
    bool gen = false;
};

// 0 <= s'(mismatch) <= s'(match) <= 3, s' = s - 2*gap: every difference fits two bits.
bool bits_scoring_ok(const nw_scoring &sc);
// Orients, groups and uploads the tasks (reordered in place), sizes the
// scratch; scores[out0] (and scores[out1]) receive each task's score.
int bits_prepare(nw_ctx *ctx, const uint8_t *pool, std::vector<BatchTask> &tasks,
                 const nw_scoring &sc, int32_t *scores, uint32_t score_cap, const std::string &prefix, BitsPlan *plan);
// Enqueues the planar copy of the pool and the fill (no host copies: it can
// be captured into a graph).
int bits_launch(nw_ctx *ctx, const BitsPlan &plan);

// ---- one long pair on the bit-sliced stripes (nw_bits_pair.cu)
// Whether the pair runs there (the paper's scoring, long enough to spread
// over several warps, every warp co-resident, pointers within the budget).
bool bits_pair_takes(nw_ctx *ctx, uint32_t m, uint32_t n, const nw_scoring &sc, bool want);
// Score (and with `want` the CIGAR, written by the CIGAR assembly) of one pair.
int bits_pair(nw_ctx *ctx, const uint8_t *a2b, uint32_t m, const uint8_t *b2b, uint32_t n, const nw_scoring &sc,
              bool want, uint32_t mflag, int32_t *score, char *cigar, uint64_t *cigar_len);
// Many pairs, each on its own warps: waves of pairs whose warps are all
// resident at once, longest chains first.  a_off / b_off: byte offsets into
// `pool` (device addresses when it is null).  Every job must pass
// bits_pair_takes.
struct PairJob {
    uint64_t a_off, b_off;
    uint32_t m, n;
    int32_t *score;
    char *cigar;
    uint64_t *cigar_len;
};
int bits_pairs(nw_ctx *ctx, const uint8_t *pool, const std::vector<PairJob> &jobs, const nw_scoring &sc, bool want,
               uint32_t mflag);

// ---- the certified band on the bit-sliced window (nw_bits_band.cu)
// Window of one pair: g lanes (a power of two) x Q words of 32 rows, its
// anchor diagonal hi (the band's upper diagonal raised to the parity of
// m+n), and its anti-diagonals a_first .. m+n in chunks of 64.
struct BandBitsShape {
    uint32_t g = 1, Q = 1, nchunks = 0;
    int32_t hi = 0, a_first = 0;
    uint32_t words = 1;  // the band needs this many 32-row words (g * Q >= words)
};
// One banded pair of a round: pool offsets, sizes, score slot, window, and
// its first pointer record (16 bytes per word and pair of anti-diagonals).
struct BandBitsItem {
    uint64_t a_off, b_off, ptr_off;  // pool byte offsets (the walk), first pointer record
    int64_t a_slot, b_slot;          // the sequences' planar slots (the fill)
    uint32_t m, n, out0;
    BandBitsShape shape;
};
// Most words per lane of the throughput shape: 4, or NW_BBAND_MAXQ (1..4)
// when set (read on each call; a round reads it once).
int band_bits_max_q();
// The window of the band of diagonals [lo, hi] on the fewest lanes of at
// most max_q words each; false when it needs more than 128 words (4,096
// rows).
bool band_bits_shape(uint32_t m, uint32_t n, int32_t lo, int32_t hi, BandBitsShape *s, int max_q);
// The same window spread over as many lanes as it has words (up to 32):
// fewer instructions per lane and step, so a shorter time for the pair.
void band_bits_fast(BandBitsShape *s);
uint64_t band_bits_records(const BandBitsShape &s);  // pointer records of the pair
// The widest half-width whose band fits the window of an m x n pair.
uint32_t band_bits_max_width(uint32_t m, uint32_t n);
double band_bits_seconds(const BandBitsShape &s);    // estimated time of the pair on one warp
// Fills the items (the paper's scoring: s' = 3 on a match, 1 on a
// mismatch), writes scores[out0], returns the banded scores in item order,
// and with `want` the pointer records at ptr + ptr_off.
int band_bits_fill(nw_ctx *ctx, const PlaneSet &planes, const std::vector<BandBitsItem> &items, bool want, int32_t gap, int32_t *scores, uint32_t score_cap,
                   void *ptr, uint64_t ptr_records, std::vector<int32_t> &banded);
// Walks the items `which` of a filled wave and writes their CIGARs.
int band_bits_walk(nw_ctx *ctx, const void *ptr, const std::vector<BandBitsItem> &items,
                   const std::vector<uint32_t> &which, const uint8_t *pool, char *cigar_pool,
                   const uint64_t *cigar_off, uint64_t *cigar_len, uint32_t mflag);

}  // namespace nw
