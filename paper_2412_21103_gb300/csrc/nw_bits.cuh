// Bit-sliced score-only fill (nw_bits.cu): shared declarations.
#pragma once

#include <string>
#include <vector>

#include "nw_internal.cuh"

namespace nw {

constexpr int64_t kPlanePad = 64;  // bases of padding in front of base 0 of the planar pool
constexpr int kBitsWarps = 8;      // warps per CTA

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
    const uint32_t *pl0, *pl1;  // planar pool: bit k of global base g at word (g+64)>>5, bit (g+64)&31
    const BatchTask *tasks;
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

// Everything a launch needs, prepared (sorted, uploaded, scratch sized)
// ahead of the launch so that the launch itself only enqueues kernels.
struct BitsPlan {
    BitsArgs ba{};
    uint32_t blocks = 0, nwords = 0;
    const uint8_t *pool = nullptr;
    uint64_t pool_bytes = 0;
    bool gen = false;
};

// 0 <= s'(mismatch) <= s'(match) <= 3, s' = s - 2*gap: every difference fits two bits.
bool bits_scoring_ok(const nw_scoring &sc);
// Bytes of the pool the tasks read.
uint64_t bits_pool_bytes(const std::vector<BatchTask> &tasks);
// Orients, groups and uploads the tasks (reordered in place), sizes the
// scratch; scores[out0] (and scores[out1]) receive each task's score.
int bits_prepare(nw_ctx *ctx, const uint8_t *pool, uint64_t pool_bytes, std::vector<BatchTask> &tasks,
                 const nw_scoring &sc, int32_t *scores, uint32_t score_cap, const std::string &prefix, BitsPlan *plan);
// Enqueues the planar copy of the pool and the fill (no host copies: it can
// be captured into a graph).
int bits_launch(nw_ctx *ctx, const BitsPlan &plan);

}  // namespace nw
