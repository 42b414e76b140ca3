// Batched pairs and all-vs-all scores.
#include "nw_internal.cuh"

using namespace nw;

extern "C" int nw_align_batch(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *a_off, const uint32_t *a_len,
                              const uint64_t *b_off, const uint32_t *b_len, uint32_t npairs, nw_scoring sc,
                              uint32_t flags, int32_t *scores, char *cigar_pool, const uint64_t *cigar_off,
                              uint64_t *cigar_len) {
    (void)pool2b; (void)a_off; (void)a_len; (void)b_off; (void)b_len; (void)npairs; (void)sc; (void)flags;
    (void)scores; (void)cigar_pool; (void)cigar_off; (void)cigar_len;
    return fail(ctx, NW_ERR_UNSUPPORTED, "batched alignment is not built yet");
}

extern "C" int nw_score_all_pairs(nw_ctx *ctx, const uint8_t *pool2b, const uint64_t *off, const uint32_t *len,
                                  uint32_t nseq, nw_scoring sc, uint32_t flags, int32_t *out) {
    (void)pool2b; (void)off; (void)len; (void)nseq; (void)sc; (void)flags; (void)out;
    return fail(ctx, NW_ERR_UNSUPPORTED, "all-pairs scoring is not built yet");
}
