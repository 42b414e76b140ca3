/* Plain C99 user of the library's C ABI: includes nw.h from a C compiler,
 * links libnw.so and calls the entry points that need no GPU.  Prints one
 * line of results for tests/test_abi.py to compare. */
#include <stdint.h>
#include <stdio.h>

#include "nw.h"

int main(void) {
    uint8_t packed[3] = {0, 0, 0};
    int rc_pack = nw_pack("ACGTacgtA", 9, packed);
    uint8_t dummy[1];
    int rc_bad = nw_pack("ACGN", 4, dummy);
    int64_t bound = 0;
    nw_scoring sc = {1, -1, -1};
    int rc_bound = nw_band_exit_bound(100, 120, 5, sc, &bound);
    int cert = nw_band_certifies(1000, 1000, 64, 900, sc, 1);
    long long next = (long long)nw_band_next_width(1000, 1000, 64, 500, sc, 1);
    nw_ctx *ctx = nw_ctx_create(0, NULL, 0); /* NULL without a usable GPU */
    printf("%d %u %u %u %d %d %lld %llu %d %lld %s\n", rc_pack, packed[0], packed[1], packed[2], rc_bad, rc_bound,
           (long long)bound, (unsigned long long)nw_cigar_bound(3, 4), cert, next, nw_strerror(NW_ERR_BAD_BASE));
    if (ctx) nw_ctx_destroy(ctx);
    return 0;
}
