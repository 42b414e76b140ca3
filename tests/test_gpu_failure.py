"""Failure detection without a GPU fault: a producer that never releases its
progress counter (test hook) makes the consumers' bounded waits run out;
the call reports NW_ERR_TIMEOUT after the limit and the same context then
aligns exactly.  The failure is made on the host side of the protocol (a
counter nothing sets), never by faulting, trapping or hanging the GPU."""
import time

import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu


def test_dropped_progress_times_out_and_context_recovers():
    import torch
    import paper_2412_21103_gb300 as nw
    p = seqgen.long_mutated_pair(4242, m=6000)   # several row groups
    a, b = nw.pack_codes(p.a), nw.pack_codes(p.b)
    with nw.Context(0, torch.cuda.current_stream()) as ctx:
        assert nw.load().nw_ctx_set_test_hook(ctx.handle, 0x80) == nw.NW_ERR_ARG   # unknown hook
        ctx_hook = nw.load().nw_ctx_set_test_hook(ctx.handle, nw.NW_TEST_DROP_PROGRESS)
        assert ctx_hook == nw.NW_OK
        t0 = time.perf_counter()
        with pytest.raises(nw.NWError) as e:
            nw.nw_align(ctx, a, p.a.size, b, p.b.size, (1, -1, -1), 0)
        waited = time.perf_counter() - t0
        assert e.value.status == nw.NW_ERR_TIMEOUT
        assert 1.0 < waited < 30.0          # the 2 s limit, not a hang
        # the hook was used up; the context is usable and exact again
        want_s, ops = oracle.align(p.a, p.b)
        s, cig = nw.nw_align(ctx, a, p.a.size, b, p.b.size, (1, -1, -1), nw.NW_CIGAR)
        assert s == want_s and cig == oracle.rle(ops)
