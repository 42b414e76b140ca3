"""The allocation-free score entry point, for callers that cannot allocate
device memory while aligning (a server that owns all device memory, a
plug-in inside a runtime that owns the allocator, a path where cudaMalloc
would synchronize the device).  Its scores must equal those of nw_align,
bit for bit, on consecutive calls that reuse the shared static scratch.

This file is collected last on purpose, so a failure here never hides the
result of another test."""
import numpy as np
import pytest

import seqgen

pytestmark = pytest.mark.gpu


def _dev(codes):
    import torch
    import paper_2412_21103_gb300 as nw
    return torch.from_numpy(nw.pack_codes(codes)).cuda()


def _reference_score(ctx, a, b, sc):
    import paper_2412_21103_gb300 as nw
    s, _ = nw.nw_align(ctx, nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, sc, 0)
    return s


def test_noalloc_matches_nw_align_on_consecutive_calls():
    import torch
    import paper_2412_21103_gb300 as nw
    ctx = nw.Context(0, torch.cuda.current_stream())
    stream = torch.cuda.current_stream()
    cases = [
        (seqgen.random_pair(1001, 1000, 1000), (1, -1, -1)),       # two 512-row stripes
        (seqgen.long_mutated_pair(3, m=5000), (2, -1, -2)),        # ten stripes: boundary rows used
        (seqgen.long_mutated_pair(4, m=1700), (1, -1, -1)),        # fewer stripes after more: the
    ]                                                              # array still holds the last call
    for pair, sc in cases:
        a, b = pair.a, pair.b
        out = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        rc = nw.nw_align_score_noalloc(_dev(a), a.size, _dev(b), b.size, sc, out, stream)
        assert rc == nw.NW_OK
        assert int(out.item()) == _reference_score(ctx, a, b, sc)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    import torch
    import paper_2412_21103_gb300 as nw
    a = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    # 3 * 2^20 words cannot hold (ceil(m/512) - 1) boundary rows of 200,000 columns for m = 20,000
    rc = nw.nw_align_score_noalloc(a, 20000, a, 200000, (1, -1, -1), out, None)
    assert rc == nw.NW_ERR_ARG


def test_noalloc_empty_side():
    import torch
    import paper_2412_21103_gb300 as nw
    b = seqgen.Stream(1).bases(37)
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = nw.nw_align_score_noalloc(_dev(np.zeros(1, np.uint8)), 0, _dev(b), 37, (1, -1, -1), out, None)
    assert rc == nw.NW_OK and int(out.item()) == -37
