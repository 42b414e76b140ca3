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
    """Consecutive calls share the static scratch: each one must equal both
    nw_align and the oracle.  The cases shrink and grow the stripe count,
    the largest square pair the array allows comes right before the
    longest one (m = 2,000,000 against 64 bases: 3,907 stripes of 512 rows,
    near the 4,096-stripe maximum)."""
    import torch
    import oracle
    import paper_2412_21103_gb300 as nw
    ctx = nw.Context(0, torch.cuda.current_stream())
    stream = torch.cuda.current_stream()
    rs = seqgen.Stream(77)
    cases = [
        (seqgen.random_pair(1001, 1000, 1000), (1, -1, -1)),       # two 512-row stripes
        (seqgen.long_mutated_pair(3, m=5000), (2, -1, -2)),        # ten stripes: boundary rows used
        (seqgen.long_mutated_pair(4, m=1700), (1, -1, -1)),        # fewer stripes after more: the
                                                                   # array still holds the last call
        (seqgen.long_mutated_pair(5, m=32768), (1, -1, -1)),       # 64 stripes of 32,768 columns
        (seqgen.Pair(rs.bases(2_000_000), rs.bases(64)), (1, -1, -1)),  # 3,907 stripes
        (seqgen.random_pair(9, 700, 900), (-3, -5, -1)),           # diagonal never beats two gaps
    ]
    for pair, sc in cases:
        a, b = pair.a, pair.b
        out = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        rc = nw.nw_align_score_noalloc(_dev(a), a.size, _dev(b), b.size, sc, out, stream)
        assert rc == nw.NW_OK
        got = int(out.item())
        assert got == _reference_score(ctx, a, b, sc)
        assert got == oracle.score(a, b, *sc)
    ctx.close()


def test_noalloc_rejects_tensors_off_the_device():
    """The binding refuses host tensors and a wrong score type before any
    pointer reaches the kernel."""
    import torch
    import paper_2412_21103_gb300 as nw
    a = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        nw.nw_align_score_noalloc(a.cpu(), 8, a, 8, (1, -1, -1), torch.zeros(1, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        nw.nw_align_score_noalloc(a, 8, a, 8, (1, -1, -1), torch.zeros(1, dtype=torch.int64, device="cuda"))


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
