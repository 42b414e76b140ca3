"""GPU parity of the bit-sliced single-pair fill (one 31-row stripe per lane,
warps chained through a tagged ring, pointer records per stripe and step)
and its stripe-parallel walk, against the oracle: scores and CIGAR strings
bit-exact.  Shapes cover one warp and many, ragged stripe counts (the last
warp partly empty), spare rows below row m, one column chunk and many,
pairs much taller than wide and the reverse; scorings with s' = (3, 1)
(the paper's) and the general two-plane form; repeated calls (new ring
epochs) and a second context (a ring that must be cleared first)."""
import os

import numpy as np
import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_2412_21103_gb300 as nw
    c = nw.Context(0, torch.cuda.current_stream())
    c.set_profiling(True)
    yield c
    c.close()


def _align(ctx, a, b, sc=(1, -1, -1), cigar=True):
    import paper_2412_21103_gb300 as nw
    return nw.nw_align(ctx, nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, sc, nw.NW_CIGAR if cigar else 0)


def _launches(ctx, name):
    return ctx.kernel_stats().get(name, (0, 0.0))[0]


def _pair(seed, m, n, div=0.1):
    rs = seqgen.Stream(seed)
    a = rs.bases(m)
    if n <= m:
        b, _ = seqgen.mutate_distinct(a[:n].copy(), rs, div, indel_frac=0.2, indel_mean=3.0)
    else:
        b, _ = seqgen.mutate_distinct(np.concatenate([a, rs.bases(n - m)]), rs, div, indel_frac=0.2, indel_mean=3.0)
    return a, b


def _check(ctx, a, b, sc=(1, -1, -1)):
    f0, p0 = _launches(ctx, "bpair_fill"), _launches(ctx, "bpair_fill_ptr")
    want_s, want_ops = oracle.align(a, b, *sc)
    s, cig = _align(ctx, a, b, sc)
    assert s == want_s, (a.size, b.size)
    assert cig == oracle.rle(want_ops), (a.size, b.size)
    s2, _ = _align(ctx, a, b, sc, cigar=False)
    assert s2 == want_s
    assert _launches(ctx, "bpair_fill_ptr") == p0 + 1 and _launches(ctx, "bpair_fill") == f0 + 1


SHAPES = [(64, 64), (100, 64), (64, 3000), (1000, 1000), (1023, 97), (1024, 500), (1025, 500), (1056, 64),
          (2047, 333), (2100, 2100), (3000, 70), (4133, 1200), (70, 5000), (6000, 6100)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_shapes_exact(ctx, m, n):
    a, b = _pair(9100 + m + 7 * n, m, n)
    _check(ctx, a, b)


@pytest.mark.parametrize("m,n", [(1500, 1400), (3000, 200)])
def test_unrelated_sequences(ctx, m, n):
    rs = seqgen.Stream(9200 + m)
    _check(ctx, rs.bases(m), rs.bases(n))


@pytest.mark.parametrize("sc", [(1, 0, -1), (0, -1, -1), (1, 1, -1), (0, 0, -1), (0, -2, -1), (-1, -3, -2), (-2, -3, -2)])
def test_general_scorings(ctx, sc):
    a, b = _pair(9300, 1500, 1450, div=0.15)
    _check(ctx, a, b, sc)


def test_identical_and_shifted(ctx):
    rs = seqgen.Stream(9400)
    a = rs.bases(2500)
    _check(ctx, a, a.copy())
    _check(ctx, a, a[37:].copy())
    _check(ctx, a[:2000].copy(), np.concatenate([rs.bases(300), a[:2000]]))


def test_repeated_calls_and_second_context(ctx):
    """New epochs on the same ring give the same results; a second context
    clears its own ring before its first launch."""
    import torch
    import paper_2412_21103_gb300 as nw
    a, b = _pair(9500, 3000, 2900)
    want_s, want_ops = oracle.align(a, b)
    for _ in range(3):
        assert _align(ctx, a, b) == (want_s, oracle.rle(want_ops))
    with nw.Context(0, torch.cuda.current_stream()) as c2:
        for _ in range(2):
            assert _align(c2, a, b) == (want_s, oracle.rle(want_ops))
    assert _align(ctx, a, b) == (want_s, oracle.rle(want_ops))


def test_scalar_and_bits_paths_agree(ctx):
    a, b = _pair(9600, 2500, 2600, div=0.2)
    s1 = _align(ctx, a, b)
    os.environ["NW_PAIR_SCALAR"] = "1"
    try:
        before = _launches(ctx, "bpair_fill_ptr")
        s2 = _align(ctx, a, b)
        assert _launches(ctx, "bpair_fill_ptr") == before
    finally:
        del os.environ["NW_PAIR_SCALAR"]
    assert s1 == s2


def test_small_sides_take_the_scalar_kernel(ctx):
    a, b = _pair(9700, 2000, 40)
    before = _launches(ctx, "bpair_fill_ptr")
    want_s, want_ops = oracle.align(a, b)
    assert _align(ctx, a, b) == (want_s, oracle.rle(want_ops))
    assert _launches(ctx, "bpair_fill_ptr") == before


def test_config2_pair_exact(ctx):
    """The 32,768-base pair with 10 % substitutions and 2 % indels: score and
    CIGAR equal the oracle's."""
    p = seqgen.long_mutated_pair(1002)
    before = _launches(ctx, "bpair_fill_ptr")
    want_s, want_ops = oracle.align(p.a, p.b)
    s, cig = _align(ctx, p.a, p.b)
    assert _launches(ctx, "bpair_fill_ptr") == before + 1
    assert s == want_s and cig == oracle.rle(want_ops)
