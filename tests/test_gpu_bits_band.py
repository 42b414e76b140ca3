"""GPU parity of the bit-sliced certified band (the window kernel that follows
the band, pointer records per pair of anti-diagonals, and its walk) against
the oracle.  Every result of a certified-band call equals full NW exactly
(score and CIGAR); the certificate's decisions on the window kernel's scores
lie between what the strict band and what the full grid allow; the scalar
banded kernel (NW_BAND_SCALAR=1) and the window kernel give the same
results; shapes cover one to 32 lanes per pair and one to eight words per
lane, ragged lengths, large length differences and tiny pairs."""
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


def _pool(pairs):
    import paper_2412_21103_gb300 as nw
    seqs = [s for p in pairs for s in p]
    pool, off, lens = nw.pool_of(seqs)
    return pool, off[0::2], lens[0::2], off[1::2], lens[1::2]


def _pairs(seed, count, lmin, lmax, divergence=(0.01, 0.25), shrink=0.2):
    rs = seqgen.Stream(seed)
    out = []
    for k in range(count):
        m = int(rs.integers(lmin, lmax, 1)[0])
        a = rs.bases(m)
        d = float(divergence[0] + (divergence[1] - divergence[0]) * rs.uniform(1)[0])
        b, _ = seqgen.mutate_distinct(a, rs, d, indel_frac=0.3, indel_mean=3.0)
        if k % 4 == 0 and b.size > 4:
            b = b[: max(1, int(b.size * (1 - shrink * rs.uniform(1)[0])))]   # length difference
        if k % 7 == 3:
            a, b = b, a
        out.append((a, b))
    return out


def _launches(c, name):
    return c.kernel_stats().get(name, (0, 0.0))[0]


def _check_exact(pairs, scores, cigars, sc=(1, -1, -1)):
    want = oracle.align_many(pairs, *sc)
    for k, (s, ops) in enumerate(want):
        assert scores[k] == s, (k, pairs[k][0].size, pairs[k][1].size)
        if cigars is not None:
            assert cigars[k] == oracle.rle(ops), (k, pairs[k][0].size, pairs[k][1].size)


@pytest.mark.parametrize("w", [0, 2, 9, 40, 150, 700])
def test_fixed_widths_exact(ctx, w):
    """Half-widths from 0 (one word) to 700 (many lanes and words); the wide
    bands on longer pairs, so that the band stays below the share of the grid
    that sends a pair straight to the full kernel."""
    import paper_2412_21103_gb300 as nw
    pairs = _pairs(600 + w, 48, 1, 1800 if w < 150 else 7000)
    pool, ao, al, bo, bl = _pool(pairs)
    before = _launches(ctx, "bband_fill_ptr")
    scores, cigars = nw.nw_align_batch_banded(ctx, pool, ao, al, bo, bl, np.full(len(pairs), w, np.uint32),
                                              (1, -1, -1), nw.NW_CIGAR)
    assert _launches(ctx, "bband_fill_ptr") > before
    _check_exact(pairs, scores, cigars)
    s_only, _ = nw.nw_align_batch_banded(ctx, pool, ao, al, bo, bl, np.full(len(pairs), w, np.uint32),
                                         (1, -1, -1), 0)
    assert s_only.tolist() == list(scores)


@pytest.mark.parametrize("fast", ["1", "0"])
def test_every_window_shape(ctx, fast):
    """Bands from one word to 255 words: up to 128 words on the window
    kernel, wider ones on the scalar banded kernel.  A batch this small puts
    most pairs on the latency shape (one word per lane up to 32 lanes, then
    32 lanes of up to 4 words); NW_BBAND_FAST=0 keeps them on the throughput
    shape (the fewest lanes of up to 4 words: every word count 1..4 and lane
    count 1..32)."""
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(610)
    pairs, ws = [], []
    for words in [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16, 17, 24, 30, 33, 40, 50, 64, 65, 100, 128, 129, 200, 255]:
        w = max(0, (64 * words - 8) // 2 - 2)
        m = int(rs.integers(max(200, w), 2 * w + 600, 1)[0])
        a = rs.bases(m)
        b, _ = seqgen.mutate_distinct(a, rs, 0.3, indel_frac=0.3, indel_mean=3.0)
        pairs.append((a, b))
        ws.append(w)
    pool, ao, al, bo, bl = _pool(pairs)
    os.environ["NW_BBAND_FAST"] = fast
    os.environ["NW_BAND_KEEP"] = "1"  # no pair leaves for the full grid
    try:
        scores, cigars = nw.nw_align_batch_banded(ctx, pool, ao, al, bo, bl, np.array(ws, np.uint32), (1, -1, -1),
                                                  nw.NW_CIGAR)
    finally:
        del os.environ["NW_BBAND_FAST"]
        del os.environ["NW_BAND_KEEP"]
    _check_exact(pairs, scores, cigars)


def test_tiny_and_skewed_pairs(ctx):
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(620)
    shapes = [(1, 1), (1, 2), (2, 1), (1, 40), (40, 1), (3, 3), (31, 33), (64, 64), (65, 1), (1, 65),
              (100, 900), (900, 100), (5, 600), (600, 5), (257, 255)]
    pairs = [(rs.bases(m), rs.bases(n)) for m, n in shapes]
    pairs += [(a, a.copy()) for a in (rs.bases(1), rs.bases(33), rs.bases(500))]
    pool, ao, al, bo, bl = _pool(pairs)
    for w in (0, 3, 50):
        scores, cigars = nw.nw_align_batch_banded(ctx, pool, ao, al, bo, bl, np.full(len(pairs), w, np.uint32),
                                                  (1, -1, -1), nw.NW_CIGAR)
        _check_exact(pairs, scores, cigars)


def test_certificate_decisions_lie_between_band_and_full(ctx):
    """The window contains the band and every computed value is reached by
    a path, so the first round certifies every pair whose strict banded score
    beats the exit bound, and only pairs whose full score does."""
    import torch
    import paper_2412_21103_gb300 as nw
    pairs = _pairs(630, 40, 200, 1500, divergence=(0.02, 0.3))
    pool, ao, al, bo, bl = _pool(pairs)
    w = 24
    with nw.Context(0, torch.cuda.current_stream()) as c:
        nw.nw_align_batch_banded(c, pool, ao, al, bo, bl, np.full(len(pairs), w, np.uint32), (1, -1, -1),
                                 nw.NW_CIGAR)
        rnd = nw.nw_ctx_band_outcome(c)["round"]
    full = oracle.score_many(pairs)
    for k, (a, b) in enumerate(pairs):
        U = oracle.exit_bound(a.size, b.size, w)
        sb, _ = oracle.banded(a, b, w)
        if rnd[k] == 1:
            assert U is None or full[k] > U, k
        else:
            # not certified in round 1: the strict band did not beat U either,
            # unless the pair went straight to the full kernel (round 0)
            assert rnd[k] == 0 or (U is not None and sb <= U), k


def test_window_and_scalar_band_kernels_agree(ctx):
    import paper_2412_21103_gb300 as nw
    pairs = _pairs(640, 60, 100, 2500)
    pool, ao, al, bo, bl = _pool(pairs)
    ws = np.array([[8, 30, 64, 200][k % 4] for k in range(len(pairs))], np.uint32)
    s1, c1 = nw.nw_align_batch_banded(ctx, pool, ao, al, bo, bl, ws, (1, -1, -1), nw.NW_CIGAR)
    os.environ["NW_BAND_SCALAR"] = "1"
    try:
        s2, c2 = nw.nw_align_batch_banded(ctx, pool, ao, al, bo, bl, ws, (1, -1, -1), nw.NW_CIGAR)
    finally:
        del os.environ["NW_BAND_SCALAR"]
    assert s1.tolist() == s2.tolist() and c1 == c2
    _check_exact(pairs, s1, c1)


def test_small_budget_waves(ctx):
    """A context whose budget holds only a few pairs' pointer records runs
    the window kernel in many waves."""
    import torch
    import paper_2412_21103_gb300 as nw
    pairs = _pairs(650, 30, 500, 3000)
    pool, ao, al, bo, bl = _pool(pairs)
    ws = np.full(len(pairs), 48, np.uint32)
    with nw.Context(0, torch.cuda.current_stream(), mem_budget=64 << 20) as c:
        scores, cigars = nw.nw_align_batch_banded(c, pool, ao, al, bo, bl, ws, (1, -1, -1), nw.NW_CIGAR)
    _check_exact(pairs, scores, cigars)


def test_learned_band_on_config4_sample_exact(ctx):
    """The certified learned band (no model: fixed start) on a sample of the
    2-20 kb workload: every score and CIGAR equals the oracle's."""
    import paper_2412_21103_gb300 as nw
    pairs = [(p.a, p.b) for p in seqgen.band_pairs(1004, npairs=24)]
    pool, ao, al, bo, bl = _pool(pairs)
    before = _launches(ctx, "bband_fill_ptr")
    scores, cigars = nw.nw_align_batch(ctx, pool, ao, al, bo, bl, (1, -1, -1), nw.NW_CIGAR | nw.NW_LEARNED_BAND)
    assert _launches(ctx, "bband_fill_ptr") > before
    _check_exact(pairs, scores, cigars)
