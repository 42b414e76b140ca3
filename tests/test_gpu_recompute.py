"""Stripe-checkpoint recompute (a6): when the 2-bit pointer matrix does not
fit the context's memory budget (or NW_RECOMPUTE asks for it), the single-
pair path keeps one W row per group of stripes, refills the pointers wave by
wave from the bottom and walks each wave.  Scores and CIGARs must stay
bit-exact against the oracle, and the recompute kernels must really run."""
import numpy as np
import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu


def _geometry(m, n):
    """Rows per lane, groups and per-group pointer bytes of the single-pair
    path (R = 8 from m >= 2048, else 4; 4 stripes per group)."""
    R = 8 if m >= 2048 else 4
    cpw = 16 // R
    ncg = -(-(-(-n // cpw)) // 32) * 32
    S = -(-m // (32 * R))
    groups = -(-S // 4)
    return R, groups, 4 * 32 * ncg * 4, S * 32 * ncg * 4


def _budget_for(m, n, waves_of=2):
    """A budget that holds the checkpoints, the host staging and `waves_of`
    groups of pointers, but not the whole pointer matrix."""
    R, groups, group_bytes, full = _geometry(m, n)
    bstride = (n + 64 + 63) // 64 * 64
    rows = max(groups - 1, 0) * bstride * 4 + 4 * bstride
    small = 64 * 1024 + 8 * (m + n)
    return rows + small + int(waves_of * group_bytes * 1.13) + 4096, full


def _align(ctx, a, b, sc=(1, -1, -1), flags=0):
    import paper_2412_21103_gb300 as nw
    return nw.nw_align(ctx, nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, sc, nw.NW_CIGAR | flags)


def _pairs():
    rs = seqgen.Stream(6006)
    out = [
        ("random 3000x3000", rs.bases(3000), rs.bases(3000)),
        ("ragged 3333x2900", rs.bases(3333), rs.bases(2900)),
        ("tall 3000x200 (path reaches column 0)", rs.bases(3000), rs.bases(200)),
        ("wide 700x5000 (three groups)", rs.bases(700), rs.bases(5000)),
    ]
    p = seqgen.long_mutated_pair(6007, m=4100)
    out.append(("mutated 4100", p.a, p.b))
    return out


@pytest.mark.parametrize("k", range(5))
def test_budget_below_pointer_matrix_recomputes_exactly(k):
    import torch
    import paper_2412_21103_gb300 as nw
    name, a, b = _pairs()[k]
    groups = _geometry(a.size, b.size)[1]
    budget, full = _budget_for(a.size, b.size, waves_of=2 if groups > 3 else 1)
    assert budget < full, name
    with nw.Context(0, torch.cuda.current_stream(), mem_budget=budget) as ctx:
        ctx.set_profiling(True)
        s, cig = _align(ctx, a, b)
        stats = ctx.kernel_stats()
    want_s, ops = oracle.align(a, b)
    assert s == want_s, name
    assert cig == oracle.rle(ops), name
    assert stats.get("fill_recompute", (0, 0))[0] >= 1, (name, stats)


@pytest.mark.parametrize("m,n", [(1, 1), (1, 700), (700, 1), (5, 9), (64, 64), (129, 257), (513, 300),
                                 (1024, 1024), (1025, 2049), (2048, 31), (4097, 4095)])
@pytest.mark.parametrize("sc", [(1, -1, -1), (2, -1, -2), (3, -3, -1)])
def test_recompute_flag_matches_oracle(m, n, sc):
    import torch
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(m * 7919 + n)
    a, b = rs.bases(m), rs.bases(n)
    with nw.Context(0, torch.cuda.current_stream()) as ctx:
        ctx.set_profiling(True)
        s, cig = _align(ctx, a, b, sc, nw.NW_RECOMPUTE)
        stats = ctx.kernel_stats()
        s_full, cig_full = _align(ctx, a, b, sc)
    want_s, ops = oracle.align(a, b, *sc)
    assert (s, cig) == (want_s, oracle.rle(ops))
    assert (s_full, cig_full) == (s, cig)
    assert stats.get("fill_recompute", (0, 0))[0] >= 1


def test_one_wave_per_group_and_repeat_calls():
    """The tightest budget (one group per wave) and a second call on the same
    context (checkpoint buffers reused) give the same exact result."""
    import torch
    import paper_2412_21103_gb300 as nw
    p = seqgen.long_mutated_pair(6010, m=3500)
    budget, _ = _budget_for(p.a.size, p.b.size, waves_of=1)
    want_s, ops = oracle.align(p.a, p.b)
    with nw.Context(0, torch.cuda.current_stream(), mem_budget=budget) as ctx:
        for _ in range(2):
            s, cig = _align(ctx, p.a, p.b)
            assert s == want_s and cig == oracle.rle(ops)


def test_budget_below_one_group_is_oom():
    import torch
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(6011)
    a, b = rs.bases(3000), rs.bases(3000)
    with nw.Context(0, torch.cuda.current_stream(), mem_budget=96 * 1024) as ctx:
        with pytest.raises(nw.NWError) as e:
            _align(ctx, a, b)
        assert e.value.status == nw.NW_ERR_OOM
        ctx.sync()


def test_batch_pair_over_budget_takes_recompute():
    """In a CIGAR batch, a pair whose pointers exceed half the remaining
    budget goes to the single-pair path, which recomputes; the small pairs
    stay batched.  Every result is the oracle's."""
    import torch
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(6012)
    big = seqgen.long_mutated_pair(6013, m=3600)
    pairs = [(big.a, big.b)] + [(rs.bases(int(L)), rs.bases(int(L) + 3)) for L in rs.integers(50, 400, 12)]
    seqs = []
    for a, b in pairs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    budget, full = _budget_for(big.a.size, big.b.size, waves_of=2)
    budget += 2 * pool.nbytes + 64 * 1024
    with nw.Context(0, torch.cuda.current_stream(), mem_budget=budget) as ctx:
        ctx.set_profiling(True)
        scores, cigars = nw.nw_align_batch(ctx, pool, off[0::2], lens[0::2], off[1::2], lens[1::2], (1, -1, -1),
                                           nw.NW_CIGAR)
        stats = ctx.kernel_stats()
    want = oracle.align_many(pairs)
    for k, (s, ops) in enumerate(want):
        assert scores[k] == s and cigars[k] == oracle.rle(ops), k
    assert stats.get("fill_recompute", (0, 0))[0] >= 1, stats
