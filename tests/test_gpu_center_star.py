"""GPU parity of the center-star multiple alignment (Sec. 3.2) against the
CPU oracle: the center, the row sums, every score and CIGAR against the
center and every merged row, bit-exact -- on the hand-worked family, on
edge cases (empty sequences, one and two sequences, ties) and on the
512-sequence all-vs-all family at full size."""
import os

import numpy as np
import pytest

import oracle
import seqgen
from oracle import center_star as cs

from helpers import GOLDEN, codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_2412_21103_gb300 as nw
    c = nw.Context(0, torch.cuda.current_stream())
    yield c
    c.close()


def _check(ctx, seqs, sc=(1, -1, -1)):
    import paper_2412_21103_gb300 as nw
    pool, off, lens = nw.pool_of(seqs)
    got = nw.nw_center_star(ctx, pool, off, lens, sc)
    c, sums, aligned, rows = cs.center_star(seqs, *sc)
    assert got["center"] == c
    assert got["row_sums"].tolist() == sums.tolist()
    assert got["scores"].tolist() == [s for s, _ in aligned]
    assert got["cigars"] == [oracle.rle(ops) for _, ops in aligned]
    assert got["rows"] == rows
    return got


def test_hand_worked_family(ctx):
    d = {}
    for ln in open(os.path.join(GOLDEN, "center_star_hand.txt")):
        if not ln.startswith("#") and ":" in ln:
            k, _, v = ln.partition(":")
            d[k.strip()] = v.split()
    got = _check(ctx, [codes(s) for s in d["seqs"]])
    assert got["rows"] == d["rows"]


@pytest.mark.parametrize("case", ["one", "two", "empty", "ties", "mixed"])
def test_edge_families(ctx, case):
    rs = seqgen.Stream(31)
    if case == "one":
        seqs = [rs.bases(300)]
    elif case == "two":
        seqs = [rs.bases(200), rs.bases(260)]
    elif case == "empty":
        seqs = [np.zeros(0, np.uint8), rs.bases(40), np.zeros(0, np.uint8), rs.bases(1)]
    elif case == "ties":
        s = rs.bases(120)
        seqs = [s, s.copy(), s.copy()]
    else:
        seqs = seqgen.all_vs_all_family(11, nseq=37, root_len=700, lmin=1, lmax=700)
    _check(ctx, seqs)


@pytest.mark.parametrize("sc", [(2, -1, -2), (1, -3, -1)])
def test_other_scorings(ctx, sc):
    _check(ctx, seqgen.all_vs_all_family(12, nseq=24, root_len=400, lmin=100, lmax=400), sc)


def test_full_family_device_buffers(ctx):
    """The 512-sequence family (130,816 scored pairs, 512 alignments) in the
    benchmark's launch configuration (device buffers, graph-captured scoring
    stage, rows written on the device), against the oracle."""
    import torch
    import paper_2412_21103_gb300 as nw
    seqs = seqgen.all_vs_all_family(1003)
    pool, off, lens = nw.pool_of(seqs)
    n = len(seqs)
    coff = nw._center_cigar_offsets(lens)
    dpool = torch.from_numpy(pool).cuda()
    sums = torch.zeros(n, dtype=torch.int64, device="cuda")
    scores = torch.zeros(n, dtype=torch.int32, device="cuda")
    cpool = torch.zeros(int(coff[-1]), dtype=torch.uint8, device="cuda")
    clen = torch.zeros(n, dtype=torch.int64, device="cuda")
    # first the column count (no rows), then the rows at that stride; the
    # second call replays the captured scoring stage
    center, cols, ok = nw.nw_center_star(ctx, dpool, off, lens, (1, -1, -1), nw.NW_GRAPH, sums, scores, cpool,
                                         coff, clen, None, 0)
    assert ok
    ld = cols + 1
    msa = torch.zeros(n * ld, dtype=torch.uint8, device="cuda")
    center, cols, ok = nw.nw_center_star(ctx, dpool, off, lens, (1, -1, -1), nw.NW_GRAPH, sums, scores, cpool,
                                         coff, clen, msa, ld)
    assert ok
    ctx.sync()
    c, want_sums, aligned, rows = cs.center_star(seqs)
    assert center == c and cols == len(rows[0])
    assert sums.cpu().tolist() == want_sums.tolist()
    assert scores.cpu().tolist() == [s for s, _ in aligned]
    cp, cl = cpool.cpu().numpy(), clen.cpu().numpy()
    for k, (_, ops) in enumerate(aligned):
        assert cp[int(coff[k]): int(coff[k]) + int(cl[k])].tobytes().decode() == oracle.rle(ops), k
    m = msa.cpu().numpy().reshape(n, ld)
    for k in range(n):
        assert m[k, :cols].tobytes().decode() == rows[k], k
        assert m[k, cols] == 0


def test_short_row_stride_reports_the_column_count(ctx):
    import torch
    import paper_2412_21103_gb300 as nw
    seqs = seqgen.all_vs_all_family(13, nseq=8, root_len=300, lmin=200, lmax=300)
    pool, off, lens = nw.pool_of(seqs)
    n = len(seqs)
    coff = nw._center_cigar_offsets(lens)
    dpool = torch.from_numpy(pool).cuda()
    scores = torch.zeros(n, dtype=torch.int32, device="cuda")
    cpool = torch.zeros(int(coff[-1]), dtype=torch.uint8, device="cuda")
    clen = torch.zeros(n, dtype=torch.int64, device="cuda")
    msa = torch.zeros(n * 16, dtype=torch.uint8, device="cuda")
    center, cols, ok = nw.nw_center_star(ctx, dpool, off, lens, (1, -1, -1), 0, None, scores, cpool, coff, clen,
                                         msa, 16)
    assert not ok and cols > 16
    # the CIGARs are written: the merge alone completes the rows
    ld = cols + 1
    msa = torch.zeros(n * ld, dtype=torch.uint8, device="cuda")
    assert nw.nw_msa_merge(ctx, dpool, off, lens, center, cpool, coff, clen, msa, ld) == cols
    rows = cs.center_star(seqs)[3]
    m = msa.cpu().numpy().reshape(n, ld)
    assert [m[k, :cols].tobytes().decode() for k in range(n)] == rows


def test_merge_rejects_a_cigar_that_does_not_fit_its_sequences(ctx):
    """A CIGAR that consumes more bases than its sequence has is caught by
    the merge kernel's own check (NW_ERR_ARG), and no row is written."""
    import paper_2412_21103_gb300 as nw
    seqs = [codes("ACGT"), codes("ACT")]
    pool, off, lens = nw.pool_of(seqs)
    cig = b"4=\x00" + b"5=\x00"                 # the second consumes 5 bases of a 3-base sequence
    cpool = np.frombuffer(cig, np.uint8).copy()
    coff = np.array([0, 3], np.uint64)
    clen = np.array([2, 2], np.uint64)
    msa = np.zeros(2 * 8, np.uint8)
    with pytest.raises(nw.NWError) as e:
        nw.nw_msa_merge(ctx, pool, off, lens, 0, cpool, coff, clen, msa, 8)
    assert e.value.status == nw.NW_ERR_ARG
    assert not msa.any()
    ctx.sync()
