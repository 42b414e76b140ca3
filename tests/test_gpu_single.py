"""GPU parity of the single-pair path (pack, fill, traceback, CIGAR) against
the CPU oracle, element by element: scores and CIGAR strings bit-exact."""
import numpy as np
import pytest

import oracle
import seqgen
from helpers import consumed, parse_cigar, rescore

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_2412_21103_gb300 as nw
    c = nw.Context(0, torch.cuda.current_stream())
    yield c
    c.close()


def _align(ctx, a, b, sc=(1, -1, -1), cigar=True):
    import paper_2412_21103_gb300 as nw
    return nw.nw_align(ctx, nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, sc,
                       nw.NW_CIGAR if cigar else 0)


def _check(ctx, a, b, sc=(1, -1, -1)):
    want_s, want_ops = oracle.align(a, b, *sc)
    s, cig = _align(ctx, a, b, sc)
    assert s == want_s
    assert cig == oracle.rle(want_ops)
    s2, _ = _align(ctx, a, b, sc, cigar=False)
    assert s2 == want_s


def test_config1_random_1000(ctx):
    p = seqgen.random_pair(1001, 1000, 1000)
    _check(ctx, p.a, p.b)


EDGE = [1, 2, 3, 31, 32, 33, 127, 128, 129, 255, 256, 257, 511, 513, 1023, 1025]


@pytest.mark.parametrize("m", EDGE)
def test_edge_lengths_rows(ctx, m):
    rs = seqgen.Stream(m)
    for n in (1, 5, 32, 33, 100):
        _check(ctx, rs.bases(m), rs.bases(n))


@pytest.mark.parametrize("n", EDGE)
def test_edge_lengths_cols(ctx, n):
    rs = seqgen.Stream(7000 + n)
    for m in (1, 31, 130, 700):
        _check(ctx, rs.bases(m), rs.bases(n))


@pytest.mark.parametrize("sc", [(1, -1, -1), (2, -1, -2), (0, -1, -1), (1, 0, 0), (3, -2, -1), (1, -3, -1),
                                (5, 4, -3), (40, -40, -40)])
def test_scoring_schemes(ctx, sc):
    rs = seqgen.Stream(sum(sc) + 50)
    for _ in range(3):
        m, n = (int(x) for x in rs.integers(1, 900, 2))
        _check(ctx, rs.bases(m), rs.bases(n), sc)


def test_empty_sides(ctx):
    z = np.zeros(0, np.uint8)
    b = seqgen.Stream(3).bases(17)
    assert _align(ctx, z, b) == (-17, "17D")
    assert _align(ctx, b, z) == (-17, "17I")
    assert _align(ctx, z, z) == (0, "")


def test_identity_and_mutated(ctx):
    p = seqgen.long_mutated_pair(77, m=5000)
    _check(ctx, p.a, p.b)
    s, cig = _align(ctx, p.a, p.a)
    assert (s, cig) == (5000, "5000=")


@pytest.mark.parametrize("m,n", [(4096 + 17, 300), (300, 9000), (20000, 64), (64, 20000)])
def test_ragged_many_stripes(ctx, m, n):
    rs = seqgen.Stream(m * 7 + n)
    _check(ctx, rs.bases(m), rs.bases(n))


def test_wide_rows_path(ctx):
    """Enough rows that the fill uses 16 rows per lane."""
    p = seqgen.long_mutated_pair(91, m=160000)
    b = p.b[:900]
    _check(ctx, p.a, b)


def test_config2_full_size(ctx):
    """The 32,768-base mutated pair: full score and CIGAR bit-exact."""
    p = seqgen.long_mutated_pair(1002)
    want_s, want_ops = oracle.align(p.a, p.b)
    s, cig = _align(ctx, p.a, p.b)
    assert s == want_s
    assert cig == oracle.rle(want_ops)
    ops = parse_cigar(cig)
    assert consumed(ops) == (p.a.size, p.b.size)
    assert rescore(ops, p.a, p.b, 1, -1, -1) == s


def test_device_io_and_device_pack(ctx):
    import torch
    import paper_2412_21103_gb300 as nw
    p = seqgen.random_pair(5, 777, 901)
    dev = torch.device("cuda")
    asc = torch.tensor(np.frombuffer(seqgen.to_ascii(p.a).lower().encode(), np.uint8), device=dev)
    bsc = torch.tensor(np.frombuffer(seqgen.to_ascii(p.b).encode(), np.uint8), device=dev)
    a2b = torch.zeros((p.a.size + 3) // 4, dtype=torch.uint8, device=dev)
    b2b = torch.zeros((p.b.size + 3) // 4, dtype=torch.uint8, device=dev)
    nw.nw_pack_device(ctx, asc, p.a.size, a2b)
    nw.nw_pack_device(ctx, bsc, p.b.size, b2b)
    ctx.sync()
    assert a2b.cpu().numpy().tolist() == nw.pack_codes(p.a).tolist()
    score = torch.zeros(1, dtype=torch.int32, device=dev)
    cig = torch.zeros(nw.nw_cigar_bound(p.a.size, p.b.size), dtype=torch.uint8, device=dev)
    clen = torch.zeros(1, dtype=torch.int64, device=dev)
    nw.nw_align(ctx, a2b, p.a.size, b2b, p.b.size, (1, -1, -1), nw.NW_CIGAR, score, cig, clen)
    ctx.sync()
    want_s, want_ops = oracle.align(p.a, p.b)
    assert int(score.item()) == want_s
    assert bytes(cig[: int(clen.item())].cpu().numpy()).decode() == oracle.rle(want_ops)


def test_device_pack_bad_base(ctx):
    import torch
    import paper_2412_21103_gb300 as nw
    asc = torch.tensor(np.frombuffer(b"ACGTNACG", np.uint8), device="cuda")
    out = torch.zeros(2, dtype=torch.uint8, device="cuda")
    nw.nw_pack_device(ctx, asc, 8, out)
    with pytest.raises(nw.NWError) as e:
        ctx.sync()
    assert e.value.status == nw.NW_ERR_BAD_BASE
    ctx.sync()  # the error word was cleared


def test_bad_arguments_are_rejected(ctx):
    import paper_2412_21103_gb300 as nw
    a = nw.pack_codes(np.zeros(10, np.uint8))
    with pytest.raises(nw.NWError) as e:
        nw.nw_align(ctx, a, 10, a, 10, (1, -1, 1), 0)
    assert e.value.status == nw.NW_ERR_ARG
    with pytest.raises(nw.NWError):
        nw.nw_align(ctx, a, 10, a, 10, (-1, 1, -1), 0)


def test_cigar_m_flag(ctx):
    import paper_2412_21103_gb300 as nw
    p = seqgen.random_pair(9, 200, 180)
    _, ops = oracle.align(p.a, p.b)
    s, cig = nw.nw_align(ctx, nw.pack_codes(p.a), 200, nw.pack_codes(p.b), 180, (1, -1, -1),
                         nw.NW_CIGAR | nw.NW_CIGAR_M)
    assert cig == oracle.rle(ops.replace("=", "M").replace("X", "M"))


@pytest.mark.parametrize("R,C", [(2, 2), (2, 4), (2, 8), (4, 2), (4, 4), (8, 2)])
@pytest.mark.parametrize("nwarps", [1, 2, 4, 8])
def test_pair_kernel_shapes(ctx, R, C, nwarps, monkeypatch):
    """Every block shape (rows per lane x columns per step) and warps-per-CTA
    count of the single-pair fill: several CTA stripes (global handoffs),
    several warps per CTA (shared memory handoffs), ragged last stripe, rows
    whose last pointer word is short."""
    monkeypatch.setenv("NW_PAIR_R", str(R))
    monkeypatch.setenv("NW_PAIR_C", str(C))
    monkeypatch.setenv("NW_PAIR_WARPS", str(nwarps))
    for seed, m, n in [(1, 32 * R * nwarps * 3 + 17, 700), (2, 5000, 301), (3, 64, 2000), (4, 2 * 32 * R + 1, 31),
                       (5, 300, 16 // R * 7 + 1)]:
        p = seqgen.long_mutated_pair(seed, m=m)
        _check(ctx, p.a, p.b[:n] if n < p.b.size else p.b)


@pytest.mark.parametrize("cls", [2, 4, 8])
@pytest.mark.parametrize("R,C,nwarps", [(8, 2, 4), (4, 2, 2), (4, 4, 1)])
def test_pair_kernel_cluster_handoffs(ctx, cls, R, C, nwarps, monkeypatch):
    """Row groups handed over through distributed shared memory inside a
    thread-block cluster (opt-in path): exact, including partial clusters
    (groups not a multiple of the cluster size) and several clusters."""
    monkeypatch.setenv("NW_PAIR_CLUSTER", str(cls))
    monkeypatch.setenv("NW_PAIR_R", str(R))
    monkeypatch.setenv("NW_PAIR_C", str(C))
    monkeypatch.setenv("NW_PAIR_WARPS", str(nwarps))
    group_rows = 32 * R * nwarps
    cases = [(1, 2), (2, cls + 1)] + ([(3, 3 * cls)] if group_rows * 3 * cls <= 6200 else [])
    for seed, groups in cases:
        p = seqgen.long_mutated_pair(900 + seed, m=group_rows * groups - 13)
        _check(ctx, p.a, p.b)
