"""Host arithmetic of the CUDA path that needs no GPU, against the oracle:
the banded certificate's exit bound -- a path that leaves the band of
half-width w makes at least G gap moves, so it scores at most
match*floor((m+n-G)/2) + gap*(m+n-2*floor((m+n-G)/2)) -- the certificate
and the next round's width built on it, the learned start width and the
straggler rule.  The oracle's `exit_bound` is pinned by brute force over
every path in test_oracle_pins."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def nw():
    import paper_2412_21103_gb300 as nw
    nw.load()
    return nw


def test_exit_bound_matches_the_oracle(nw):
    rng = np.random.default_rng(17)
    cases = [(0, 0, 0), (0, 5, 1), (7, 0, 3), (1, 1, 0), (10, 10, 20), (50, 3, 2), (3, 50, 2)]
    cases += [(int(rng.integers(0, 3000)), int(rng.integers(0, 3000)), int(rng.integers(0, 400))) for _ in range(3000)]
    scorings = [(1, -1, -1), (2, -1, -3), (3, -2, -1), (1, 0, 0), (0, -1, -1)]
    for m, n, w in cases:
        for sc in scorings:
            got = nw.nw_band_exit_bound(m, n, w, sc)
            want = oracle.exit_bound(m, n, w, sc[0], sc[2])
            assert got == want, (m, n, w, sc, got, want)


def test_exit_bound_large_sizes_match(nw):
    for m, n, w in [(20000, 20000, 64), (32768, 32741, 1000), (50000, 2000, 10), (2000, 50000, 10),
                    (1 << 30, (1 << 30) + 7, 5000)]:
        assert nw.nw_band_exit_bound(m, n, w) == oracle.exit_bound(m, n, w)


def test_exit_bound_rejects_bad_arguments(nw):
    with pytest.raises(nw.NWError):
        nw.nw_band_exit_bound(1 << 31, 10, 1)
    with pytest.raises(nw.NWError):
        nw.nw_band_exit_bound(10, 10, 1, (1, -1, 1))  # positive gap


def test_binding_cigar_offsets_follow_the_library_bound(nw):
    rng = np.random.default_rng(3)
    a = rng.integers(0, 50000, 500).astype(np.uint32)
    b = rng.integers(0, 50000, 500).astype(np.uint32)
    off = nw._cigar_offsets(a, b)
    caps = [nw.nw_cigar_bound(int(x), int(y)) for x, y in zip(a, b)]
    assert off[0] == 0 and np.array_equal(np.diff(off), np.array(caps, np.uint64))


def test_binding_cigar_decoding(nw):
    pool = np.zeros(32, np.uint8)
    pool[0:4] = np.frombuffer(b"3=1X", np.uint8)
    pool[20:22] = np.frombuffer(b"5D", np.uint8)
    c = nw._cigars(None, pool, np.array([0, 10, 20], np.uint64), np.array([4, 0, 2], np.uint64), 3)
    assert c == ["3=1X", "", "5D"] and ["3=1X", "", "5D"] == c and c != ["3=1X", "", "5E"] and c != ["3=1X"]
    assert len(c) == 3 and c[0] == "3=1X" and c[-1] == "5D" and c[1:] == ["", "5D"] and list(c) == c.tolist()
    assert c.nbytes() == 6
    with pytest.raises(IndexError):
        c[3]


def test_host_cigar_buffer_returns_to_the_context(nw):
    """The host CIGAR buffer a call fills is lent to its Cigars view and
    comes back to the context when the view is released, so a later call
    reuses it; a view still alive keeps its bytes."""
    class Ctx:
        handle = 1
    ctx = Ctx()
    buf = nw._host_cigar_pool(ctx, 100)
    buf[:2] = np.frombuffer(b"7=", np.uint8)
    c = nw._cigars(ctx, buf, np.array([0], np.uint64), np.array([2], np.uint64), 1)
    other = nw._host_cigar_pool(ctx, 50)          # the first view is alive: a new buffer
    assert other is not buf
    other[:2] = np.frombuffer(b"9I", np.uint8)
    assert c[0] == "7=" and nw._cigars(ctx, other, [0], [2], 1)[0] == "9I"
    del c
    assert nw._host_cigar_pool(ctx, 80) is buf    # released: the larger buffer comes back


def test_certificate_and_next_width_match_the_oracle(nw):
    """The banded rounds' certificate and next-width rule (host code of the
    library) against the oracle's plain definitions."""
    rng = np.random.default_rng(23)
    for _ in range(1500):
        m, n = int(rng.integers(1, 2500)), int(rng.integers(1, 2500))
        w = int(rng.integers(0, 300))
        sc = [(1, -1, -1), (2, -1, -3), (1, 0, 0)][int(rng.integers(0, 3))]
        U = oracle.exit_bound(m, n, w, sc[0], sc[2])
        base = U if U is not None else sc[0] * min(m, n)
        sb = int(base + rng.integers(-400, 3))
        for want in (False, True):
            assert nw.nw_band_certifies(m, n, w, sb, want, sc) == oracle.certifies(m, n, w, sb, want, sc[0], sc[2])
            assert nw.nw_band_next_width(m, n, w, sb, want, sc) == oracle.next_width(m, n, w, sb, want, sc[0], sc[2])


def test_start_width_matches_the_oracle(nw):
    from oracle import band_model as bm
    rng = np.random.default_rng(31)
    ys = list(rng.normal(4.0, 2.0, 3000)) + [-50.0, -3.0, 0.0, 2.0794415, 9.9, 15.0, 30.0, 80.0]
    for y in ys:
        m, n = int(rng.integers(1, 60000)), int(rng.integers(1, 60000))
        y32 = float(np.float32(y))
        assert nw.nw_band_start_width(y32, m, n) == bm.start_width(y32, m, n), (y32, m, n)


def test_straggler_rule_properties(nw):
    """The batched paths' straggler rule (host code): a balanced batch stays
    on the batched kernel, a pair that would hold one warp far longer than
    the batch goes to the single-pair kernel, pairs under 1e7 cells never
    move, and what moves is always the costliest prefix."""
    assert nw.nw_route_stragglers(np.full(10000, 1e6), np.full(10000, 1e6)) == []
    w = np.concatenate([[1e6] * 500, [1e9], [1e6] * 500])
    assert nw.nw_route_stragglers(w, w) == [500]
    assert nw.nw_route_stragglers([5e6], [5e6]) == []
    assert nw.nw_route_stragglers([], []) == []
    rng = np.random.default_rng(41)
    for _ in range(200):
        n = int(rng.integers(1, 3000))
        wc = np.exp(rng.uniform(np.log(1e5), np.log(rng.choice([1e7, 1e9, 1e10])), n))
        fc = wc * rng.uniform(1.0, 3.0, n)
        got = nw.nw_route_stragglers(wc, fc)
        order = list(np.argsort(-wc, kind="stable"))
        assert got == [int(k) for k in order[: len(got)]]
        assert all(fc[k] >= 1e7 for k in got)
