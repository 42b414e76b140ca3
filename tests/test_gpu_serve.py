"""The continuous-batching server (a10): requests submitted while others
are running are admitted as workers and traceback memory free up, and every
result equals the one the same pair gets alone (nw_align), and the oracle's."""
import time

import numpy as np
import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu


def _requests(seed, count):
    rs = seqgen.Stream(seed)
    out = []
    for k in range(count):
        m = int(np.exp(rs.uniform(1)[0] * np.log(6000)))
        if k % 17 == 0:
            m = 0 if k % 34 == 0 else 1
        p = seqgen.long_mutated_pair(seed * 1000 + k, m=max(m, 1), p_sub=0.03 + 0.07 * (k % 4))
        a = p.a[:m]
        b = p.b if k % 13 else p.b[: max(0, p.b.size // 2)]
        out.append((a, b, k % 2 == 1))
    return out


def test_server_mix_equals_alone_and_oracle():
    import torch
    import paper_2412_21103_gb300 as nw
    ctx = nw.Context(0, torch.cuda.current_stream())
    # a small traceback budget so admission has to wait for memory
    srv = nw.Server(ctx, workers=3, max_batch=24, trace_budget=24 << 20, flags=nw.NW_LEARNED_BAND)
    reqs = _requests(3, 150)
    tickets = {}
    results = {}
    for wave in range(3):
        for k in range(wave * 50, wave * 50 + 50):
            a, b, cig = reqs[k]
            t = srv.submit(nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, cig)
            tickets[t] = k
        time.sleep(0.05)
        for t, st, sc, cg, lat in srv.poll():
            results[tickets[t]] = (st, sc, cg, lat)
    assert srv.drain(120.0)
    for t, st, sc, cg, lat in srv.poll():
        results[tickets[t]] = (st, sc, cg, lat)
    stats = srv.stats()
    assert stats["completed"] == 150 and stats["reserved"] == 0 and stats["batches"] > 3
    assert len(results) == 150
    for k, (a, b, cig) in enumerate(reqs):
        st, sc, cg, lat = results[k]
        assert st == nw.NW_OK and lat >= 0
        alone = nw.nw_align(ctx, nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, (1, -1, -1),
                            nw.NW_CIGAR if cig else 0)
        assert sc == alone[0], k
        if cig:
            assert cg == alone[1], k
        else:
            assert cg is None
    for k in range(0, 150, 7):
        a, b, cig = reqs[k]
        s, ops = oracle.align(a, b)
        assert results[k][1] == s
        if cig:
            assert results[k][2] == oracle.rle(ops)
    srv.close()
    ctx.close()


def test_server_submit_many_and_budget_admission():
    import torch
    import paper_2412_21103_gb300 as nw
    ctx = nw.Context(0, torch.cuda.current_stream())
    srv = nw.Server(ctx, workers=2, max_batch=8, trace_budget=1 << 20)
    reqs = _requests(5, 40)
    seqs = []
    for a, b, _ in reqs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    tickets = srv.submit_many(pool, off[0::2], lens[0::2], off[1::2], lens[1::2], [c for _, _, c in reqs])
    assert srv.drain(120.0)
    # a CIGAR buffer smaller than one CIGAR: poll grows it on NW_ERR_CIGAR_TRUNC, and poll_all
    # keeps polling while one poll returns only the part that fits
    srv._cbuf = np.zeros(16, np.uint8)
    got = {t: (sc, cg) for t, st, sc, cg, lat in srv.poll_all()}
    assert len(got) == len(tickets)
    for k, t in enumerate(tickets):
        a, b, cig = reqs[k]
        s, ops = oracle.align(a, b)
        assert got[int(t)][0] == s
        if cig:
            assert got[int(t)][1] == oracle.rle(ops)
    srv.close()
    ctx.close()


def test_device_queue_word_after_drain():
    """The queue's consumer state lives on the device: after a drain its word
    says every submitted request was admitted and no traceback bytes are
    reserved."""
    import torch
    import paper_2412_21103_gb300 as nw
    ctx = nw.Context(0, torch.cuda.current_stream())
    srv = nw.Server(ctx, workers=2, max_batch=16, trace_budget=4 << 20)
    reqs = _requests(7, 30)
    for a, b, cig in reqs:
        srv.submit(nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, cig)
    assert srv.drain(120.0)
    assert srv.queue_state() == {"admitted": 30, "reserved": 0}
    assert len(srv.poll_all()) == 30
    srv.close()
    ctx.close()


def test_small_arena_and_ring_wrap_and_wait():
    """An arena of 12 KiB and a ring of 8 slots: submissions wait for
    completions, placements wrap around both, and every result still equals
    the oracle's."""
    import torch
    import paper_2412_21103_gb300 as nw
    ctx = nw.Context(0, torch.cuda.current_stream())
    srv = nw.Server(ctx, workers=2, max_batch=3, trace_budget=64 << 20, queue_bytes=12 << 10, queue_slots=8)
    reqs = _requests(11, 60)
    seqs = []
    for a, b, _ in reqs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    tickets = srv.submit_many(pool, off[0::2], lens[0::2], off[1::2], lens[1::2], [c for _, _, c in reqs])
    assert srv.drain(120.0)
    got = {t: (st, sc, cg) for t, st, sc, cg, lat in srv.poll_all()}
    assert len(got) == 60
    for k, t in enumerate(tickets):
        a, b, cig = reqs[k]
        st, sc, cg = got[int(t)]
        assert st == nw.NW_OK
        s, ops = oracle.align(a, b)
        assert sc == s, k
        if cig:
            assert cg == oracle.rle(ops), k
    assert srv.queue_state() == {"admitted": 60, "reserved": 0}
    # a request larger than the arena is refused
    big = np.zeros(40000, np.uint8)
    with pytest.raises(nw.NWError):
        srv.submit(nw.pack_codes(big), big.size, nw.pack_codes(big), big.size, False)
    srv.close()
    ctx.close()


def test_failed_batch_reports_its_status_and_message():
    """A batch the worker cannot run (its context's memory budget is far too
    small for the batch's scratch: a failure made on the host) completes
    every request of it with the batch's status, and the server keeps that
    status's text and the context's message."""
    import torch
    import paper_2412_21103_gb300 as nw
    ctx = nw.Context(0, torch.cuda.current_stream(), mem_budget=64 << 10)  # 16 KiB per worker
    srv = nw.Server(ctx, workers=3, max_batch=8, trace_budget=1 << 30)
    assert srv.last_message() == ""
    rs = seqgen.Stream(41)
    tickets = [srv.submit(nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, True)
               for a, b in ((rs.bases(3000), rs.bases(3100)), (rs.bases(2000), rs.bases(1900)))]
    assert srv.drain(60.0)
    res = {t: st for t, st, sc, cg, lat in srv.poll()}
    st = {res[t] for t in tickets}
    assert len(res) == 2 and nw.NW_OK not in st
    msg = srv.last_message()
    assert any(msg.startswith(nw.load().nw_strerror(x).decode()) for x in st) and "requests)" in msg
    srv.close()
    ctx.close()
