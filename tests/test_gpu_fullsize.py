"""Full-size parity of the certified learned band and of the server, in the
launch configuration the benchmark times.

Config 4: all 20,000 pairs of 2-20 kb through nw_align_batch(NW_CIGAR |
NW_LEARNED_BAND) on device buffers, after training the band network on the
GPU from the committed oracle labels.  Every score and every CIGAR string
(byte for byte) equals the plain full-grid batch's; at least 400 pairs equal
the oracle's score and CIGAR: every pair the first banded round certified
at the narrowest certified half-width of that round (where an unsound
certificate would show first), the longest pairs, the largest length
differences and a seeded random sample.

Config 5: 2,000 requests of the serving stream (lengths 50-50,000, half with
CIGAR) through the server with the learned band: every score equals the
oracle's, every CIGAR of a request up to 3e7 cells equals the oracle's, the
rest equal the single-pair path's."""
import os

import numpy as np
import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu

LABELS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "band_labels_seed9004.npz")
SC = (1, -1, -1)


def _pool(pairs):
    import paper_2412_21103_gb300 as nw
    seqs = []
    for a, b in pairs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    return pool, off[0::2], lens[0::2], off[1::2], lens[1::2]


@pytest.fixture(scope="module")
def trained_ctx():
    """A context whose band network was trained on the GPU (60 epochs of
    batches of 512, Adam at 2e-3: the benchmark's schedule)."""
    import torch
    import paper_2412_21103_gb300 as nw
    ctx = nw.Context(0, torch.cuda.current_stream())
    ctx.set_autotune(True)
    lab = np.load(LABELS)
    count = int(lab["label"].size)
    pairs = seqgen.band_pairs(int(lab["seed"]), npairs=count)
    pool, ao, al, bo, bl = _pool([(p.a, p.b) for p in pairs])
    feat = nw.nw_band_features(ctx, torch.from_numpy(pool).cuda(), ao, al, bo, bl)
    target = torch.from_numpy(np.log(np.maximum(lab["label"], 1)).astype(np.float32)).cuda()
    nw.nw_band_model_init(ctx, 0)
    g = torch.Generator().manual_seed(0)
    for _ in range(60):
        perm = torch.randperm(count, generator=g).cuda()
        for k in range(0, count - 511, 512):
            idx = perm[k:k + 512]
            nw.nw_band_model_train_step(ctx, feat[idx].contiguous(), target[idx].contiguous(), 2e-3)
    ctx.sync()
    yield ctx
    ctx.close()


def test_config4_full_size_learned_band(trained_ctx):
    import torch
    import paper_2412_21103_gb300 as nw
    ctx = trained_ctx
    pairs = seqgen.band_pairs(1004, npairs=20000)
    pool, ao, al, bo, bl = _pool([(p.a, p.b) for p in pairs])
    dpool = torch.from_numpy(pool).cuda()
    coff = nw._cigar_offsets(al, bl)
    n = len(pairs)

    def run(flags):
        scores = torch.zeros(n, dtype=torch.int32, device="cuda")
        cpool = torch.zeros(int(coff[-1]), dtype=torch.uint8, device="cuda")
        clen = torch.zeros(n, dtype=torch.int64, device="cuda")
        nw.nw_align_batch(ctx, dpool, ao, al, bo, bl, SC, flags, scores, cpool, coff, clen)
        ctx.sync()
        return scores.cpu().numpy(), cpool, clen.cpu().numpy()

    s_band, c_band, l_band = run(nw.NW_CIGAR | nw.NW_LEARNED_BAND)
    st = nw.nw_ctx_band_stats(ctx)
    assert st["certified_round"][0] > 0 and st["certified_round"][1] > 0  # both rounds certify some pairs
    outcome = nw.nw_ctx_band_outcome(ctx)
    s_full, c_full, l_full = run(nw.NW_CIGAR)
    assert np.array_equal(s_band, s_full)
    assert np.array_equal(l_band, l_full)
    cb, cf = c_band.cpu().numpy(), c_full.cpu().numpy()
    bad = [k for k in range(n)
           if cb[int(coff[k]): int(coff[k]) + int(l_band[k])].tobytes()
           != cf[int(coff[k]): int(coff[k]) + int(l_full[k])].tobytes()]
    assert not bad, f"{len(bad)} CIGAR strings differ from the plain batch, first {bad[:5]}"

    # oracle sample: the narrowest round-1 certificates, extremes, random
    r1 = np.nonzero(outcome["round"] == 1)[0]
    assert r1.size > 0
    wmin = int(outcome["cert_width"][r1].min())
    narrowest = r1[outcome["cert_width"][r1] == wmin]
    longest = np.argsort(-(al.astype(np.int64) * bl.astype(np.int64)))[:16]
    skewed = np.argsort(-np.abs(bl.astype(np.int64) - al.astype(np.int64)))[:16]
    sample = set(int(k) for k in np.concatenate([narrowest, longest, skewed]))
    rs = seqgen.Stream(4242)
    for k in rs.integers(0, n - 1, 4 * n):
        if len(sample) >= 400:
            break
        sample.add(int(k))
    sample = sorted(sample)
    assert len(sample) >= 400
    want = oracle.align_many([(pairs[k].a, pairs[k].b) for k in sample])
    for k, (s, ops) in zip(sample, want):
        assert int(s_band[k]) == s, k
        got = cb[int(coff[k]): int(coff[k]) + int(l_band[k])].tobytes().decode()
        assert got == oracle.rle(ops), k
    print(f"config 4: {narrowest.size} pairs certified in round 1 at half-width {wmin}; "
          f"{len(sample)} pairs checked against the oracle")


def test_config5_two_thousand_requests(trained_ctx):
    import paper_2412_21103_gb300 as nw
    reqs = list(seqgen.serving_stream(1005, rate=50000.0, limit=2000))
    assert len(reqs) == 2000
    srv = nw.Server(trained_ctx, workers=8, max_batch=64, trace_budget=64 << 30, flags=nw.NW_LEARNED_BAND)
    pool, ao, al, bo, bl = _pool([(r.pair.a, r.pair.b) for r in reqs])
    tickets = srv.submit_many(pool, ao, al, bo, bl, [r.want_cigar for r in reqs])
    assert srv.drain(300.0), srv.stats()
    got = {t: (st, sc, cg) for t, st, sc, cg, lat in srv.poll_all()}
    failure = srv.last_message()
    srv.close()
    assert len(got) == 2000, len(got)
    bad = {st for st, _, _ in got.values() if st != nw.NW_OK}
    assert not bad, (bad, failure)
    res = [got[int(t)] for t in tickets]
    want = oracle.score_many([(r.pair.a, r.pair.b) for r in reqs])
    wrong = [k for k in range(len(reqs)) if res[k][1] != want[k]]
    assert not wrong, [(k, reqs[k].pair.a.size, reqs[k].pair.b.size, res[k][1], want[k]) for k in wrong[:10]]
    small = [k for k, r in enumerate(reqs) if r.want_cigar and r.pair.a.size * r.pair.b.size <= 3e7]
    big = [k for k, r in enumerate(reqs) if r.want_cigar and r.pair.a.size * r.pair.b.size > 3e7]
    for k, (s, ops) in zip(small, oracle.align_many([(reqs[k].pair.a, reqs[k].pair.b) for k in small])):
        assert res[k][2] == oracle.rle(ops), k
    for k in big[:40]:
        a, b = reqs[k].pair.a, reqs[k].pair.b
        s, cig = nw.nw_align(trained_ctx, nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, SC, nw.NW_CIGAR)
        assert res[k][1] == s and res[k][2] == cig, k
    for k, r in enumerate(reqs):
        assert (res[k][2] is None) == (not r.want_cigar)
