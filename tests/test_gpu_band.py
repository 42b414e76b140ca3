"""GPU parity of the certified band (a8) and the learned-band pieces (a9):
banded scores bit-exact against the oracle's banded DP, certified results
bit-exact against full NW, features and network against the CPU reference."""
import numpy as np
import pytest

import oracle
import seqgen
from oracle import band_model as bm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_2412_21103_gb300 as nw
    c = nw.Context(0, torch.cuda.current_stream())
    yield c
    c.close()


def _pool(pairs):
    import paper_2412_21103_gb300 as nw
    seqs = []
    for a, b in pairs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    return pool, off[0::2], lens[0::2], off[1::2], lens[1::2]


def _band_pairs(seed, count, lmax=1500):
    rs = seqgen.Stream(seed)
    out = []
    for k in range(count):
        m = int(rs.integers(1, lmax, 1)[0])
        p = seqgen.long_mutated_pair(seed * 100 + k, m=max(m, 2), p_sub=0.05 + 0.1 * (k % 3),
                                     p_indel=0.01 * (k % 4))
        b = p.b
        if k % 5 == 0:
            b = b[: max(1, b.size - int(rs.integers(0, 200, 1)[0]))]   # length difference
        out.append((p.a, b))
    return out


@pytest.mark.parametrize("w", [0, 1, 3, 17, 64, 200])
def test_raw_banded_scores_equal_oracle_banded_dp(ctx, w):
    import paper_2412_21103_gb300 as nw
    pairs = _band_pairs(40 + w, 24, lmax=700)
    pool, ao, al, bo, bl = _pool(pairs)
    ws = np.full(len(pairs), w, np.uint32)
    got, _ = nw.nw_align_batch_banded(ctx, pool, ao, al, bo, bl, ws, (1, -1, -1), nw.NW_BAND_RAW)
    for k, (a, b) in enumerate(pairs):
        sb, _ = oracle.banded(a, b, w)
        assert got[k] == sb, (k, a.size, b.size)


@pytest.mark.parametrize("sc", [(1, -1, -1), (2, -1, -2), (3, -3, -1)])
def test_certified_band_scores_and_cigars_exact(ctx, sc):
    import paper_2412_21103_gb300 as nw
    pairs = _band_pairs(7 + sc[0], 40)
    pool, ao, al, bo, bl = _pool(pairs)
    ws = np.array([[8, 16, 40, 2, 100][k % 5] for k in range(len(pairs))], np.uint32)
    scores, cigars = nw.nw_align_batch_banded(ctx, pool, ao, al, bo, bl, ws, sc, nw.NW_CIGAR)
    want = oracle.align_many(pairs, *sc)
    for k, (s, ops) in enumerate(want):
        assert scores[k] == s, k
        assert cigars[k] == oracle.rle(ops), k
    s_only, _ = nw.nw_align_batch_banded(ctx, pool, ao, al, bo, bl, ws, sc, 0)
    assert s_only.tolist() == [s for s, _ in want]


BAND_R = 16  # rows per lane of the certified band's kernel (stripes of 32 * BAND_R rows)


def _region_score(a, b, w, SH=32 * BAND_R):
    """The banded kernel's cell set: per stripe of SH rows, the columns from
    the band's left edge at its top row to its right edge at its bottom row
    (the stripe rectangle); boundary cells only where the band reaches them."""
    m, n = a.size, b.size
    lo, hi = oracle.band_limits(m, n, w)
    i = np.arange(1, m + 1)
    s = (i - 1) // SH
    cbeg = np.maximum(0, s * SH + lo)
    cend = np.minimum(n - 1, s * SH + SH - 1 + hi)
    return oracle.region(a, b, cbeg + 1, cend + 1, min(n, hi), min(m, max(0, -lo)))


def test_certificate_decisions_match_the_closed_form(ctx):
    """Round-1 certifications = pairs whose oracle score over the kernel's
    cell region (stripe rectangles around the band) beats U0."""
    import torch
    import paper_2412_21103_gb300 as nw
    c = nw.Context(0, torch.cuda.current_stream())
    pairs = _band_pairs(99, 30, lmax=900)
    pool, ao, al, bo, bl = _pool(pairs)
    w = 24
    nw.nw_align_batch_banded(c, pool, ao, al, bo, bl, np.full(len(pairs), w, np.uint32), (1, -1, -1), nw.NW_CIGAR)
    st = nw.nw_ctx_band_stats(c)
    expect = 0
    tried = 0
    for a, b in pairs:
        lo, hi = oracle.band_limits(a.size, b.size, w)
        R = BAND_R
        SH = 32 * R
        width = min(b.size, SH + hi - lo)
        period = max(width, SH + 96)
        rows = -(-a.size // SH) * SH
        if rows * period * 20 >= rows * max(b.size, 96) * 17:
            continue            # the band would cover most of the grid: straight to full
        tried += 1
        sb = _region_score(a, b, w)
        sb_strict, _ = oracle.banded(a, b, w)
        assert sb >= sb_strict  # a superset of the band
        U = oracle.exit_bound(a.size, b.size, w)
        expect += U is None or sb > U
    assert st["tried"] == tried
    assert st["certified_round"][0] == expect
    c.close()


def test_learned_flag_without_model_is_exact(ctx):
    import paper_2412_21103_gb300 as nw
    pairs = _band_pairs(5, 20)
    pool, ao, al, bo, bl = _pool(pairs)
    scores, cigars = nw.nw_align_batch(ctx, pool, ao, al, bo, bl, (1, -1, -1), nw.NW_CIGAR | nw.NW_LEARNED_BAND)
    want = oracle.align_many(pairs)
    for k, (s, ops) in enumerate(want):
        assert scores[k] == s and cigars[k] == oracle.rle(ops)


def test_features_match_reference(ctx):
    import torch
    import paper_2412_21103_gb300 as nw
    pairs = _band_pairs(11, 12) + [(np.zeros(3, np.uint8), np.zeros(10, np.uint8))]
    pool, ao, al, bo, bl = _pool(pairs)
    f = nw.nw_band_features(ctx, torch.from_numpy(pool).cuda(), ao, al, bo, bl).cpu().numpy()
    for k, (a, b) in enumerate(pairs):
        assert np.allclose(f[k], bm.features(a, b), atol=1e-6), k


def test_network_forward_and_gradients_match_reference(ctx):
    import torch
    import paper_2412_21103_gb300 as nw
    nw.nw_band_model_init(ctx, 1234)
    params = nw.nw_band_model_get(ctx).astype(np.float64)
    rs = np.random.default_rng(0)
    X = rs.uniform(0, 1, (64, 65)).astype(np.float32)
    X[:, 64] = rs.uniform(-0.3, 0.3, 64)
    t = rs.normal(4.0, 1.0, 64).astype(np.float32)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    y = nw.nw_band_model_forward(ctx, Xd).cpu().numpy()
    y_ref, _ = bm.forward(params, X.astype(np.float64))
    assert np.allclose(y, y_ref, rtol=1e-2, atol=1e-3)
    g, loss = nw.nw_band_model_grad(ctx, Xd, td)
    loss_ref, g_ref = bm.loss_and_grad(params, X.astype(np.float64), t.astype(np.float64))
    g = g.cpu().numpy()
    assert float(loss.item()) == pytest.approx(loss_ref, rel=1e-2)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= 1e-2


def test_training_lowers_the_loss(ctx):
    import torch
    import paper_2412_21103_gb300 as nw
    nw.nw_band_model_init(ctx, 7)
    rs = np.random.default_rng(1)
    X = rs.uniform(0, 1, (512, 65)).astype(np.float32)
    t = (2.0 + 3.0 * X[:, 10] - 2.0 * X[:, 40]).astype(np.float32)   # a learnable target
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    first = float(nw.nw_band_model_train_step(ctx, Xd, td, 3e-3).item())
    for _ in range(300):
        last = nw.nw_band_model_train_step(ctx, Xd, td, 3e-3)
    assert float(last.item()) < 0.1 * first
    p = nw.nw_band_model_get(ctx)
    nw.nw_band_model_set(ctx, p)
    assert np.array_equal(nw.nw_band_model_get(ctx), p)
