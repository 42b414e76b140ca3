"""What the trained band-width network gains (a9): on held-out pairs of the
band workload, the certified band started from the network's prediction
certifies more pairs in its first round than the same certified band
started from a fixed width without the network -- fewer pairs need a second
banded fill -- and sweeps far fewer cells than the full grid, with every
score and CIGAR equal to the oracle's.  The network is trained on the GPU by
the library's own kernels from the committed oracle labels.  (The window
kernel sweeps whole 32-row words, so the learned start's wider first round
sweeps more window cells than the fixed start; the end-to-end time of both
starts on the whole workload is the benchmark's comparison.)"""
import os

import numpy as np
import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu

LABELS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "band_labels_seed9004.npz")


def _pool(pairs):
    import paper_2412_21103_gb300 as nw
    seqs = []
    for a, b in pairs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    return pool, off[0::2], lens[0::2], off[1::2], lens[1::2]


def _train(nw, ctx, epochs=40):
    import torch
    lab = np.load(LABELS)
    count = int(lab["label"].size)
    pairs = seqgen.band_pairs(int(lab["seed"]), npairs=count)
    pool, ao, al, bo, bl = _pool([(p.a, p.b) for p in pairs])
    feat = nw.nw_band_features(ctx, torch.from_numpy(pool).cuda(), ao, al, bo, bl)
    target = torch.from_numpy(np.log(np.maximum(lab["label"], 1)).astype(np.float32)).cuda()
    nw.nw_band_model_init(ctx, 0)
    g = torch.Generator().manual_seed(0)
    first = last = None
    for _ in range(epochs):
        perm = torch.randperm(count, generator=g).cuda()
        for k in range(0, count - 511, 512):
            idx = perm[k:k + 512]
            loss = float(nw.nw_band_model_train_step(ctx, feat[idx].contiguous(), target[idx].contiguous(),
                                                      2e-3).item())
            first = loss if first is None else first
            last = loss
    return first, last


def test_learned_band_beats_fixed_start_and_full_grid():
    import torch
    import paper_2412_21103_gb300 as nw
    if not os.path.exists(LABELS):
        pytest.fail("training labels missing: run tests/golden/make_band_labels.py")
    held_out = [(p.a, p.b) for p in seqgen.band_pairs(1004, npairs=160)]
    pool, ao, al, bo, bl = _pool(held_out)
    want = oracle.align_many(held_out)
    full_cells = sum(int(x) * int(y) for x, y in zip(al, bl))

    # every pair stays in the banded rounds (none is sent to the full-grid
    # kernel for scheduling), so that the certificates measure the widths
    os.environ["NW_BAND_KEEP"] = "1"
    try:
        # without the network: certified band from the fixed start (64)
        c0 = nw.Context(0, torch.cuda.current_stream())
        s0, g0 = nw.nw_align_batch(c0, pool, ao, al, bo, bl, (1, -1, -1), nw.NW_CIGAR | nw.NW_LEARNED_BAND)
        st0 = nw.nw_ctx_band_stats(c0)

        # with the network trained on the GPU
        c1 = nw.Context(0, torch.cuda.current_stream())
        first, last = _train(nw, c1)
        assert last < 0.5 * first
        s1, g1 = nw.nw_align_batch(c1, pool, ao, al, bo, bl, (1, -1, -1), nw.NW_CIGAR | nw.NW_LEARNED_BAND)
        st1 = nw.nw_ctx_band_stats(c1)
    finally:
        del os.environ["NW_BAND_KEEP"]
    # with scheduling on, the same results whatever the rounds keep
    s2, g2 = nw.nw_align_batch(c1, pool, ao, al, bo, bl, (1, -1, -1), nw.NW_CIGAR | nw.NW_LEARNED_BAND)

    for k, (s, ops) in enumerate(want):
        assert s0[k] == s and g0[k] == oracle.rle(ops)
        assert s1[k] == s and g1[k] == oracle.rle(ops)
        assert s2[k] == s and g2[k] == oracle.rle(ops)

    def swept(st):
        # banded cells plus the full grid of every pair that fell back
        fb = sum(int(al[k]) * int(bl[k]) for k in range(len(held_out)))  # upper bound used only below
        return st["band_cells"], st["full_fallback"]

    band1, fb1 = swept(st1)
    band0, fb0 = swept(st0)
    print(f"learned: band cells {band1:.3g}, fallbacks {fb1}; fixed start: band cells {band0:.3g}, "
          f"fallbacks {fb0}; full grid {full_cells:.3g}")
    # the network's start certifies more pairs in the first round (so fewer
    # pairs need a second banded fill) than the fixed start; with the full
    # grids of every pair that went to the full kernel (certificate or
    # scheduling) the work stays far below the full grids of all pairs
    r0_learned, r0_fixed = st1["certified_round"][0], st0["certified_round"][0]
    print(f"first-round certifications: learned {r0_learned}, fixed start {r0_fixed}")
    assert r0_learned > 2 * r0_fixed
    per_pair = full_cells / len(held_out)
    assert band1 + fb1 * per_pair < 0.8 * full_cells
    c0.close()
    c1.close()


def test_model_checkpoint_roundtrip(tmp_path):
    """A trained model saved to a file and loaded into a fresh context gives
    bit-identical network outputs; a file of the wrong size is refused."""
    import torch
    import paper_2412_21103_gb300 as nw
    c1 = nw.Context(0, torch.cuda.current_stream())
    _train(nw, c1, epochs=2)
    path = tmp_path / "band_model.bin"
    nw.nw_band_model_save(c1, path)
    assert path.stat().st_size == 16 + 4 * nw.nw_band_model_size()
    pairs = [(p.a, p.b) for p in seqgen.band_pairs(1004, npairs=64)]
    pool, ao, al, bo, bl = _pool(pairs)
    feat = nw.nw_band_features(c1, torch.from_numpy(pool).cuda(), ao, al, bo, bl)
    y1 = nw.nw_band_model_forward(c1, feat).cpu().numpy()
    c2 = nw.Context(0, torch.cuda.current_stream())
    nw.nw_band_model_load(c2, path)
    y2 = nw.nw_band_model_forward(c2, feat).cpu().numpy()
    assert np.array_equal(y1, y2)
    assert np.array_equal(nw.nw_band_model_get(c1), nw.nw_band_model_get(c2))
    bad = tmp_path / "short.bin"
    bad.write_bytes(path.read_bytes()[:-4])
    with pytest.raises(nw.NWError):
        nw.nw_band_model_load(c2, bad)
    c1.close()
    c2.close()
