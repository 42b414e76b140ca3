"""The seeded synthetic inputs have the shapes the workloads state: lengths,
mutation rates, arrival process, and every generated pair's transcript turns
A into B."""
import numpy as np

import seqgen


def _apply(a, b, ops):
    """Walk a '=XID' transcript over A and B; returns (=, X, I, D) counts."""
    i = j = 0
    counts = dict.fromkeys("=XID", 0)
    for o in ops:
        counts[o] += 1
        if o == "=":
            assert a[i] == b[j]
            i += 1
            j += 1
        elif o == "X":
            assert a[i] != b[j]
            i += 1
            j += 1
        elif o == "I":
            i += 1
        else:
            j += 1
    assert i == a.size and j == b.size
    return counts


def test_config1_uniform_pair():
    p = seqgen.random_pair(1001, 1000, 1000)
    assert p.a.size == 1000 and p.b.size == 1000
    for s in (p.a, p.b):
        assert set(np.unique(s)) <= {0, 1, 2, 3}
        freq = np.bincount(s, minlength=4) / s.size
        assert np.all(np.abs(freq - 0.25) < 0.05)


def test_config2_mutation_rates():
    p = seqgen.long_mutated_pair(1002)
    assert p.a.size == 32768
    c = _apply(p.a, p.b, p.transcript)
    assert abs(c["X"] / p.a.size - 0.10) < 0.01          # substitutions, 10 %
    assert 0.5 * 0.02 < (c["I"] + c["D"]) / p.a.size / 3.0 < 2.0 * 0.02  # indel starts ~2 %, mean length 3


def test_config3_family_lengths():
    fam = seqgen.all_vs_all_family(1003, nseq=512)
    lens = np.array([s.size for s in fam])
    # root prefixes of U{500..1500} bases; the 1-bp indels move a mutant's length a little
    assert lens.size == 512 and lens.min() >= 0.95 * 500 and lens.max() <= 1.05 * 1500
    assert abs(np.mean(lens) - 1000) < 50


def test_config4_lengths_and_transcripts():
    pairs = seqgen.band_pairs(1004, npairs=300)
    lens = np.array([p.a.size for p in pairs])
    assert lens.min() >= 2000 and lens.max() <= 20000
    med = np.median(lens)
    assert 0.7 * np.sqrt(2000 * 20000) < med < 1.3 * np.sqrt(2000 * 20000)  # log-uniform
    for p in pairs[:40]:
        c = _apply(p.a, p.b, p.transcript)
        assert c["X"] <= round(0.25 * p.a.size)   # substitutions are at most the 25 % of mutations


def test_config5_arrivals_and_mix():
    reqs = list(seqgen.serving_stream(1005, rate=50000.0, limit=4000))
    t = np.array([r.t_arrival for r in reqs])
    gaps = np.diff(t)
    assert np.all(gaps >= 0)
    assert abs(gaps.mean() * 50000.0 - 1.0) < 0.1          # Poisson at 50k req/s
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1       # exponential gaps
    lens = np.array([r.pair.a.size for r in reqs])
    assert lens.min() >= 50 and lens.max() <= 50000
    frac = np.mean([r.want_cigar for r in reqs])
    assert 0.45 < frac < 0.55
