"""Write band_labels_seed9004.npz: training labels for the learned band.

Calls only oracle/ (and the seeded generator).  The training pairs are the
band workload's distribution (lengths log-uniform in [2,000, 20,000],
divergence U[0.01, 0.25], geometric indels, indel bursts with probability
0.3) drawn from seed 9004, disjoint from the evaluation seed 1004.  For every
pair the oracle aligns it (score S and the traceback); the label is the
smallest band half-width w whose closed-form exit bound U0(w) lies strictly
below S -- the narrowest band the certificate accepts -- which is never
below the traceback's excursion from the diagonals between 0 and n-m (both
are stored).

    python tests/golden/make_band_labels.py [count]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import seqgen  # noqa: E402
from oracle import band_model as bm  # noqa: E402

SEED = 9004


def main():
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 4000
    t0 = time.time()
    pairs = seqgen.band_pairs(SEED, npairs=count)
    res = oracle.align_many([(p.a, p.b) for p in pairs], threads=min(8, os.cpu_count() or 1))
    m = np.array([p.a.size for p in pairs], np.int64)
    n = np.array([p.b.size for p in pairs], np.int64)
    score = np.array([s for s, _ in res], np.int64)
    exc = np.array([bm.excursion(ops, p.a.size, p.b.size) for (s, ops), p in zip(res, pairs)], np.int64)
    label = np.array([bm.band_label(int(a), int(b), int(s), int(e)) for a, b, s, e in zip(m, n, score, exc)],
                     np.int64)
    assert (label >= exc).all()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"band_labels_seed{SEED}.npz")
    np.savez_compressed(out, seed=SEED, m=m, n=n, score=score, excursion=exc, label=label)
    print(f"{count} pairs in {time.time() - t0:.0f} s -> {out}")


if __name__ == "__main__":
    main()
