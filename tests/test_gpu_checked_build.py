"""The bounds-checked debug build (libnw_checks.so, -DNW_CHECKS) on the GPU:
in a fresh process with NW_CHECKS=1 the binding loads the checked library,
and every path whose kernels carry checked stores -- the batched global
kernel (plain, certified band, all pairs), local alignment, affine gaps and
the center-star merge -- gives the oracle's results with no out-of-range
store reported (NW_ERR_BOUNDS would surface at the next sync)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import numpy as np, torch
import oracle, seqgen
from oracle import center_star as cs
import paper_2412_21103_gb300 as nw
from paper_2412_21103_gb300 import build
assert nw.lib_path() == build.CHECKS_LIB
build.build(checks=True)
ctx = nw.Context(0, torch.cuda.current_stream())
rs = seqgen.Stream(2024)
pairs = []
for k in range(40):
    m, n = (int(x) for x in rs.integers(0, 1200, 2))
    if k % 2:
        p = seqgen.long_mutated_pair(700 + k, m=max(m, 2))
        pairs.append((p.a, p.b))
    else:
        pairs.append((rs.bases(m), rs.bases(n)))
seqs = []
for a, b in pairs:
    seqs += [a, b]
pool, off, lens = nw.pool_of(seqs)
ao, al, bo, bl = off[0::2], lens[0::2], off[1::2], lens[1::2]
want = oracle.align_many(pairs)
for flags in (nw.NW_CIGAR, nw.NW_CIGAR | nw.NW_LEARNED_BAND):
    s, c = nw.nw_align_batch(ctx, pool, ao, al, bo, bl, (1, -1, -1), flags)
    assert s.tolist() == [x for x, _ in want] and c == [oracle.rle(o) for _, o in want], flags
ctx.sync()
fam = seqgen.all_vs_all_family(5, nseq=24, root_len=500, lmin=100, lmax=500)
fp, fo, fl = nw.pool_of(fam)
mat = nw.nw_score_all_pairs(ctx, fp, fo, fl)
assert mat[0, 1] == oracle.score(fam[0], fam[1]) and mat[3, 7] == oracle.score(fam[3], fam[7])
got = nw.nw_center_star(ctx, fp, fo, fl)
c0, _, _, rows = cs.center_star(fam)
assert got["center"] == c0 and got["rows"] == rows
sc, ends, cig = nw.nw_local_align_batch(ctx, pool, ao, al, bo, bl, (1, -1, -1), nw.NW_CIGAR)
for k, (s_, e_, o_) in enumerate(oracle.local_align_many(pairs)):
    assert int(sc[k]) == s_ and tuple(int(x) for x in ends[k]) == e_ and cig[k] == oracle.rle(o_), k
sa, ca = nw.nw_affine_align_batch(ctx, pool, ao, al, bo, bl, (2, -3, -5, -2), nw.NW_CIGAR)
for k, (s_, o_) in enumerate(oracle.affine_align_many(pairs, 2, -3, -5, -2)):
    assert int(sa[k]) == s_ and ca[k] == oracle.rle(o_), k
ctx.sync()
ctx.close()
print("checked build ok")
"""


def test_checked_build_runs_every_checked_path_exactly():
    env = dict(os.environ, NW_CHECKS="1")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout
