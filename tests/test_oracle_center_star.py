"""Pins for the CPU reference of the center-star multiple alignment (Sec.
3.2): a hand-worked family, brute force over every alignment of tiny
families, and the properties that fix the merge (every row is its sequence,
every pairwise alignment with the center survives, no column is all
gaps)."""
import os

import numpy as np
import pytest

import oracle
import seqgen
from oracle import center_star as cs

from helpers import GOLDEN, brute_force, codes, ops_to_moves, parse_cigar


def _hand():
    d = {}
    for ln in open(os.path.join(GOLDEN, "center_star_hand.txt")):
        if ln.startswith("#") or ":" not in ln:
            continue
        k, _, v = ln.partition(":")
        d[k.strip()] = v.split()
    return d


def test_hand_worked_family():
    d = _hand()
    seqs = [codes(s) for s in d["seqs"]]
    c, sums, aligned, rows = cs.center_star(seqs)
    assert c == int(d["center"][0])
    assert sums.tolist() == [int(x) for x in d["sums"]]
    assert [s for s, _ in aligned] == [int(x) for x in d["scores"]]
    assert [oracle.rle(ops) for _, ops in aligned] == d["cigars"]
    assert rows == d["rows"]


def _tiny_family(seed, nseq, lmax):
    rs = seqgen.Stream(seed)
    lens = rs.integers(0, lmax, nseq)
    return [rs.bases(int(L)) for L in lens]


@pytest.mark.parametrize("seed", range(6))
def test_score_matrix_and_center_by_brute_force(seed):
    """Every entry by enumerating all alignments of the pair; the center is
    the first index of the largest sum over the other sequences."""
    seqs = _tiny_family(100 + seed, 5, 5)
    M = cs.score_matrix(seqs)
    n = len(seqs)
    for i in range(n):
        for j in range(n):
            want = len(seqs[i]) if i == j else brute_force(seqs[i], seqs[j], 1, -1, -1)[0]
            assert M[i, j] == want
    best = None
    for i in range(n):
        tot = sum(brute_force(seqs[i], seqs[j], 1, -1, -1)[0] for j in range(n) if j != i)
        if best is None or tot > best[1]:
            best = (i, tot)
    assert cs.choose_center(M)[0] == best[0]


def test_center_ties_go_to_the_lowest_index():
    seqs = [codes("ACGT")] * 3
    assert cs.choose_center(cs.score_matrix(seqs))[0] == 0


def _projection(row, crow):
    """The pairwise alignment a merged row makes with the center row: the
    columns where not both are gaps, as '=XID' ops."""
    ops = []
    for x, y in zip(row, crow):
        if x == "-" and y == "-":
            continue
        if x == "-":
            ops.append("D")
        elif y == "-":
            ops.append("I")
        else:
            ops.append("=" if x == y else "X")
    return "".join(ops)


@pytest.mark.parametrize("seed,nseq,lmax", [(1, 6, 12), (2, 9, 30), (3, 4, 0), (4, 12, 60)])
def test_merge_keeps_sequences_and_pairwise_alignments(seed, nseq, lmax):
    if lmax == 0:
        seqs = [np.zeros(0, np.uint8), codes("ACG"), np.zeros(0, np.uint8), codes("T")]
    else:
        seqs = _tiny_family(seed, nseq, lmax)
    c, sums, aligned, rows = cs.center_star(seqs)
    assert len({len(r) for r in rows}) == 1
    ncols = len(rows[0])
    for k, (s, row) in enumerate(zip(seqs, rows)):
        assert row.replace("-", "") == "".join("ACGT"[int(x)] for x in s)
        assert _projection(row, rows[c]) == aligned[k][1]
    # no all-gap column: with the projections above this fixes every slot at
    # the most insertions any alignment puts there
    for j in range(ncols):
        assert any(r[j] != "-" for r in rows)


def test_alignment_with_center_is_the_global_alignment():
    """Each pairwise alignment with the center is the Sec. 2 alignment of
    that pair (brute force: best score, diagonal > vertical > horizontal)."""
    seqs = _tiny_family(9, 5, 5)
    c, _, aligned, _ = cs.center_star(seqs)
    for s, (sc, ops) in zip(seqs, aligned):
        best, path = brute_force(s, seqs[c], 1, -1, -1)
        assert sc == best and ops_to_moves(ops) == path


def test_family_recipe_center_star_shape():
    """A mutant family (the all-vs-all recipe, small): every row has the
    merged length and parses back."""
    seqs = seqgen.all_vs_all_family(7, nseq=20, root_len=200, lmin=60, lmax=200)
    c, sums, aligned, rows = cs.center_star(seqs)
    assert 0 <= c < 20 and sums[c] == sums.max()
    for k, (sc, ops) in enumerate(aligned):
        assert oracle.rle(ops) and parse_cigar(oracle.rle(ops)) == ops


def test_merge_slots_by_hand():
    """Center AC (index 0) and four alignments given as ops, worked by hand:
    GAC puts one base before A (slot 0), AGGC two and AGC one between A and
    C (slot 1, filled from its left), ACTT two after C (slot 2).  So G =
    [1, 2, 2] and the merge has 2 + 5 = 7 columns: [s0] A [s1 s1] C [s2 s2]."""
    seqs = [codes("AC"), codes("GAC"), codes("ACTT"), codes("AGGC"), codes("AGC")]
    ops = ["==", "I==", "==II", "=II=", "=I="]
    assert cs.slot_gaps(ops, 2).tolist() == [1, 2, 2]
    assert cs.merge(seqs, 0, ops) == ["-A--C--", "GA--C--", "-A--CTT", "-AGGC--", "-AG-C--"]
