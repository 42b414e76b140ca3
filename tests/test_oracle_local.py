"""Pins for the local-alignment oracle (Smith-Waterman: the global grid with a
floor of 0; not in the paper): every cell by brute force over all substring
pairs and all their alignments, the end cell and the walk checked against
those brute-force values, the longest-common-substring special case, and
invariants."""
import numpy as np
import pytest

import oracle
import seqgen

from helpers import brute_force, codes, rescore


def _brute_grid(a, b, sc):
    """H(i,j) = the best score of any alignment of a suffix of A[:i] with a
    suffix of B[:j], the empty one (0) included."""
    m, n = len(a), len(b)
    H = np.zeros((m + 1, n + 1), np.int64)
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            best = 0
            for i0 in range(i + 1):
                for j0 in range(j + 1):
                    if i0 == i and j0 == j:
                        continue
                    best = max(best, brute_force(a[i0:i], b[j0:j], *sc)[0])
            H[i, j] = best
    return H


def _tiny_pairs():
    rs = seqgen.Stream(606)
    out = [(codes("ACGT"), codes("ACGT")), (codes("AAAA"), codes("CCCC")), (codes("ACG"), codes("")),
           (codes("GATT"), codes("TTGA"))]
    for _ in range(8):
        m, n = (int(x) for x in rs.integers(1, 4, 2))
        out.append((rs.bases(m), rs.bases(n)))
    return out


@pytest.mark.parametrize("sc", [(1, -1, -1), (2, -1, -2), (1, -3, -1)])
def test_grid_by_brute_force(sc):
    for a, b in _tiny_pairs():
        assert (oracle.local_fill(a, b, *sc) == _brute_grid(a, b, sc)).all()


@pytest.mark.parametrize("sc", [(1, -1, -1), (2, -1, -2), (1, -3, -1)])
def test_end_cell_and_walk_against_brute_force(sc):
    """The end is the first cell in row-major order holding the largest
    value; every step of the walk takes the highest-priority predecessor
    (diagonal > vertical > horizontal) that the brute-force values allow, and
    the walk stops at the first cell whose value is 0."""
    for a, b in _tiny_pairs():
        H = _brute_grid(a, b, sc)
        s, (i0, j0, i1, j1), ops = oracle.local_align(a, b, *sc)
        assert s == H.max()
        first = np.argwhere(H == H.max())[0]
        assert (i1, j1) == (int(first[0]), int(first[1]))
        i, j = i1, j1
        for o in reversed(ops):
            assert H[i, j] > 0
            d = sc[0] if (i and j and a[i - 1] == b[j - 1]) else sc[1]
            can_d = i > 0 and j > 0 and H[i, j] == H[i - 1, j - 1] + d
            can_u = i > 0 and H[i, j] == H[i - 1, j] + sc[2]
            if o in "=X":
                assert can_d
                i, j = i - 1, j - 1
            elif o == "I":
                assert not can_d and can_u
                i -= 1
            else:
                assert not can_d and not can_u and H[i, j] == H[i, j - 1] + sc[2]
                j -= 1
        assert (i, j) == (i0, j0) and H[i, j] == 0
        assert rescore(ops, a[i0:i1], b[j0:j1], *sc) == s


def _longest_common_substring(a, b):
    best = 0
    for i in range(len(a)):
        for j in range(len(b)):
            k = 0
            while i + k < len(a) and j + k < len(b) and a[i + k] == b[j + k]:
                k += 1
            best = max(best, k)
    return best


def test_longest_common_substring_special_case():
    """match 1, mismatch and gap -40: below 40 matched bases no mismatch or
    gap can pay for itself, so the score is the longest common substring."""
    rs = seqgen.Stream(707)
    for _ in range(25):
        m, n = (int(x) for x in rs.integers(0, 35, 2))
        a, b = rs.bases(m), rs.bases(n)
        assert oracle.local_score(a, b, 1, -40, -40) == _longest_common_substring(a, b)
        s, (i0, j0, i1, j1), ops = oracle.local_align(a, b, 1, -40, -40)
        assert ops == "=" * s and (a[i0:i1] == b[j0:j1]).all()


def test_invariants():
    rs = seqgen.Stream(808)
    for _ in range(30):
        m, n = (int(x) for x in rs.integers(0, 120, 2))
        a, b = rs.bases(m), rs.bases(n)
        s = oracle.local_score(a, b)
        assert s == oracle.local_score(b, a)
        assert s >= max(0, oracle.score(a, b))
        assert s == oracle.local_align(a, b)[0]
        assert oracle.local_score(a, a) == m
