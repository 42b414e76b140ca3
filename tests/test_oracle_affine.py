"""Pins for the affine-gap oracle (Gotoh; a run of k gap moves of one kind
scores open + k * extend): the three grids by brute force over every
alignment, each step of the walk against those brute-force values, the
reduction to the linear oracle when the open cost is 0, closed forms."""
import numpy as np
import pytest

import oracle
import seqgen

from helpers import all_paths, codes, ops_to_moves

NEG = -(2 ** 31) // 4


def _path_score(path, a, b, match, mismatch, go, ge):
    i = j = 0
    s = 0
    prev = ""
    for mv in path:
        if mv == "d":
            s += match if a[i] == b[j] else mismatch
            i, j = i + 1, j + 1
        else:
            s += ge + (go if mv != prev else 0)
            if mv == "u":
                i += 1
            else:
                j += 1
        prev = mv
    return s


def _brute_grids(a, b, sc):
    """H, E, F by enumerating every alignment of every prefix pair."""
    m, n = len(a), len(b)
    H = np.full((m + 1, n + 1), NEG, np.int64)
    E = np.full((m + 1, n + 1), NEG, np.int64)
    F = np.full((m + 1, n + 1), NEG, np.int64)
    for i in range(m + 1):
        for j in range(n + 1):
            for p in all_paths(i, j):
                s = _path_score(p, a[:i], b[:j], *sc)
                H[i, j] = max(H[i, j], s)
                if p and p[-1] == "l":
                    E[i, j] = max(E[i, j], s)
                if p and p[-1] == "u":
                    F[i, j] = max(F[i, j], s)
    H[0, 0] = 0
    return H, E, F


def _tiny_pairs():
    rs = seqgen.Stream(909)
    out = [(codes("ACGT"), codes("AGT")), (codes("AAAA"), codes("A")), (codes(""), codes("CG")),
           (codes("GATTACA"), codes("GCA"))]
    for _ in range(8):
        m, n = (int(x) for x in rs.integers(0, 5, 2))
        out.append((rs.bases(m), rs.bases(n)))
    return out


SCORINGS = [(1, -1, -2, -1), (2, -1, -3, -1), (1, -2, -1, -1), (1, -1, 0, -1)]


@pytest.mark.parametrize("sc", SCORINGS)
def test_grids_by_brute_force(sc):
    for a, b in _tiny_pairs():
        H, E, F = oracle.affine_fill(a, b, *sc)
        bH, bE, bF = _brute_grids(a, b, sc)
        assert (H == bH).all()
        mask = bE > NEG          # cells no alignment reaches stay at the oracle's -inf
        assert (E[mask] == bE[mask]).all() and (E[~mask] <= NEG).all()
        mask = bF > NEG
        assert (F[mask] == bF[mask]).all() and (F[~mask] <= NEG).all()


@pytest.mark.parametrize("sc", SCORINGS)
def test_walk_against_brute_force(sc):
    """The walk takes the diagonal when it gives H, else the vertical gap
    when F gives H, else the horizontal one; inside a gap it extends only
    when extending is strictly better than opening."""
    match, mismatch, go, ge = sc
    for a, b in _tiny_pairs():
        H, E, F = _brute_grids(a, b, sc)
        s, ops = oracle.affine_align(a, b, *sc)
        assert s == H[len(a), len(b)]
        mv = ops_to_moves(ops)
        assert _path_score(mv, a, b, *sc) == s
        i, j, state = len(a), len(b), "H"
        for o in reversed(mv):
            if i == 0:
                assert o == "l"
                j -= 1
                continue
            if j == 0:
                assert o == "u"
                i -= 1
                continue
            if state == "H":
                d = match if a[i - 1] == b[j - 1] else mismatch
                if H[i, j] == H[i - 1, j - 1] + d:
                    assert o == "d"
                    i, j = i - 1, j - 1
                    continue
                state = "F" if H[i, j] == F[i, j] else "E"
            if state == "F":
                assert o == "u"
                state = "F" if F[i - 1, j] > NEG and F[i - 1, j] + ge > H[i - 1, j] + go + ge else "H"
                i -= 1
            else:
                assert o == "l"
                state = "E" if E[i, j - 1] > NEG and E[i, j - 1] + ge > H[i, j - 1] + go + ge else "H"
                j -= 1
        assert (i, j) == (0, 0)


def test_open_cost_zero_is_the_linear_alignment():
    """With open 0 a gap run of k scores k * extend, the linear penalty: the
    score and the walk equal the linear oracle's, move for move."""
    rs = seqgen.Stream(1212)
    for _ in range(40):
        m, n = (int(x) for x in rs.integers(0, 150, 2))
        a, b = rs.bases(m), rs.bases(n)
        for sc in [(1, -1, -1), (2, -1, -2), (1, -3, -1)]:
            assert oracle.affine_align(a, b, sc[0], sc[1], 0, sc[2]) == oracle.align(a, b, *sc)


def test_closed_forms_and_score_only():
    rs = seqgen.Stream(1313)
    a = rs.bases(77)
    assert oracle.affine_align(a, a, 2, -1, -5, -1) == (154, "=" * 77)
    assert oracle.affine_align([], rs.bases(9), 1, -1, -3, -2) == (-3 - 18, "D" * 9)
    assert oracle.affine_align(rs.bases(4), [], 1, -1, -3, -2) == (-3 - 8, "I" * 4)
    assert oracle.affine_align([], [], 1, -1, -3, -2) == (0, "")
    for _ in range(20):
        m, n = (int(x) for x in rs.integers(0, 300, 2))
        x, y = rs.bases(m), rs.bases(n)
        assert oracle.affine_score(x, y, 1, -2, -4, -1) == oracle.affine_align(x, y, 1, -2, -4, -1)[0]
        assert oracle.affine_score(x, y, 1, -2, -4, -1) == oracle.affine_score(y, x, 1, -2, -4, -1)
