"""Pins for the CPU oracle: each check comes from the paper's definition or
from mathematics, never from the oracle itself (Sec. 2.2-2.4, Eq. 1, Eq. 2)."""
import itertools

import numpy as np
import pytest

import oracle
import seqgen
from helpers import (all_paths, ascii_of, brute_force, codes, consumed, lcs_bitparallel, lcs_brute,
                     levenshtein_myers, load_hand_grids, ops_to_moves, parse_cigar, path_score, rescore)

SCHEMES = [(1, -1, -1), (2, -1, -2), (0, -1, -1), (1, 0, 0), (3, -2, -1), (1, -3, -1), (5, 4, -3)]


# --------------------------------------------------------- hand-worked grids
@pytest.mark.parametrize("case", load_hand_grids(), ids=lambda c: c["case"])
def test_hand_worked_grid(case):
    a, b = codes(case["a"]), codes(case["b"])
    ma, mm, g = case["scoring"]
    H = oracle.fill(a, b, ma, mm, g)
    assert H.tolist() == case["grid"]
    s, ops = oracle.align(a, b, ma, mm, g)
    assert s == case["score"]
    assert oracle.rle(ops) == case["cigar"]
    assert oracle.score(a, b, ma, mm, g) == case["score"]


def test_boundary_decreases_by_one_per_cell():
    """Sec. 2.2: H(0,0)=0 and the first row/column fall by one per cell."""
    rs = seqgen.Stream(7)
    H = oracle.fill(rs.bases(9), rs.bases(13))
    assert H[0, 0] == 0
    assert H[0, :].tolist() == [-j for j in range(14)]
    assert H[:, 0].tolist() == [-i for i in range(10)]


# ------------------------------------------------------------- brute force
def _brute_cases():
    rs = seqgen.Stream(11)
    out = []
    for k in range(140):
        m = int(rs.integers(0, 6, 1)[0])
        n = int(rs.integers(0, 6, 1)[0])
        scheme = SCHEMES[k % len(SCHEMES)]
        out.append((rs.bases(m), rs.bases(n), scheme))
    # every pair of length-2 sequences over a 2-letter sub-alphabet (many ties)
    for x in itertools.product([0, 1], repeat=2):
        for y in itertools.product([0, 1], repeat=3):
            out.append((np.array(x, np.uint8), np.array(y, np.uint8), (1, -1, -1)))
    return out


def test_delannoy_path_count():
    """Sanity of the brute-force enumerator: D(m,n) Delannoy numbers."""
    assert len(all_paths(6, 6)) == 8989
    assert len(all_paths(3, 2)) == 25


@pytest.mark.parametrize("idx", range(len(_brute_cases())))
def test_brute_force_score_and_tiebreak(idx):
    a, b, (ma, mm, g) = _brute_cases()[idx]
    best, path = brute_force(a, b, ma, mm, g)
    s, ops = oracle.align(a, b, ma, mm, g)
    assert s == best
    # the single path is the lexicographically greatest reversed move string
    # among the optimal ones (diagonal > vertical > horizontal)
    assert ops_to_moves(ops) == path
    assert path_score(ops_to_moves(ops), a, b, ma, mm, g) == best
    assert oracle.score(a, b, ma, mm, g) == best


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("L", [0, 1, 7, 64, 333])
def test_identity(L):
    """score(a,a) = |a|*match with CIGAR '|a|='."""
    a = seqgen.Stream(L + 3).bases(L)
    s, ops = oracle.align(a, a, 1, -1, -1)
    assert s == L
    assert oracle.rle(ops) == (f"{L}=" if L else "")


@pytest.mark.parametrize("L", [1, 5, 40])
def test_empty_side(L):
    b = seqgen.Stream(L).bases(L)
    s, ops = oracle.align(np.zeros(0, np.uint8), b, 1, -1, -1)
    assert (s, oracle.rle(ops)) == (-L, f"{L}D")
    s, ops = oracle.align(b, np.zeros(0, np.uint8), 2, -1, -3)
    assert (s, oracle.rle(ops)) == (-3 * L, f"{L}I")


@pytest.mark.parametrize("L", [1, 6, 50])
def test_all_mismatch(L):
    """Equal length, no common base at any position and no shared letters at
    all: one mismatch (-1) beats two gaps (-2), so the optimum is L mismatches."""
    a = np.zeros(L, np.uint8)          # all A
    b = np.full(L, 3, np.uint8)        # all T
    s, ops = oracle.align(a, b, 1, -1, -1)
    assert (s, oracle.rle(ops)) == (-L, f"{L}X")


# ------------------------------------------ special cases with other algorithms
@pytest.mark.parametrize("seed", range(12))
def test_levenshtein_special_case(seed):
    """(match, mismatch, gap) = (0, -1, -1) turns NW into minus the unit-cost
    edit distance, computed here by Myers' bit-vector algorithm."""
    rs = seqgen.Stream(100 + seed)
    m, n = (int(x) for x in rs.integers(0, 90, 2))
    a, b = rs.bases(m), rs.bases(n)
    assert oracle.score(a, b, 0, -1, -1) == -levenshtein_myers(a, b)


@pytest.mark.parametrize("seed", range(12))
def test_lcs_special_case(seed):
    """(1, 0, 0) turns NW into the LCS length (bit-vector LCS)."""
    rs = seqgen.Stream(200 + seed)
    m, n = (int(x) for x in rs.integers(0, 90, 2))
    a, b = rs.bases(m), rs.bases(n)
    assert oracle.score(a, b, 1, 0, 0) == lcs_bitparallel(a, b)


def test_bitparallel_checkers_against_brute_force():
    rs = seqgen.Stream(5)
    for _ in range(60):
        m, n = (int(x) for x in rs.integers(0, 6, 2))
        a, b = rs.bases(m), rs.bases(n)
        assert lcs_bitparallel(a, b) == lcs_brute(a, b)
        best, _ = brute_force(a, b, 0, -1, -1)
        assert levenshtein_myers(a, b) == -best


# -------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", range(8))
def test_invariants(seed):
    rs = seqgen.Stream(300 + seed)
    m, n = (int(x) for x in rs.integers(0, 200, 2))
    a, b = rs.bases(m), rs.bases(n)
    for (ma, mm, g) in [(1, -1, -1), (2, -1, -2)]:
        s, ops = oracle.align(a, b, ma, mm, g)
        assert consumed(ops) == (m, n)
        assert rescore(ops, a, b, ma, mm, g) == s
        assert oracle.score(b, a, ma, mm, g) == s                 # symmetry
        assert oracle.score(a[::-1], b[::-1], ma, mm, g) == s     # reversal
        assert s <= ma * min(m, n) + g * abs(m - n)                # upper bound
        assert s >= g * (m + n)                                    # all-gap path


@pytest.mark.parametrize("seed", range(4))
def test_generator_transcript_is_a_lower_bound(seed):
    p = seqgen.long_mutated_pair(400 + seed, m=700)
    s, ops = oracle.align(p.a, p.b)
    assert s >= rescore(p.transcript, p.a, p.b, 1, -1, -1)
    assert rescore(ops, p.a, p.b, 1, -1, -1) == s


def test_pair_count_eq2():
    """Eq. 2: n sequences give n(n-1)/2 pairwise alignments."""
    n = 512
    assert len(list(itertools.combinations(range(n), 2))) == n * (n - 1) // 2 == 130816


# ------------------------------------------------------------------ banded
@pytest.mark.parametrize("seed", range(30))
def test_banded_brute_force(seed):
    """Banded optimum = best path that stays inside the band; U >= every path
    that leaves it; a band covering the grid reproduces full NW."""
    rs = seqgen.Stream(500 + seed)
    m, n = (int(x) for x in rs.integers(0, 6, 2))
    a, b = rs.bases(m), rs.bases(n)
    ma, mm, g = SCHEMES[seed % 3] if seed % 3 != 2 else (1, -1, -1)
    w = int(rs.integers(0, 3, 1)[0])
    delta = n - m
    lo, hi = min(0, delta) - w, max(0, delta) + w

    def inside(path):
        i = j = 0
        for mv in path:
            i += mv in "du"
            j += mv in "dl"
            if not (lo <= j - i <= hi):
                return False
        return True
    scores_in = []
    scores_out = []
    for p in all_paths(m, n):
        (scores_in if inside(p) else scores_out).append(path_score(p, a, b, ma, mm, g))
    sb, U = oracle.banded(a, b, w, ma, mm, g)
    assert sb == max(scores_in)
    if scores_out:
        assert U >= max(scores_out)
    else:
        assert U == oracle.NEG_INF
    full = oracle.score(a, b, ma, mm, g)
    sb_wide, _ = oracle.banded(a, b, max(m, n) + 1, ma, mm, g)
    assert sb_wide == full
    if sb >= U:
        assert sb == full


def test_rle_roundtrip():
    for ops in ["", "=", "==X", "IIDD=X", "X" * 17]:
        assert parse_cigar(oracle.rle(ops)) == ops
    assert ascii_of(codes("GATTACA")) == "GATTACA"


@pytest.mark.parametrize("seed", range(40))
def test_exit_bound_brute_force(seed):
    """U0 bounds every band-leaving path and is attained when a path with
    the minimal gap count exists with all-match diagonals (A == B here for
    the attainment check is not required: only the bound is asserted, plus
    None exactly when no path leaves the band)."""
    rs = seqgen.Stream(900 + seed)
    m, n = (int(x) for x in rs.integers(0, 6, 2))
    a, b = rs.bases(m), rs.bases(n)
    ma, mm, g = [(1, -1, -1), (2, -1, -2), (3, 1, -1), (0, -1, -1)][seed % 4]
    w = int(rs.integers(0, 3, 1)[0])
    lo, hi = oracle.band_limits(m, n, w)

    def leaves(path):
        i = j = 0
        for mv in path:
            i += mv in "du"
            j += mv in "dl"
            if not (lo <= j - i <= hi):
                return True
        return False
    out = [path_score(p, a, b, ma, mm, g) for p in all_paths(m, n) if leaves(p)]
    U0 = oracle.exit_bound(m, n, w, ma, g)
    if not out:
        assert U0 is None
    else:
        assert U0 is not None and U0 >= max(out)
    # certificate soundness: S_b > U0 implies the banded score is the full one
    sb, _ = oracle.banded(a, b, w, ma, mm, g)
    if U0 is None or sb > U0:
        assert sb == oracle.score(a, b, ma, mm, g)


def test_exit_bound_is_attained_by_identical_sequences():
    """With A == B (all diagonals match) the best band-leaving path makes
    exactly the minimal number of gap moves, so U0 is attained."""
    for L in range(1, 7):
        a = np.arange(L, dtype=np.uint8) % 4
        for w in range(0, 3):
            lo, hi = oracle.band_limits(L, L, w)

            def leaves(path):
                i = j = 0
                for mv in path:
                    i += mv in "du"
                    j += mv in "dl"
                    if not (lo <= j - i <= hi):
                        return True
                return False
            out = [path_score(p, a, a, 1, -1, -1) for p in all_paths(L, L) if leaves(p)]
            U0 = oracle.exit_bound(L, L, w, 1, -1)
            assert (U0 is None) == (not out)
            if out:
                assert U0 == max(out)


def _path_cells(path):
    i = j = 0
    cells = [(0, 0)]
    for mv in path:
        i += mv in "du"
        j += mv in "dl"
        cells.append((i, j))
    return cells


def _allowed(i, j, lo, hi, row0_hi, col0_hi):
    if i == 0:
        return j <= row0_hi
    if j == 0:
        return i <= col0_hi
    return lo[i - 1] <= j <= hi[i - 1]


@pytest.mark.parametrize("seed", range(40))
def test_region_dp_brute_force(seed):
    """The region DP is the best path that stays inside the allowed cells
    (brute force over every path for lengths <= 6, random regions)."""
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(1, 7)), int(rng.integers(1, 7))
    a, b = rng.integers(0, 4, m).astype(np.uint8), rng.integers(0, 4, n).astype(np.uint8)
    lo = rng.integers(1, n + 1, m)
    hi = np.minimum(n, lo + rng.integers(0, n, m))
    row0_hi, col0_hi = int(rng.integers(0, n + 1)), int(rng.integers(0, m + 1))
    sc = [(1, -1, -1), (2, -1, -2), (1, 0, 0)][seed % 3]
    best = None
    for p in all_paths(m, n):
        if all(_allowed(i, j, lo, hi, row0_hi, col0_hi) for i, j in _path_cells(p)):
            s = path_score(p, a, b, *sc)
            best = s if best is None else max(best, s)
    got = oracle.region(a, b, lo, hi, row0_hi, col0_hi, *sc)
    assert got == (best if best is not None else oracle.NEG_INF)


@pytest.mark.parametrize("seed", range(6))
def test_region_dp_reduces_to_full_and_band(seed):
    """Whole grid -> full NW; exactly the band -> the banded DP."""
    p = seqgen.long_mutated_pair(500 + seed, m=150 + 37 * seed)
    a, b = p.a, p.b
    m, n = a.size, b.size
    full = oracle.region(a, b, np.ones(m, np.int64), np.full(m, n, np.int64), n, m)
    assert full == oracle.score(a, b)
    for w in (0, 3, 20):
        lo_d, hi_d = oracle.band_limits(m, n, w)
        i = np.arange(1, m + 1)
        lo = np.maximum(1, i + lo_d)
        hi = np.minimum(n, i + hi_d)
        sb, _ = oracle.banded(a, b, w)
        got = oracle.region(a, b, lo, hi, max(0, hi_d), max(0, -lo_d))
        assert got == sb, w


@pytest.mark.parametrize("seed", range(6))
def test_certificate_soundness_and_next_width_guarantee(seed):
    """Reading 9 by brute force on small pairs: a certified banded score
    equals the full score, and after a failed round the next width's round
    certifies (its banded score is no lower, and the same score already
    clears that width's bound)."""
    rng = np.random.default_rng(600 + seed)
    for _ in range(40):
        m, n = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        a = rng.integers(0, 4, m).astype(np.uint8)
        b = a[: n].copy() if n <= m else np.concatenate([a, rng.integers(0, 4, n - m).astype(np.uint8)])
        mut = rng.random(n) < 0.3
        b[mut] = rng.integers(0, 4, int(mut.sum())).astype(np.uint8)
        full = oracle.score(a, b)
        for want in (False, True):
            for w in range(0, 6):
                sb, _ = oracle.banded(a, b, w)
                if oracle.certifies(m, n, w, sb, want):
                    assert sb == full, (seed, m, n, w)
                else:
                    w2 = oracle.next_width(m, n, w, sb, want)
                    assert w2 >= 2 * w and w2 > w
                    sb2, _ = oracle.banded(a, b, w2)
                    assert sb2 >= sb
                    if w2 <= max(m, n):
                        assert oracle.certifies(m, n, w2, sb2, want)
                        assert sb2 == full
