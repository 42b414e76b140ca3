"""Independent checks used to pin the oracle and to check the GPU path.

Nothing here shares code with ``oracle/`` or with the library: brute-force
enumeration, bit-parallel edit distance and LCS, CIGAR parsing and re-scoring.
"""
from __future__ import annotations

import os
import re
from functools import lru_cache

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
LUT = {"A": 0, "C": 1, "G": 2, "T": 3}


def codes(s: str) -> np.ndarray:
    return np.array([LUT[c] for c in s], dtype=np.uint8)


def ascii_of(c) -> str:
    return "".join("ACGT"[int(x)] for x in c)


# ---------------------------------------------------------------- CIGAR ----
def parse_cigar(cigar: str) -> str:
    """'3=1X' -> '===X'."""
    out = []
    for cnt, op in re.findall(r"(\d+)([=XIDM])", cigar):
        out.append(op * int(cnt))
    joined = "".join(out)
    assert len(re.sub(r"\d+[=XIDM]", "", cigar)) == 0, f"bad cigar {cigar!r}"
    return joined


def consumed(ops: str) -> tuple[int, int]:
    qa = sum(1 for o in ops if o in "=XMI")
    rb = sum(1 for o in ops if o in "=XMD")
    return qa, rb


def rescore(ops: str, a, b, match: int, mismatch: int, gap: int) -> int:
    """Score of an explicit alignment; also checks that '='/'X' agree with the
    sequences and that both sequences are consumed exactly."""
    i = j = 0
    total = 0
    for o in ops:
        if o in "=X":
            eq = int(a[i]) == int(b[j])
            assert eq == (o == "="), f"op {o} at ({i},{j}) disagrees with the bases"
            total += match if eq else mismatch
            i += 1
            j += 1
        elif o == "I":
            total += gap
            i += 1
        elif o == "D":
            total += gap
            j += 1
        else:
            raise AssertionError(f"unexpected op {o}")
    assert i == len(a) and j == len(b), "alignment does not consume both sequences"
    return total


# ---------------------------------------------------------- brute force ----
def all_paths(m: int, n: int):
    """Every monotone path (0,0)->(m,n) as a forward move string over
    'd' (diagonal), 'u' (vertical: A_i alone), 'l' (horizontal: B_j alone)."""
    @lru_cache(maxsize=None)
    def rec(i, j):
        if i == m and j == n:
            return [""]
        out = []
        if i < m and j < n:
            out += ["d" + s for s in rec(i + 1, j + 1)]
        if i < m:
            out += ["u" + s for s in rec(i + 1, j)]
        if j < n:
            out += ["l" + s for s in rec(i, j + 1)]
        return out
    return rec(0, 0)


def path_score(path: str, a, b, match, mismatch, gap) -> int:
    i = j = 0
    s = 0
    for mv in path:
        if mv == "d":
            s += match if a[i] == b[j] else mismatch
            i += 1
            j += 1
        elif mv == "u":
            s += gap
            i += 1
        else:
            s += gap
            j += 1
    return s


def brute_force(a, b, match, mismatch, gap):
    """(best score, the optimal path whose reversed move string is
    lexicographically greatest under diagonal > vertical > horizontal)."""
    rank = {"d": "2", "u": "1", "l": "0"}
    best = None
    best_key = None
    best_path = None
    for p in all_paths(len(a), len(b)):
        s = path_score(p, a, b, match, mismatch, gap)
        key = "".join(rank[c] for c in reversed(p))
        if best is None or s > best or (s == best and key > best_key):
            best, best_key, best_path = s, key, p
    return best, best_path


def ops_to_moves(ops: str) -> str:
    return "".join("d" if o in "=X" else ("u" if o == "I" else "l") for o in ops)


# ------------------------------------------------- bit-parallel checks ----
def levenshtein_myers(a, b) -> int:
    """Global unit-cost edit distance with Myers' bit-vector algorithm
    (Myers 1999, in Hyyro's global-distance form: the row-0 horizontal delta
    is +1, carried in by OR-ing 1 into the shifted Ph)."""
    m = len(a)
    if m == 0:
        return len(b)
    mask = (1 << m) - 1
    top = 1 << (m - 1)
    peq = {c: 0 for c in range(4)}
    for i, c in enumerate(a):
        peq[int(c)] |= 1 << i
    pv, mv, dist = mask, 0, m
    for c in b:
        eq = peq[int(c)]
        xv = eq | mv
        xh = ((((eq & pv) + pv) & mask) ^ pv) | eq
        ph = (mv | ~(xh | pv)) & mask
        mh = pv & xh
        if ph & top:
            dist += 1
        elif mh & top:
            dist -= 1
        ph = ((ph << 1) | 1) & mask
        mh = (mh << 1) & mask
        pv = (mh | ~(xv | ph)) & mask
        mv = ph & xv
    return dist


def lcs_bitparallel(a, b) -> int:
    """LCS length with the bit-vector recurrence V' = (V + U) | (V - U),
    U = V & match-mask (Allison-Dix 1986 / Hyyro 2004)."""
    m = len(a)
    if m == 0:
        return 0
    mask = (1 << m) - 1
    peq = {c: 0 for c in range(4)}
    for i, c in enumerate(a):
        peq[int(c)] |= 1 << i
    v = mask
    for c in b:
        u = v & peq[int(c)]
        v = ((v + u) | (v - u)) & mask
    return m - bin(v).count("1")


def lcs_brute(a, b) -> int:
    """LCS by enumerating subsequences of the shorter sequence (tiny inputs)."""
    from itertools import combinations
    if len(a) > len(b):
        a, b = b, a
    a = list(map(int, a))
    b = list(map(int, b))

    def is_subseq(s):
        it = iter(b)
        return all(any(x == y for y in it) for x in s)
    for k in range(len(a), -1, -1):
        for idx in combinations(range(len(a)), k):
            if is_subseq([a[i] for i in idx]):
                return k
    return 0


# --------------------------------------------------------------- golden ----
def load_hand_grids():
    path = os.path.join(GOLDEN, "hand_grids.txt")
    text = open(path).read()
    cases = []
    for block in re.split(r"\n\s*\n", text):
        lines = [ln for ln in block.strip().splitlines() if ln and not ln.startswith("#")]
        if not lines or not lines[0].startswith("case:"):
            continue
        d = {}
        k = 0
        while k < len(lines):
            ln = lines[k]
            if ln.startswith("grid:"):
                d["grid"] = [list(map(int, r.split())) for r in lines[k + 1:]]
                break
            key, _, val = ln.partition(":")
            d[key.strip()] = val.strip()
            k += 1
        d["scoring"] = tuple(map(int, d["scoring"].split()))
        d["score"] = int(d["score"])
        cases.append(d)
    return cases
