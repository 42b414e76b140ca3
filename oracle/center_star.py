"""CPU reference of the center-star multiple alignment -- TEST
INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``: only tests, the
smoke check and the benchmark's CPU legs use it).

Sec. 3.2 of the paper: a scoring matrix of every pair of sequences (the
n(n-1)/2 alignments of Eq. 2), the center = the sequence most similar to the
rest through that matrix, every sequence aligned with the center, then the
pairwise alignments merged with the aligned center as the reference.

Readings taken where the paper is silent:
  * "most similar to the rest" = the largest sum of a sequence's scores
    against the other sequences (its row of the score matrix without the
    diagonal entry len * match, which would favour long sequences and says
    nothing about the rest); ties go to the lowest index.
  * each sequence k is aligned as the query (rows, A) against the center as
    the reference (columns, B) with the global alignment of Sec. 2 and its
    diagonal > vertical > horizontal order; the center against itself is
    that alignment too (all matches).
  * merge ("once a gap, always a gap"): before center base p (p = 0..|C|;
    p = |C| is after the last base) the merged alignment keeps
    G[p] = max over k of the number of 'I' ops (bases of sequence k facing
    no center base) that alignment k places there; the center's base p
    lands in column p + G[0] + ... + G[p]; in a row, the I-bases of slot p
    fill the slot from its left and the rest of the slot is '-'; a 'D' op
    (center base facing no base of sequence k) leaves '-' in the center's
    column.
"""
from __future__ import annotations

import numpy as np

from . import align_many, score_many

GAP_CHAR = "-"
BASES = "ACGT"


def score_matrix(seqs, match: int = 1, mismatch: int = -1, gap: int = -1) -> np.ndarray:
    """All-vs-all global alignment scores (Sec. 3.2 scoring matrix), int64,
    symmetric, diagonal len * match."""
    n = len(seqs)
    M = np.zeros((n, n), np.int64)
    iu, ju = np.triu_indices(n, 1)
    vals = score_many([(seqs[i], seqs[j]) for i, j in zip(iu.tolist(), ju.tolist())], match, mismatch, gap)
    M[iu, ju] = vals
    M[ju, iu] = vals
    for i, s in enumerate(seqs):
        M[i, i] = len(s) * match
    return M


def choose_center(M: np.ndarray) -> tuple[int, np.ndarray]:
    """(center index, row sums over the other sequences): the largest sum,
    lowest index on ties."""
    n = M.shape[0]
    sums = np.array([sum(int(M[i, j]) for j in range(n) if j != i) for i in range(n)], np.int64)
    return int(np.argmax(sums)), sums   # argmax returns the first maximum


def slot_gaps(ops_list, center_len: int) -> np.ndarray:
    """G[p] for p = 0..center_len: the most 'I' ops any alignment places
    before center base p."""
    G = np.zeros(center_len + 1, np.int64)
    for ops in ops_list:
        p = 0
        run = 0
        for o in ops:
            if o == "I":
                run += 1
            else:                      # '=', 'X' or 'D' consume center base p
                G[p] = max(G[p], run)
                run = 0
                p += 1
        G[p] = max(G[p], run)          # insertions after the last center base
    return G


def merge(seqs, center: int, ops_list) -> list[str]:
    """Rows of the merged alignment (strings over 'ACGT-')."""
    C = len(seqs[center])
    G = slot_gaps(ops_list, C)
    ncols = C + int(G.sum())
    col = np.zeros(C, np.int64)        # column of center base p
    start = np.zeros(C + 1, np.int64)  # first column of insertion slot p
    pos = 0
    for p in range(C + 1):
        start[p] = pos
        pos += int(G[p])
        if p < C:
            col[p] = pos
            pos += 1
    rows = []
    for s, ops in zip(seqs, ops_list):
        row = [GAP_CHAR] * ncols
        p = i = 0
        used = 0                       # I-bases written into slot p so far
        for o in ops:
            if o == "I":
                row[start[p] + used] = BASES[int(s[i])]
                used += 1
                i += 1
            elif o == "D":
                p += 1
                used = 0
            else:
                row[col[p]] = BASES[int(s[i])]
                i += 1
                p += 1
                used = 0
        rows.append("".join(row))
    return rows


def center_star(seqs, match: int = 1, mismatch: int = -1, gap: int = -1):
    """The whole method: (center, row sums, per-sequence (score, ops) against
    the center, merged rows)."""
    M = score_matrix(seqs, match, mismatch, gap)
    c, sums = choose_center(M)
    aligned = align_many([(s, seqs[c]) for s in seqs], match, mismatch, gap)
    rows = merge(seqs, c, [ops for _, ops in aligned])
    return c, sums, aligned, rows
