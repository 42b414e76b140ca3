"""Seeded synthetic DNA workloads.

This module is shared by the tests, the benchmark and the CPU oracle's
callers.  It holds no alignment arithmetic: it only draws random bases and
mutation events and records which edit it applied (the transcript), so that a
caller can score that transcript itself.

Random numbers come from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): value k
of stream ``key`` is ``mix64(key + (k + 1) * 0x9E3779B97F4A7C15)``.  Being
counter-based it vectorises in numpy and gives identical values on x86 and Arm.

Base codes: A=0, C=1, G=2, T=3.  Transcript ops, with A the query (DP rows)
and B the reference (DP columns): ``=`` match, ``X`` substitution, ``I`` a base
of A absent from B, ``D`` a base of B absent from A.

Workload recipes (the paper's COL1A1/THAP11 gene pairs are not available, so
these synthetic shapes stand in for them):

* ``random_pair``         i.i.d. uniform A and B (1,000 x 1,000 single pair).
* ``long_mutated_pair``   A uniform; B from A with per-position substitution
                          probability 0.10 and indel-start probability 0.02,
                          geometric indel lengths (mean 3) -- the long pair.
* ``all_vs_all_family``   512 mutants of one random root, lengths U{500..1500},
                          divergence U[0.05, 0.30], 80% substitutions and 20%
                          1-bp indels at distinct positions.
* ``band_pairs``          lengths log-uniform in [2,000, 20,000], divergence
                          U[0.01, 0.25], geometric indels, and with probability
                          0.3 one to three indel bursts of 50..500 bp.
* ``serving_stream``      Poisson arrivals; lengths log-uniform in [50, 50,000];
                          divergence U[0.01, 0.30]; half score-only requests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1

BASES = "ACGT"


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrap-around arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _mix64_int(z: int) -> int:
    z &= _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


class Stream:
    """One counter-based SplitMix64 stream, keyed by (seed, tag)."""

    def __init__(self, seed: int, tag: int = 0):
        self.key = _mix64_int((int(seed) * 0xD1B54A32D192ED03 + int(tag) * 0x8CB92BA72F3D8DD7 + 1) & _MASK)
        self.ctr = 0

    def u64(self, count: int) -> np.ndarray:
        idx = np.arange(self.ctr + 1, self.ctr + 1 + count, dtype=np.uint64)
        self.ctr += count
        with np.errstate(over="ignore"):
            z = np.uint64(self.key) + idx * _GOLDEN
        return _mix64(z)

    def uniform(self, count: int) -> np.ndarray:
        """Floats in [0, 1) with 53 random bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Integers uniform in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return lo + np.minimum((self.uniform(count) * span).astype(np.int64), span - 1)

    def bases(self, count: int) -> np.ndarray:
        """Uniform base codes 0..3 (top two bits of each draw)."""
        return (self.u64(count) >> np.uint64(62)).astype(np.uint8)

    def geometric(self, p: float, count: int) -> np.ndarray:
        """Geometric on {1, 2, ...} with success probability p (mean 1/p)."""
        u = self.uniform(count)
        return 1 + np.floor(np.log1p(-u) / math.log1p(-p)).astype(np.int64)

    def child(self, tag: int) -> "Stream":
        return Stream(self.key ^ 0x5851F42D4C957F2D, tag)


def to_ascii(codes: np.ndarray) -> str:
    return np.frombuffer(np.frombuffer(b"ACGT", dtype=np.uint8)[codes].tobytes(), dtype="S1").tobytes().decode()


def from_ascii(s: str) -> np.ndarray:
    lut = np.full(256, 255, dtype=np.uint8)
    for k, ch in enumerate(BASES):
        lut[ord(ch)] = k
        lut[ord(ch.lower())] = k
    out = lut[np.frombuffer(s.encode(), dtype=np.uint8)]
    if (out == 255).any():
        raise ValueError("sequence contains a non-ACGT character")
    return out


@dataclass
class Pair:
    a: np.ndarray                  # query codes (rows)
    b: np.ndarray                  # reference codes (columns)
    transcript: str | None = None  # the edit the generator applied, '=XID' ops


def _apply_edits(a: np.ndarray, rs: Stream, sub: np.ndarray, dele: np.ndarray, ins_len: np.ndarray):
    """Build B from A.

    ``sub``: bool per position (substitute), ``dele``: bool per position
    (drop from B), ``ins_len``: number of random bases inserted after the
    position.  Returns (b, transcript)."""
    m = a.shape[0]
    shift = rs.integers(1, 3, m).astype(np.uint8)
    newbase = np.where(sub & ~dele, (a + shift) % 4, a).astype(np.uint8)
    keep = (~dele).astype(np.int64)
    per_pos = keep + ins_len
    total = int(per_pos.sum())
    b = np.empty(total, dtype=np.uint8)
    ops = np.empty(m + int(ins_len.sum()), dtype="S1")
    # positions of kept bases in b
    starts = np.concatenate([[0], np.cumsum(per_pos)[:-1]]).astype(np.int64)
    kept_idx = np.nonzero(keep)[0]
    b[starts[kept_idx]] = newbase[kept_idx]
    ins_total = int(ins_len.sum())
    if ins_total:
        ins_bases = rs.bases(ins_total)
        owner = np.repeat(np.arange(m), ins_len)
        within = np.arange(ins_total) - np.repeat(np.cumsum(ins_len) - ins_len, ins_len)
        b[starts[owner] + keep[owner] + within] = ins_bases
    # transcript: per position one of = X I, then 'D' * ins_len
    op_pos = np.where(dele, b"I", np.where(sub, b"X", b"="))
    ostarts = np.concatenate([[0], np.cumsum(1 + ins_len)[:-1]]).astype(np.int64)
    ops[ostarts] = op_pos
    if ins_total:
        ops[ostarts[owner] + 1 + within] = b"D"
    return b, ops.tobytes().decode()


def random_pair(seed: int, m: int = 1000, n: int = 1000) -> Pair:
    rs = Stream(seed, 1)
    return Pair(rs.bases(m), rs.bases(n), None)


def long_mutated_pair(seed: int, m: int = 32768, p_sub: float = 0.10, p_indel: float = 0.02,
                      indel_mean: float = 3.0) -> Pair:
    """A uniform of length m; B derived from A by per-position substitutions
    (probability p_sub) and indel starts (probability p_indel, 50/50 insertion
    or deletion, geometric length with the given mean)."""
    rs = Stream(seed, 2)
    a = rs.bases(m)
    u_ev = rs.uniform(m)
    u_kind = rs.uniform(m)
    lens = rs.geometric(1.0 / indel_mean, m)
    indel = u_ev < p_indel
    is_ins = indel & (u_kind < 0.5)
    is_del = indel & ~is_ins
    sub = (~indel) & (u_ev < p_indel + p_sub)
    dele = np.zeros(m, dtype=bool)
    for p in np.nonzero(is_del)[0]:  # sparse: about p_indel/2 * m events
        dele[p:p + int(lens[p])] = True
    ins_len = np.where(is_ins & ~dele, lens, 0).astype(np.int64)
    sub &= ~dele
    b, tr = _apply_edits(a, rs, sub, dele, ins_len)
    return Pair(a, b, tr)


def mutate_distinct(a: np.ndarray, rs: Stream, delta: float, indel_frac: float = 0.2,
                    indel_mean: float | None = None, bursts: int = 0,
                    burst_range: tuple[int, int] = (50, 500)) -> tuple[np.ndarray, str]:
    """round(delta * len) mutations at distinct positions: a fraction
    ``indel_frac`` are indels (50/50 insertion/deletion, 1 bp, or geometric with
    ``indel_mean`` when given), the rest substitutions; then ``bursts``
    contiguous indel bursts with lengths uniform in ``burst_range``."""
    m = a.shape[0]
    k = min(m, int(round(delta * m)))
    order = np.argsort(rs.u64(m), kind="stable")
    pos = order[:k]
    kind = rs.uniform(k)
    lens = rs.geometric(1.0 / indel_mean, k) if indel_mean else np.ones(k, dtype=np.int64)
    sub = np.zeros(m, dtype=bool)
    dele = np.zeros(m, dtype=bool)
    ins_len = np.zeros(m, dtype=np.int64)
    is_indel = kind < indel_frac
    is_ins = is_indel & (kind < indel_frac / 2)
    sub[pos[~is_indel]] = True
    ins_len[pos[is_ins]] = lens[is_ins]
    for p, ln in zip(pos[is_indel & ~is_ins], lens[is_indel & ~is_ins]):
        dele[p:p + int(ln)] = True
    if bursts:
        bpos = rs.integers(0, max(m - 1, 0), bursts)
        blen = rs.integers(burst_range[0], burst_range[1], bursts)
        bkind = rs.uniform(bursts)
        for p, ln, kd in zip(bpos, blen, bkind):
            if kd < 0.5:
                ins_len[p] += int(ln)
            else:
                dele[p:p + int(ln)] = True
    sub &= ~dele
    ins_len[dele] = 0
    return _apply_edits(a, rs, sub, dele, ins_len)


def all_vs_all_family(seed: int, nseq: int = 512, root_len: int = 1500, lmin: int = 500, lmax: int = 1500,
                      dmin: float = 0.05, dmax: float = 0.30) -> list[np.ndarray]:
    """nseq mutants of one random root (the multiple-sequence workload)."""
    rs = Stream(seed, 3)
    root = rs.bases(root_len)
    lens = rs.integers(lmin, lmax, nseq)
    deltas = dmin + (dmax - dmin) * rs.uniform(nseq)
    out = []
    for k in range(nseq):
        child = rs.child(k)
        b, _ = mutate_distinct(root[: int(lens[k])], child, float(deltas[k]))
        out.append(b)
    return out


def band_pairs(seed: int, npairs: int = 20000, lmin: int = 2000, lmax: int = 20000, dmin: float = 0.01,
               dmax: float = 0.25, p_burst: float = 0.3) -> list[Pair]:
    """Pairs for the certified learned-band workload."""
    rs = Stream(seed, 4)
    lens = np.round(np.exp(math.log(lmin) + (math.log(lmax) - math.log(lmin)) * rs.uniform(npairs))).astype(np.int64)
    deltas = dmin + (dmax - dmin) * rs.uniform(npairs)
    has_burst = rs.uniform(npairs) < p_burst
    nburst = rs.integers(1, 3, npairs)
    out = []
    for k in range(npairs):
        child = rs.child(k)
        a = child.bases(int(lens[k]))
        b, tr = mutate_distinct(a, child, float(deltas[k]), indel_mean=3.0,
                                bursts=int(nburst[k]) if has_burst[k] else 0)
        out.append(Pair(a, b, tr))
    return out


@dataclass
class Request:
    t_arrival: float     # seconds since the start of the stream
    pair: Pair
    want_cigar: bool


def serving_stream(seed: int, rate: float = 50000.0, duration: float = 60.0, lmin: int = 50, lmax: int = 50000,
                   dmin: float = 0.01, dmax: float = 0.30, limit: int | None = None):
    """Yield requests of a Poisson stream (exponential inter-arrival times)."""
    rs = Stream(seed, 5)
    t = 0.0
    k = 0
    while True:
        if limit is not None and k >= limit:
            return
        u = rs.uniform(4)
        t += -math.log1p(-u[0]) / rate
        if t >= duration:
            return
        m = int(round(math.exp(math.log(lmin) + (math.log(lmax) - math.log(lmin)) * u[1])))
        delta = dmin + (dmax - dmin) * u[2]
        child = rs.child(k)
        a = child.bases(m)
        b, tr = mutate_distinct(a, child, delta, indel_mean=3.0)
        yield Request(t, Pair(a, b, tr), bool(u[3] < 0.5))
        k += 1


def local_pairs(seed: int, npairs: int = 4000, ref_min: int = 2000, ref_max: int = 10000, win_min: int = 200,
                win_max: int = 2000, flank_max: int = 500, dmin: float = 0.01, dmax: float = 0.20) -> list[Pair]:
    """Pairs for local alignment: B (the reference, columns) is random with a
    length uniform in [ref_min, ref_max]; A (the query, rows) is a mutated
    copy of a window of B (length uniform in [win_min, min(win_max, len B)],
    divergence U[dmin, dmax], geometric indels of mean 3) between random
    flanks of up to flank_max bases on each side."""
    rs = Stream(seed, 6)
    out = []
    for k in range(npairs):
        child = rs.child(k)
        nb = int(child.integers(ref_min, ref_max, 1)[0])
        b = child.bases(nb)
        w = int(child.integers(min(win_min, nb), min(win_max, nb), 1)[0])
        p0 = int(child.integers(0, nb - w, 1)[0])
        core, _ = mutate_distinct(b[p0:p0 + w], child, float(dmin + (dmax - dmin) * child.uniform(1)[0]),
                                  indel_mean=3.0)
        left, right = (int(x) for x in child.integers(0, flank_max, 2))
        a = np.concatenate([child.bases(left), core, child.bases(right)]).astype(np.uint8)
        out.append(Pair(a, b, None))
    return out
