"""CPU oracle for the Needleman-Wunsch path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2412_21103_gb300`` never imports it and shares no code with it.

``nw_oracle.c`` holds the plain full-matrix dynamic programme (Sec. 2.1-2.4 of
the paper, Eq. 1 read as standard NW) and is compiled here with gcc into
``oracle/_build/libnw_oracle.so``.  The Python helpers below only marshal
arguments and run-length encode the op string.

Functions whose result the paper or mathematics pins (see ``tests/``):
  fill / score / align  -- brute force over all alignments, closed forms,
                           Levenshtein and LCS special cases, invariants,
                           hand-worked grids in ``tests/golden``.
  banded                -- equals full NW for a band covering the grid;
                           brute force over in-band paths; the bound U is
                           checked against brute force over out-of-band paths.
  exit_bound (U0)       -- brute force over every path that leaves the band.
  affine_*              -- affine gaps (Gotoh, not in the paper): brute force
                           over every alignment with gap runs scored open +
                           length * extend, reduction to the linear oracle when
                           the open cost is 0, closed forms.
  local_*               -- local alignment (Smith-Waterman, not in the paper):
                           brute force over every pair of substrings and every
                           alignment, longest common substring special case,
                           invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nw_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libnw_oracle.so")
_lock = threading.Lock()
_lib = None

NEG_INF = -(2 ** 31) // 2   # INT32_MIN / 2, the banded "-inf"


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vector extensions)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64 = ctypes.c_int64
            i32 = ctypes.c_int32
            lib.nwo_fill.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i32p]
            lib.nwo_align.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i32p, ctypes.c_char_p,
                                      ctypes.POINTER(i64)]
            lib.nwo_score.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i32p]
            lib.nwo_banded.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i64, i32p, i32p, i32p]
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.nwo_region.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i64p, i64p, i64, i64, i32p]
            lib.nwo_local_fill.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i32p]
            lib.nwo_local_align.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i32p, i64p, ctypes.c_char_p,
                                            ctypes.POINTER(i64)]
            lib.nwo_local_score.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i32p]
            lib.nwo_affine_fill.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i32, i32p, i32p, i32p]
            lib.nwo_affine_align.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i32, i32p, ctypes.c_char_p,
                                             ctypes.POINTER(i64)]
            lib.nwo_affine_score.argtypes = [u8p, i64, u8p, i64, i32, i32, i32, i32, i32p]
            for f in (lib.nwo_fill, lib.nwo_align, lib.nwo_score, lib.nwo_banded, lib.nwo_region, lib.nwo_local_fill,
                      lib.nwo_local_align, lib.nwo_local_score, lib.nwo_affine_fill, lib.nwo_affine_align,
                      lib.nwo_affine_score):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _codes(x) -> np.ndarray:
    if isinstance(x, str):
        lut = {"A": 0, "C": 1, "G": 2, "T": 3}
        return np.array([lut[c] for c in x.upper()], dtype=np.uint8)
    arr = np.ascontiguousarray(np.asarray(x, dtype=np.uint8))
    if arr.size and arr.max() > 3:
        raise ValueError("base codes must be 0..3")
    return arr


def _ptr(arr: np.ndarray, ctype=ctypes.c_uint8):
    if arr.size == 0:
        arr = np.zeros(1, dtype=arr.dtype)
    return arr.ctypes.data_as(ctypes.POINTER(ctype)), arr


def fill(a, b, match: int = 1, mismatch: int = -1, gap: int = -1) -> np.ndarray:
    """The full (m+1) x (n+1) score grid H."""
    a, b = _codes(a), _codes(b)
    H = np.empty((a.size + 1, b.size + 1), dtype=np.int32)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    rc = _load().nwo_fill(pa, a.size, pb, b.size, match, mismatch, gap,
                          H.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert rc == 0, rc
    return H


def score(a, b, match: int = 1, mismatch: int = -1, gap: int = -1) -> int:
    a, b = _codes(a), _codes(b)
    out = ctypes.c_int32(0)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    rc = _load().nwo_score(pa, a.size, pb, b.size, match, mismatch, gap, ctypes.byref(out))
    assert rc == 0, rc
    return int(out.value)


def align(a, b, match: int = 1, mismatch: int = -1, gap: int = -1) -> tuple[int, str]:
    """(score, op string over '=XID' in forward order)."""
    a, b = _codes(a), _codes(b)
    out = ctypes.c_int32(0)
    nops = ctypes.c_int64(0)
    buf = ctypes.create_string_buffer(a.size + b.size + 1)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    rc = _load().nwo_align(pa, a.size, pb, b.size, match, mismatch, gap, ctypes.byref(out), buf,
                           ctypes.byref(nops))
    if rc == -2:
        raise MemoryError("oracle grid does not fit in host memory")
    assert rc == 0, rc
    return int(out.value), buf.raw[: nops.value].decode()


def banded(a, b, w: int, match: int = 1, mismatch: int = -1, gap: int = -1,
           want_grid: bool = False):
    """(S_b, U) for half-width w, plus the banded grid when asked."""
    a, b = _codes(a), _codes(b)
    sb = ctypes.c_int32(0)
    ub = ctypes.c_int32(0)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    H = np.empty((a.size + 1, b.size + 1), dtype=np.int32) if want_grid else None
    hp = H.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if want_grid else None
    rc = _load().nwo_banded(pa, a.size, pb, b.size, match, mismatch, gap, w, ctypes.byref(sb),
                            ctypes.byref(ub), hp)
    assert rc == 0, rc
    if want_grid:
        return int(sb.value), int(ub.value), H
    return int(sb.value), int(ub.value)


def region(a, b, row_lo, row_hi, row0_hi: int, col0_hi: int, match: int = 1, mismatch: int = -1,
           gap: int = -1) -> int:
    """Score of the DP restricted to a cell set: row i (1-based) may use
    columns row_lo[i-1]..row_hi[i-1], row 0 columns 0..row0_hi, column 0 rows
    0..col0_hi; everything else is -infinity (NEG_INF when unreachable)."""
    a, b = _codes(a), _codes(b)
    lo = np.ascontiguousarray(row_lo, dtype=np.int64)
    hi = np.ascontiguousarray(row_hi, dtype=np.int64)
    assert lo.size == a.size and hi.size == a.size
    sc = ctypes.c_int32(0)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    i64p = ctypes.POINTER(ctypes.c_int64)
    rc = _load().nwo_region(pa, a.size, pb, b.size, match, mismatch, gap, lo.ctypes.data_as(i64p),
                            hi.ctypes.data_as(i64p), row0_hi, col0_hi, ctypes.byref(sc))
    assert rc == 0, rc
    return int(sc.value)


def band_limits(m: int, n: int, w: int) -> tuple[int, int]:
    """Diagonals d = j - i of the band of half-width w: [min(0,n-m)-w, max(0,n-m)+w]."""
    delta = n - m
    return min(0, delta) - w, max(0, delta) + w


def exit_bound(m: int, n: int, w: int, match: int = 1, gap: int = -1) -> int | None:
    """Closed-form bound U0 on the score of any path that leaves the band
    (None when no path can leave it).  A path from diagonal 0 to diagonal
    n-m that visits diagonal hi+1 needs at least (hi+1) + (hi+1-(n-m)) gap
    moves; one that visits lo-1 needs (1-lo) + ((n-m)-lo+1).  A path with G
    gap moves has (m+n-G)/2 diagonal moves, each worth at most `match`, so
    its score is at most match*(m+n-G)/2 + gap*G, which falls as G grows
    (match >= 0 >= gap); the parity of m+n-G is kept exact."""
    lo, hi = band_limits(m, n, w)
    delta = n - m
    best = None
    for g_min in ((hi + 1) + (hi + 1 - delta), (1 - lo) + (delta - lo + 1)):
        if g_min > m + n:
            continue
        # paths need both ends inside the grid: the excursion must fit
        if g_min == (hi + 1) + (hi + 1 - delta) and hi + 1 > n:
            continue
        if g_min == (1 - lo) + (delta - lo + 1) and 1 - lo > m:
            continue
        k = (m + n - g_min) // 2
        val = match * k + gap * (m + n - 2 * k)
        best = val if best is None else max(best, val)
    return best


def certifies(m: int, n: int, w: int, banded_score: int, want_cigar: bool, match: int = 1, gap: int = -1) -> bool:
    """The certificate on a banded score (not in the paper; the design's
    reading of banded exactness): no path can leave the band, or the banded
    score beats every path that does -- at least equal for the score, strictly
    above for the alignment (an equal path outside the band could win the
    diagonal-first tie order)."""
    U = exit_bound(m, n, w, match, gap)
    if U is None:
        return True
    return banded_score > U if want_cigar else banded_score >= U


def next_width(m: int, n: int, w: int, banded_score: int, want_cigar: bool, match: int = 1, gap: int = -1) -> int:
    """Half-width of the next banded round after `banded_score` failed at w:
    the first w' > w (scanning upward, at most max(m,n)+1) at which the same
    banded score would certify -- a wider band scores no less, so the round
    at w' certifies -- and at least 2w."""
    wp = w + 1
    while wp <= max(m, n) and not certifies(m, n, wp, banded_score, want_cigar, match, gap):
        wp += 1
    return max(2 * w, wp)


def local_fill(a, b, match: int = 1, mismatch: int = -1, gap: int = -1) -> np.ndarray:
    """The full (m+1) x (n+1) local-alignment grid H (floor 0)."""
    a, b = _codes(a), _codes(b)
    H = np.empty((a.size + 1, b.size + 1), dtype=np.int32)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    rc = _load().nwo_local_fill(pa, a.size, pb, b.size, match, mismatch, gap,
                                H.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert rc == 0, rc
    return H


def local_align(a, b, match: int = 1, mismatch: int = -1, gap: int = -1):
    """(score, (i_start, j_start, i_end, j_end), op string): the local
    alignment covers A[i_start:i_end] and B[j_start:j_end]."""
    a, b = _codes(a), _codes(b)
    out = ctypes.c_int32(0)
    ends = (ctypes.c_int64 * 4)()
    nops = ctypes.c_int64(0)
    buf = ctypes.create_string_buffer(a.size + b.size + 1)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    rc = _load().nwo_local_align(pa, a.size, pb, b.size, match, mismatch, gap, ctypes.byref(out), ends, buf,
                                 ctypes.byref(nops))
    if rc == -2:
        raise MemoryError("oracle grid does not fit in host memory")
    assert rc == 0, rc
    return int(out.value), tuple(int(x) for x in ends), buf.raw[: nops.value].decode()


def local_score(a, b, match: int = 1, mismatch: int = -1, gap: int = -1) -> int:
    a, b = _codes(a), _codes(b)
    out = ctypes.c_int32(0)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    rc = _load().nwo_local_score(pa, a.size, pb, b.size, match, mismatch, gap, ctypes.byref(out))
    assert rc == 0, rc
    return int(out.value)


def local_align_many(pairs, match: int = 1, mismatch: int = -1, gap: int = -1, threads: int | None = None):
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda p: local_align(p[0], p[1], match, mismatch, gap), pairs))


def local_score_many(pairs, match: int = 1, mismatch: int = -1, gap: int = -1, threads: int | None = None):
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda p: local_score(p[0], p[1], match, mismatch, gap), pairs))


def affine_fill(a, b, match: int = 1, mismatch: int = -1, gap_open: int = -2, gap_extend: int = -1):
    """The three (m+1) x (n+1) grids H, E, F of affine-gap global alignment."""
    a, b = _codes(a), _codes(b)
    grids = [np.empty((a.size + 1, b.size + 1), dtype=np.int32) for _ in range(3)]
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    i32p = ctypes.POINTER(ctypes.c_int32)
    rc = _load().nwo_affine_fill(pa, a.size, pb, b.size, match, mismatch, gap_open, gap_extend,
                                 *[g.ctypes.data_as(i32p) for g in grids])
    assert rc == 0, rc
    return tuple(grids)


def affine_align(a, b, match: int = 1, mismatch: int = -1, gap_open: int = -2, gap_extend: int = -1):
    """(score, op string) of affine-gap global alignment."""
    a, b = _codes(a), _codes(b)
    out = ctypes.c_int32(0)
    nops = ctypes.c_int64(0)
    buf = ctypes.create_string_buffer(a.size + b.size + 1)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    rc = _load().nwo_affine_align(pa, a.size, pb, b.size, match, mismatch, gap_open, gap_extend, ctypes.byref(out),
                                  buf, ctypes.byref(nops))
    if rc == -2:
        raise MemoryError("oracle grids do not fit in host memory")
    assert rc == 0, rc
    return int(out.value), buf.raw[: nops.value].decode()


def affine_score(a, b, match: int = 1, mismatch: int = -1, gap_open: int = -2, gap_extend: int = -1) -> int:
    a, b = _codes(a), _codes(b)
    out = ctypes.c_int32(0)
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    rc = _load().nwo_affine_score(pa, a.size, pb, b.size, match, mismatch, gap_open, gap_extend, ctypes.byref(out))
    assert rc == 0, rc
    return int(out.value)


def affine_align_many(pairs, match: int = 1, mismatch: int = -1, gap_open: int = -2, gap_extend: int = -1,
                      threads: int | None = None):
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda p: affine_align(p[0], p[1], match, mismatch, gap_open, gap_extend), pairs))


def affine_score_many(pairs, match: int = 1, mismatch: int = -1, gap_open: int = -2, gap_extend: int = -1,
                      threads: int | None = None):
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda p: affine_score(p[0], p[1], match, mismatch, gap_open, gap_extend), pairs))


def rle(ops: str) -> str:
    """Run-length encode an op string into a CIGAR ('3=1X2I')."""
    if not ops:
        return ""
    out = []
    prev = ops[0]
    cnt = 0
    for c in ops:
        if c == prev:
            cnt += 1
        else:
            out.append(f"{cnt}{prev}")
            prev, cnt = c, 1
    out.append(f"{cnt}{prev}")
    return "".join(out)


def score_many(pairs, match: int = 1, mismatch: int = -1, gap: int = -1, threads: int | None = None):
    """Scores of many (a, b) pairs on a pool of host threads (the C call
    releases the GIL)."""
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda p: score(p[0], p[1], match, mismatch, gap), pairs))


def align_many(pairs, match: int = 1, mismatch: int = -1, gap: int = -1, threads: int | None = None):
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda p: align(p[0], p[1], match, mismatch, gap), pairs))
