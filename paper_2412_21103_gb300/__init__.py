"""Python binding of libnw, the GB300 Needleman-Wunsch library.

Argument marshalling only: every step of the alignment runs in the CUDA
kernels behind the C ABI declared in ``include/nw.h``.  Device buffers are
torch CUDA tensors (torch is used for device memory and streams), host
buffers are numpy arrays.  If ``libnw.so`` has not been built this module
raises on first use; there is no CPU fallback.

Functions keep the C names: ``nw_pack``, ``nw_pack_device``, ``nw_align``,
``nw_align_batch``, ``nw_score_all_pairs``, ``nw_peak_int``; ``Context``
wraps ``nw_ctx``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

NW_OK = 0
NW_ERR_ARG = 1
NW_ERR_BAD_BASE = 2
NW_ERR_OOM = 3
NW_ERR_CIGAR_TRUNC = 4
NW_ERR_TIMEOUT = 5
NW_ERR_CUDA = 6
NW_ERR_UNSUPPORTED = 7
NW_ERR_BOUNDS = 8

NW_SCORE_ONLY = 0
NW_CIGAR = 1
NW_LEARNED_BAND = 2
NW_HOST_IO = 4
NW_CIGAR_M = 8
NW_BAND_RAW = 16
NW_RECOMPUTE = 32
NW_GRAPH = 64
NW_TEST_DROP_PROGRESS = 1

DEFAULT_SCORING = (1, -1, -1)

_lib = None


class NWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libnw status {status}: {msg}")
        self.status = status


class Scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap", ctypes.c_int32)]


class AffineScoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("score", ctypes.c_int32),
                ("cigar_len", ctypes.c_uint64), ("cigar_off", ctypes.c_uint64), ("latency_s", ctypes.c_double)]


def lib_path() -> str:
    """libnw.so, or the bounds-checked libnw_checks.so when the environment
    sets NW_CHECKS=1 before the first call."""
    return _build.CHECKS_LIB if os.environ.get("NW_CHECKS") == "1" else _build.LIB


def load():
    """Load libnw.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libnw.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
    u64p = ctypes.POINTER(ctypes.c_uint64)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    sig = {
        "nw_ctx_create": (vp, [ctypes.c_int, vp, u64]),
        "nw_ctx_destroy": (None, [vp]),
        "nw_ctx_set_stream": (ctypes.c_int, [vp, vp]),
        "nw_ctx_sync": (ctypes.c_int, [vp]),
        "nw_ctx_last_message": (ctypes.c_char_p, [vp]),
        "nw_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "nw_ctx_set_profiling": (ctypes.c_int, [vp, ctypes.c_int]),
        "nw_ctx_kernel_stats": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_char_p), u64p,
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
        "nw_ctx_reset_stats": (ctypes.c_int, [vp]),
        "nw_ctx_set_autotune": (ctypes.c_int, [vp, ctypes.c_int]),
        "nw_ctx_set_test_hook": (ctypes.c_int, [vp, u32]),
        "nw_ctx_tuning": (ctypes.c_int64, [vp, ctypes.c_char_p, u64]),
        "nw_ctx_set_tuning": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "nw_ctx_graph_stats": (ctypes.c_int, [vp, u64p, ctypes.c_int]),
        "nw_pack": (ctypes.c_int, [ctypes.c_char_p, u64, vp]),
        "nw_pack_device": (ctypes.c_int, [vp, vp, u64, vp]),
        "nw_pack_codes": (ctypes.c_int, [vp, u64, vp]),
        "nw_pack_pool": (ctypes.c_int, [vp, u64p, u32p, u32, vp, u64p]),
        "nw_cigar_bound": (u64, [u64, u64]),
        "nw_align": (ctypes.c_int, [vp, vp, u64, vp, u64, Scoring, u32, vp, vp, u64, vp]),
        "nw_align_batch": (ctypes.c_int, [vp, vp, u64p, u32p, u64p, u32p, u32, Scoring, u32, vp, vp, u64p, vp]),
        "nw_score_all_pairs": (ctypes.c_int, [vp, vp, u64p, u32p, u32, Scoring, u32, vp]),
        "nw_peak_int": (ctypes.c_int, [vp, ctypes.c_int, u64, ctypes.POINTER(ctypes.c_double)]),
        "nw_center_star": (ctypes.c_int, [vp, vp, u64p, u32p, u32, Scoring, u32, u32p, vp, vp, vp, u64p, vp, vp, u64,
                                          u64p]),
        "nw_msa_merge": (ctypes.c_int, [vp, vp, u64p, u32p, u32, u32, u32, vp, u64p, vp, vp, u64, u64p]),
        "nw_align_score_noalloc": (ctypes.c_int, [vp, u64, vp, u64, Scoring, vp, vp]),
        "nw_align_batch_banded": (ctypes.c_int, [vp, vp, u64p, u32p, u64p, u32p, u32, u32p, Scoring, u32, vp, vp,
                                                 u64p, vp]),
        "nw_ctx_band_stats": (ctypes.c_int, [vp, u64p, ctypes.c_int]),
        "nw_ctx_band_outcome": (ctypes.c_int64, [vp, vp, vp, vp, u64]),
        "nw_band_features": (ctypes.c_int, [vp, vp, u64p, u32p, u64p, u32p, u32, vp]),
        "nw_band_model_size": (u64, []),
        "nw_band_model_init": (ctypes.c_int, [vp, u64]),
        "nw_band_model_set": (ctypes.c_int, [vp, vp, u64]),
        "nw_band_model_get": (ctypes.c_int, [vp, vp, u64]),
        "nw_band_model_clear": (ctypes.c_int, [vp]),
        "nw_band_exit_bound": (ctypes.c_int, [u64, u64, u64, Scoring, ctypes.POINTER(ctypes.c_int64)]),
        "nw_band_certifies": (ctypes.c_int, [u64, u64, u64, ctypes.c_int32, Scoring, u32]),
        "nw_band_start_width": (u32, [ctypes.c_float, u64, u64]),
        "nw_route_stragglers": (ctypes.c_int64, [vp, vp, u32, vp]),
        "nw_shard_pairs": (ctypes.c_int, [u32p, u32p, u32, u32, u32p, u64p]),
        "nw_affine_align_batch": (ctypes.c_int, [vp, vp, u64p, u32p, u64p, u32p, u32, AffineScoring, u32, vp, vp,
                                                 u64p, vp]),
        "nw_local_align_batch": (ctypes.c_int, [vp, vp, u64p, u32p, u64p, u32p, u32, Scoring, u32, vp, vp, vp, u64p,
                                                vp]),
        "nw_band_next_width": (ctypes.c_int64, [u64, u64, u64, ctypes.c_int32, Scoring, u32]),
        "nw_band_model_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "nw_band_model_load": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "nw_band_model_forward": (ctypes.c_int, [vp, vp, u32, vp]),
        "nw_band_model_grad": (ctypes.c_int, [vp, vp, vp, u32, vp, vp]),
        "nw_band_model_train_step": (ctypes.c_int, [vp, vp, vp, u32, ctypes.c_float, vp]),
        "nw_server_create": (vp, [vp, u32, u32, u64, Scoring, u32]),
        "nw_server_create_ex": (vp, [vp, u32, u32, u64, u64, u32, Scoring, u32]),
        "nw_server_queue_state": (ctypes.c_int, [vp, u64p, u64p]),
        "nw_server_submit": (ctypes.c_int, [vp, vp, u32, vp, u32, u32, u64p]),
        "nw_server_submit_many": (ctypes.c_int, [vp, vp, u64p, u32p, u64p, u32p, vp, u32, u64p]),
        "nw_server_poll": (ctypes.c_int, [vp, ctypes.POINTER(Completion), u32, u32p, vp, u64, u64p]),
        "nw_server_drain": (ctypes.c_int, [vp, ctypes.c_double]),
        "nw_server_last_message": (ctypes.c_int64, [vp, ctypes.c_char_p, ctypes.c_uint64]),
        "nw_server_stats": (ctypes.c_int, [vp, u64p, ctypes.c_int]),
        "nw_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols() -> list[str]:
    """Names declared in include/nw.h (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "nw.h")
    text = open(hdr).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nw_[a-z0-9_]+)\s*\(", text)))


# ---------------------------------------------------------------- helpers
def _ptr(x) -> int | None:
    """Raw address of a torch tensor or numpy array (None for None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _is_host(x) -> bool:
    return isinstance(x, np.ndarray)


def _sc(scoring) -> Scoring:
    if isinstance(scoring, Scoring):
        return scoring
    return Scoring(*scoring)


def _check(ctx, rc: int):
    if rc != NW_OK:
        L = load()
        msg = L.nw_ctx_last_message(ctx.handle if isinstance(ctx, Context) else ctx)
        raise NWError(rc, (msg or b"").decode() or L.nw_strerror(rc).decode())


def pack_codes(codes: np.ndarray) -> np.ndarray:
    """Pack an array of base codes 0..3 into the 2-bit layout (host numpy)
    with the library's nw_pack_codes."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.zeros(max((codes.size + 3) // 4, 1), np.uint8)
    rc = load().nw_pack_codes(_ptr(codes), codes.size, _ptr(out))
    if rc != NW_OK:
        raise NWError(rc, load().nw_strerror(rc).decode())
    return out[: (codes.size + 3) // 4]


class Context:
    """Owns an ``nw_ctx``: device, stream, scratch pool and error word."""

    def __init__(self, device: int = 0, stream=None, mem_budget: int = 0):
        L = load()
        s = None
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.handle = L.nw_ctx_create(device, s, mem_budget)
        if not self.handle:
            raise NWError(NW_ERR_CUDA, f"nw_ctx_create failed on device {device}")
        self.device = device

    def close(self):
        self._cigar_host = None
        if getattr(self, "handle", None):
            load().nw_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        _check(self, load().nw_ctx_set_stream(self.handle, s))

    def sync(self):
        _check(self, load().nw_ctx_sync(self.handle))

    def set_profiling(self, on: bool):
        _check(self, load().nw_ctx_set_profiling(self.handle, int(bool(on))))

    def reset_stats(self):
        _check(self, load().nw_ctx_reset_stats(self.handle))

    def set_autotune(self, on: bool):
        _check(self, load().nw_ctx_set_autotune(self.handle, int(bool(on))))

    def tuning(self) -> dict[str, int]:
        """The autotuner's table {key: choice}."""
        L = load()
        n = L.nw_ctx_tuning(self.handle, None, 0)
        buf = ctypes.create_string_buffer(int(n) + 1)
        L.nw_ctx_tuning(self.handle, buf, n + 1)
        out = {}
        for line in buf.value.decode().splitlines():
            k, v = line.rsplit(" ", 1)
            out[k] = int(v)
        return out

    def set_tuning(self, table: dict[str, int]):
        text = "".join(f"{k} {int(v)}\n" for k, v in table.items())
        _check(self, load().nw_ctx_set_tuning(self.handle, text.encode()))

    def graph_stats(self) -> dict[str, int]:
        out = (ctypes.c_uint64 * 3)()
        load().nw_ctx_graph_stats(self.handle, out, 3)
        return {"graphs": int(out[0]), "captures": int(out[1]), "replays": int(out[2])}

    def kernel_stats(self) -> dict[str, tuple[int, float]]:
        L = load()
        n = L.nw_ctx_kernel_stats(self.handle, None, None, None, 0)
        names = (ctypes.c_char_p * max(n, 1))()
        launches = (ctypes.c_uint64 * max(n, 1))()
        ms = (ctypes.c_double * max(n, 1))()
        n = L.nw_ctx_kernel_stats(self.handle, names, launches, ms, n)
        return {names[k].decode(): (int(launches[k]), float(ms[k])) for k in range(n)}


# ------------------------------------------------------------- entry points
def nw_pack(ascii_seq) -> np.ndarray:
    """Host packing of an ASCII sequence (str/bytes) -> uint8 numpy array."""
    data = ascii_seq.encode() if isinstance(ascii_seq, str) else bytes(ascii_seq)
    out = np.zeros(max((len(data) + 3) // 4, 1), np.uint8)
    rc = load().nw_pack(data, len(data), out.ctypes.data)
    if rc != NW_OK:
        raise NWError(rc, load().nw_strerror(rc).decode())
    return out[: (len(data) + 3) // 4]


def nw_pack_device(ctx: Context, ascii_dev, length: int, out_dev):
    """Device packing: ascii_dev / out_dev are CUDA uint8 tensors."""
    _check(ctx, load().nw_pack_device(ctx.handle, _ptr(ascii_dev), length, _ptr(out_dev)))


def nw_cigar_bound(m: int, n: int) -> int:
    return int(load().nw_cigar_bound(m, n))


def nw_align(ctx: Context, a2b, m: int, b2b, n: int, scoring=DEFAULT_SCORING, flags: int = 0,
             score=None, cigar=None, cigar_len=None):
    """Align one pair.

    Host mode (a2b, b2b numpy arrays): returns (score, cigar or None).
    Device mode (CUDA tensors): writes into the given device outputs
    (int32[1], uint8[nw_cigar_bound], int64[1]) and returns them; the call
    is asynchronous on the context's stream."""
    L = load()
    want = bool(flags & NW_CIGAR)
    if _is_host(a2b):
        flags |= NW_HOST_IO
        sc_out = np.zeros(1, np.int32)
        cap = nw_cigar_bound(m, n) if want else 0
        cbuf = np.zeros(max(cap, 1), np.uint8)
        clen = np.zeros(1, np.uint64)
        rc = L.nw_align(ctx.handle, _ptr(a2b), m, _ptr(b2b), n, _sc(scoring), flags, _ptr(sc_out),
                        _ptr(cbuf) if want else None, cap, _ptr(clen) if want else None)
        _check(ctx, rc)
        return int(sc_out[0]), (cbuf[: int(clen[0])].tobytes().decode() if want else None)
    cap = int(cigar.numel()) if (want and cigar is not None) else 0
    rc = L.nw_align(ctx.handle, _ptr(a2b), m, _ptr(b2b), n, _sc(scoring), flags, _ptr(score),
                    _ptr(cigar) if want else None, cap, _ptr(cigar_len) if want else None)
    _check(ctx, rc)
    return score, cigar, cigar_len


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _cigar_offsets(a_len, b_len) -> np.ndarray:
    """Offsets of a CIGAR pool with nw_cigar_bound(m, n) = 2*(m+n)+1 bytes
    per pair (npairs+1 entries)."""
    caps = 2 * (np.asarray(a_len, np.uint64) + np.asarray(b_len, np.uint64)) + np.uint64(1)
    out = np.zeros(caps.size + 1, np.uint64)
    np.cumsum(caps, out=out[1:])
    return out


def _host_cigar_pool(ctx: "Context", nbytes: int) -> np.ndarray:
    """A host CIGAR pool of at least nbytes.  The library writes each pair's
    bytes at its offset.  The buffer is lent to the Cigars view of the call
    that fills it and returns to the context when that view is released, so
    a later call reuses it (no fresh buffer the size of the worst-case bound
    to fault in on every call)."""
    buf = getattr(ctx, "_cigar_host", None)
    ctx._cigar_host = None
    if buf is None or buf.size < nbytes:
        buf = np.empty(max(nbytes, 1), np.uint8)
    return buf


class Cigars:
    """The CIGARs of one host-mode batch call, one per pair, in pair order.

    The bytes stay in the host buffer the library wrote (each pair's CIGAR at
    its offset); an item is decoded to a str when it is read.  Behaves as a
    read-only sequence of str: len, indexing (slices give lists), iteration,
    and == against any sequence of str."""

    __hash__ = None

    def __init__(self, ctx: "Context", buf: np.ndarray, off, length, n: int):
        self._buf = buf
        self._off = np.asarray(off[:n], np.int64).copy()
        self._len = np.asarray(length[:n], np.int64).copy()
        self._ctx = ctx

    def __len__(self) -> int:
        return int(self._len.size)

    def _item(self, k: int) -> str:
        o = int(self._off[k])
        return self._buf[o:o + int(self._len[k])].tobytes().decode("ascii")

    def __getitem__(self, k):
        if isinstance(k, slice):
            return [self._item(i) for i in range(*k.indices(len(self)))]
        k = int(k)
        if k < 0:
            k += len(self)
        if not 0 <= k < len(self):
            raise IndexError(k)
        return self._item(k)

    def __iter__(self):
        mv = memoryview(self._buf)
        for o, n in zip(self._off.tolist(), self._len.tolist()):
            yield str(mv[o:o + n], "ascii")

    def __eq__(self, other):
        try:
            if len(other) != len(self):
                return False
            return all(a == b for a, b in zip(self, other))
        except TypeError:
            return NotImplemented

    def nbytes(self) -> int:
        """Total CIGAR bytes (without terminators)."""
        return int(self._len.sum())

    def tolist(self) -> list[str]:
        return list(self)

    def __repr__(self) -> str:
        return f"Cigars({len(self)} pairs, {self.nbytes()} bytes)"

    def __del__(self):
        ctx, buf = self._ctx, self._buf
        self._buf = None
        if ctx is not None and buf is not None and getattr(ctx, "handle", None):
            cur = getattr(ctx, "_cigar_host", None)
            if cur is None or cur.size < buf.size:
                ctx._cigar_host = buf


def _cigars(ctx: "Context", cpool: np.ndarray, off, length, npairs: int) -> Cigars:
    return Cigars(ctx, cpool, off, length, npairs)


def nw_align_batch(ctx: Context, pool2b, a_off, a_len, b_off, b_len, scoring=DEFAULT_SCORING, flags: int = 0,
                   scores=None, cigar_pool=None, cigar_off=None, cigar_len=None):
    """Align many pairs from one packed pool.  Metadata arrays are host
    numpy.  Host mode (pool2b numpy) returns (scores ndarray, Cigars sequence
    or None); device mode writes into the given tensors."""
    L = load()
    npairs = len(a_len)
    ao, aop = _u64(a_off)
    al, alp = _u32(a_len)
    bo, bop = _u64(b_off)
    bl, blp = _u32(b_len)
    want = bool(flags & NW_CIGAR)
    if cigar_off is None and want:
        cigar_off = _cigar_offsets(al, bl)
    co, cop = _u64(cigar_off) if want else (None, None)
    if _is_host(pool2b):
        flags |= NW_HOST_IO
        sc_out = np.zeros(max(npairs, 1), np.int32)
        cpool = _host_cigar_pool(ctx, int(co[-1])) if want else np.empty(1, np.uint8)
        clen = np.zeros(max(npairs, 1), np.uint64)
        rc = L.nw_align_batch(ctx.handle, _ptr(pool2b), aop, alp, bop, blp, npairs, _sc(scoring), flags,
                              _ptr(sc_out), _ptr(cpool) if want else None, cop, _ptr(clen) if want else None)
        _check(ctx, rc)
        cigars = None
        if want:
            cigars = _cigars(ctx, cpool, co, clen, npairs)
        return sc_out[:npairs], cigars
    rc = L.nw_align_batch(ctx.handle, _ptr(pool2b), aop, alp, bop, blp, npairs, _sc(scoring), flags, _ptr(scores),
                          _ptr(cigar_pool) if want else None, cop, _ptr(cigar_len) if want else None)
    _check(ctx, rc)
    return scores, cigar_pool, cigar_len


def nw_local_align_batch(ctx: Context, pool2b, a_off, a_len, b_off, b_len, scoring=DEFAULT_SCORING, flags: int = 0,
                         scores=None, ends=None, cigar_pool=None, cigar_off=None, cigar_len=None):
    """Local alignment (Smith-Waterman) of many pairs.  Host mode (pool2b
    numpy) returns (scores, ends (npairs, 4): i_start, j_start, i_end, j_end,
    CIGARs or None); device mode writes into the given tensors."""
    L = load()
    npairs = len(a_len)
    ao, aop = _u64(a_off)
    al, alp = _u32(a_len)
    bo, bop = _u64(b_off)
    bl, blp = _u32(b_len)
    want = bool(flags & NW_CIGAR)
    if cigar_off is None and want:
        cigar_off = _cigar_offsets(al, bl)
    co, cop = _u64(cigar_off) if want else (None, None)
    if _is_host(pool2b):
        flags |= NW_HOST_IO
        sc_out = np.zeros(max(npairs, 1), np.int32)
        e_out = np.zeros((max(npairs, 1), 4), np.uint32)
        cpool = _host_cigar_pool(ctx, int(co[-1])) if want else np.empty(1, np.uint8)
        clen = np.zeros(max(npairs, 1), np.uint64)
        rc = L.nw_local_align_batch(ctx.handle, _ptr(pool2b), aop, alp, bop, blp, npairs, _sc(scoring), flags,
                                    _ptr(sc_out), _ptr(e_out), _ptr(cpool) if want else None, cop,
                                    _ptr(clen) if want else None)
        _check(ctx, rc)
        return sc_out[:npairs], e_out[:npairs], (_cigars(ctx, cpool, co, clen, npairs) if want else None)
    rc = L.nw_local_align_batch(ctx.handle, _ptr(pool2b), aop, alp, bop, blp, npairs, _sc(scoring), flags,
                                _ptr(scores), _ptr(ends), _ptr(cigar_pool) if want else None, cop,
                                _ptr(cigar_len) if want else None)
    _check(ctx, rc)
    return scores, ends, cigar_len


def nw_affine_align_batch(ctx: Context, pool2b, a_off, a_len, b_off, b_len, scoring=(1, -1, -2, -1), flags: int = 0,
                          scores=None, cigar_pool=None, cigar_off=None, cigar_len=None):
    """Global alignment with affine gaps; scoring = (match, mismatch,
    gap_open, gap_extend).  Host mode (pool2b numpy) returns (scores, CIGARs
    or None); device mode writes into the given tensors."""
    L = load()
    npairs = len(a_len)
    ao, aop = _u64(a_off)
    al, alp = _u32(a_len)
    bo, bop = _u64(b_off)
    bl, blp = _u32(b_len)
    sc = scoring if isinstance(scoring, AffineScoring) else AffineScoring(*scoring)
    want = bool(flags & NW_CIGAR)
    if cigar_off is None and want:
        cigar_off = _cigar_offsets(al, bl)
    co, cop = _u64(cigar_off) if want else (None, None)
    if _is_host(pool2b):
        flags |= NW_HOST_IO
        sc_out = np.zeros(max(npairs, 1), np.int32)
        cpool = _host_cigar_pool(ctx, int(co[-1])) if want else np.empty(1, np.uint8)
        clen = np.zeros(max(npairs, 1), np.uint64)
        rc = L.nw_affine_align_batch(ctx.handle, _ptr(pool2b), aop, alp, bop, blp, npairs, sc, flags, _ptr(sc_out),
                                     _ptr(cpool) if want else None, cop, _ptr(clen) if want else None)
        _check(ctx, rc)
        return sc_out[:npairs], (_cigars(ctx, cpool, co, clen, npairs) if want else None)
    rc = L.nw_affine_align_batch(ctx.handle, _ptr(pool2b), aop, alp, bop, blp, npairs, sc, flags, _ptr(scores),
                                 _ptr(cigar_pool) if want else None, cop, _ptr(cigar_len) if want else None)
    _check(ctx, rc)
    return scores, cigar_pool, cigar_len


def nw_align_batch_banded(ctx: Context, pool2b, a_off, a_len, b_off, b_len, band_w, scoring=DEFAULT_SCORING,
                          flags: int = 0, scores=None, cigar_pool=None, cigar_off=None, cigar_len=None):
    """Certified banded batch with explicit starting half-widths (host
    array band_w).  Same marshalling as nw_align_batch."""
    L = load()
    npairs = len(a_len)
    ao, aop = _u64(a_off)
    al, alp = _u32(a_len)
    bo, bop = _u64(b_off)
    bl, blp = _u32(b_len)
    ww, wwp = _u32(band_w)
    want = bool(flags & NW_CIGAR)
    if cigar_off is None and want:
        cigar_off = _cigar_offsets(al, bl)
    co, cop = _u64(cigar_off) if want else (None, None)
    if _is_host(pool2b):
        flags |= NW_HOST_IO
        sc_out = np.zeros(max(npairs, 1), np.int32)
        cpool = _host_cigar_pool(ctx, int(co[-1])) if want else np.empty(1, np.uint8)
        clen = np.zeros(max(npairs, 1), np.uint64)
        rc = L.nw_align_batch_banded(ctx.handle, _ptr(pool2b), aop, alp, bop, blp, npairs, wwp, _sc(scoring), flags,
                                     _ptr(sc_out), _ptr(cpool) if want else None, cop, _ptr(clen) if want else None)
        _check(ctx, rc)
        cigars = None
        if want:
            cigars = _cigars(ctx, cpool, co, clen, npairs)
        return sc_out[:npairs], cigars
    rc = L.nw_align_batch_banded(ctx.handle, _ptr(pool2b), aop, alp, bop, blp, npairs, wwp, _sc(scoring), flags,
                                 _ptr(scores), _ptr(cigar_pool) if want else None, cop,
                                 _ptr(cigar_len) if want else None)
    _check(ctx, rc)
    return scores, cigar_pool, cigar_len


def nw_ctx_band_stats(ctx: Context) -> dict:
    out = (ctypes.c_uint64 * 8)()
    load().nw_ctx_band_stats(ctx.handle, out, 8)
    v = [int(x) for x in out]
    return {"tried": v[0], "certified_round": v[1:4], "full_fallback": v[5], "band_cells": v[6],
            "full_cells": v[7]}


def nw_ctx_band_outcome(ctx: Context) -> dict:
    """Per pair of the last certified-band call: the round that certified it
    (1..3, 0 = the full kernel), its first and its certified half-width."""
    L = load()
    n = int(L.nw_ctx_band_outcome(ctx.handle, None, None, None, 0))
    if n < 0:
        raise NWError(-n, "nw_ctx_band_outcome: bad argument")
    rnd = np.zeros(max(n, 1), np.uint8)
    w0 = np.zeros(max(n, 1), np.uint32)
    wc = np.zeros(max(n, 1), np.uint32)
    L.nw_ctx_band_outcome(ctx.handle, _ptr(rnd), _ptr(w0), _ptr(wc), n)
    return {"round": rnd[:n], "first_width": w0[:n], "cert_width": wc[:n]}


def nw_band_features(ctx: Context, pool_dev, a_off, a_len, b_off, b_len, out=None):
    """Features of the pairs (device pool) -> CUDA float32 tensor (n, 65)."""
    import torch
    n = len(a_len)
    if out is None:
        out = torch.zeros((n, 65), dtype=torch.float32, device=pool_dev.device)
    ao, aop = _u64(a_off)
    al, alp = _u32(a_len)
    bo, bop = _u64(b_off)
    bl, blp = _u32(b_len)
    _check(ctx, load().nw_band_features(ctx.handle, _ptr(pool_dev), aop, alp, bop, blp, n, _ptr(out)))
    return out


def nw_band_model_size() -> int:
    return int(load().nw_band_model_size())


def nw_band_model_init(ctx: Context, seed: int = 0):
    _check(ctx, load().nw_band_model_init(ctx.handle, seed))


def nw_band_model_set(ctx: Context, params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, load().nw_band_model_set(ctx.handle, _ptr(p), p.size))


def nw_band_model_get(ctx: Context) -> np.ndarray:
    p = np.zeros(nw_band_model_size(), np.float32)
    _check(ctx, load().nw_band_model_get(ctx.handle, _ptr(p), p.size))
    return p


def nw_band_model_save(ctx: Context, path):
    _check(ctx, load().nw_band_model_save(ctx.handle, os.fsencode(path)))


def nw_band_model_load(ctx: Context, path):
    _check(ctx, load().nw_band_model_load(ctx.handle, os.fsencode(path)))


def nw_band_exit_bound(m: int, n: int, w: int, scoring=DEFAULT_SCORING):
    """The banded certificate's exit bound (None when no path can leave the
    band); host arithmetic of the library, no GPU needed."""
    b = ctypes.c_int64(0)
    rc = load().nw_band_exit_bound(m, n, w, _sc(scoring), ctypes.byref(b))
    if rc < 0:
        raise NWError(-rc, "nw_band_exit_bound: bad argument")
    return int(b.value) if rc == 1 else None


def nw_route_stragglers(warp_cells, full_cells) -> list[int]:
    """Indices of the pairs the batched paths run on the single-pair kernel
    (host arithmetic of the straggler rule)."""
    wc = np.ascontiguousarray(warp_cells, dtype=np.float64)
    fc = np.ascontiguousarray(full_cells, dtype=np.float64)
    out = np.zeros(max(wc.size, 1), np.uint32)
    k = int(load().nw_route_stragglers(_ptr(wc), _ptr(fc), wc.size, _ptr(out)))
    if k < 0:
        raise NWError(-k, "nw_route_stragglers: bad argument")
    return out[:k].tolist()


def nw_band_start_width(y: float, m: int, n: int) -> int:
    """First banded half-width from the network output y (host arithmetic)."""
    return int(load().nw_band_start_width(y, m, n))


def nw_band_certifies(m: int, n: int, w: int, banded_score: int, want_cigar: bool, scoring=DEFAULT_SCORING) -> bool:
    """Whether a banded score proves the full result (host arithmetic)."""
    rc = load().nw_band_certifies(m, n, w, banded_score, _sc(scoring), int(bool(want_cigar)))
    if rc < 0:
        raise NWError(-rc, "nw_band_certifies: bad argument")
    return rc == 1


def nw_band_next_width(m: int, n: int, w: int, banded_score: int, want_cigar: bool, scoring=DEFAULT_SCORING) -> int:
    """The next round's half-width after a failed certificate (host arithmetic)."""
    rc = int(load().nw_band_next_width(m, n, w, banded_score, _sc(scoring), int(bool(want_cigar))))
    if rc < 0:
        raise NWError(-rc, "nw_band_next_width: bad argument")
    return rc


def nw_band_model_clear(ctx: Context):
    _check(ctx, load().nw_band_model_clear(ctx.handle))


def nw_band_model_forward(ctx: Context, feat, out=None):
    import torch
    n = int(feat.shape[0])
    if out is None:
        out = torch.zeros(n, dtype=torch.float32, device=feat.device)
    _check(ctx, load().nw_band_model_forward(ctx.handle, _ptr(feat), n, _ptr(out)))
    return out


def nw_band_model_grad(ctx: Context, feat, target):
    import torch
    grad = torch.zeros(nw_band_model_size(), dtype=torch.float32, device=feat.device)
    loss = torch.zeros(1, dtype=torch.float32, device=feat.device)
    _check(ctx, load().nw_band_model_grad(ctx.handle, _ptr(feat), _ptr(target), int(feat.shape[0]), _ptr(grad),
                                          _ptr(loss)))
    return grad, loss


def nw_band_model_train_step(ctx: Context, feat, target, lr: float, loss=None):
    import torch
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=feat.device)
    _check(ctx, load().nw_band_model_train_step(ctx.handle, _ptr(feat), _ptr(target), int(feat.shape[0]), lr,
                                                _ptr(loss)))
    return loss


class Server:
    """Continuous-batching server (nw_server): submit host requests, poll
    completions.  See include/nw.h."""

    def __init__(self, ctx: Context, workers: int = 8, max_batch: int = 64, trace_budget: int = 16 << 30,
                 scoring=DEFAULT_SCORING, flags: int = 0, queue_bytes: int = 1 << 30, queue_slots: int = 1 << 20):
        self.handle = load().nw_server_create_ex(ctx.handle, workers, max_batch, trace_budget, queue_bytes,
                                                 queue_slots, _sc(scoring), flags)
        if not self.handle:
            raise NWError(NW_ERR_ARG, "nw_server_create failed")
        self._cbuf = np.zeros(1 << 24, np.uint8)

    def submit(self, a_codes_packed, m: int, b_codes_packed, n: int, want_cigar: bool) -> int:
        t = ctypes.c_uint64(0)
        rc = load().nw_server_submit(self.handle, _ptr(a_codes_packed), m, _ptr(b_codes_packed), n,
                                     int(bool(want_cigar)), ctypes.byref(t))
        if rc != NW_OK:
            raise NWError(rc, "submit failed")
        return int(t.value)

    def submit_many(self, pool2b, a_off, a_len, b_off, b_len, want_cigar) -> np.ndarray:
        ao, aop = _u64(a_off)
        al, alp = _u32(a_len)
        bo, bop = _u64(b_off)
        bl, blp = _u32(b_len)
        wc = np.ascontiguousarray(want_cigar, dtype=np.uint8)
        n = int(al.size)
        tickets = np.zeros(max(n, 1), np.uint64)
        rc = load().nw_server_submit_many(self.handle, _ptr(pool2b), aop, alp, bop, blp, _ptr(wc), n,
                                          tickets.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        if rc != NW_OK:
            raise NWError(rc, "submit failed")
        return tickets[:n]

    def poll(self, cap: int = 4096):
        """[(ticket, status, score, cigar or None, latency_s)]"""
        out = (Completion * cap)()
        cnt = ctypes.c_uint32(0)
        used = ctypes.c_uint64(0)
        rc = load().nw_server_poll(self.handle, out, cap, ctypes.byref(cnt), _ptr(self._cbuf), self._cbuf.size,
                                   ctypes.byref(used))
        if rc == NW_ERR_CIGAR_TRUNC:  # the oldest CIGAR needs a larger buffer
            self._cbuf = np.zeros(max(int(used.value), 2 * self._cbuf.size), np.uint8)
            return self.poll(cap)
        if rc != NW_OK:
            raise NWError(rc, "poll failed")
        res = []
        for k in range(cnt.value):
            c = out[k]
            cig = None
            if c.cigar_len:
                cig = self._cbuf[c.cigar_off: c.cigar_off + c.cigar_len].tobytes().decode()
            res.append((int(c.ticket), int(c.status), int(c.score), cig, float(c.latency_s)))
        return res

    def poll_all(self):
        """Every completion queued now: polls until the queue is empty (one poll stops when the
        CIGAR buffer fills)."""
        res = []
        while True:
            got = self.poll(1 << 16)
            if not got:
                return res
            res += got

    def queue_state(self) -> dict:
        """The device queue word: requests admitted, traceback bytes reserved."""
        adm, res = ctypes.c_uint64(0), ctypes.c_uint64(0)
        rc = load().nw_server_queue_state(self.handle, ctypes.byref(adm), ctypes.byref(res))
        if rc != NW_OK:
            raise NWError(rc, "queue state failed")
        return {"admitted": int(adm.value), "reserved": int(res.value)}

    def drain(self, timeout_s: float = 600.0) -> bool:
        return load().nw_server_drain(self.handle, timeout_s) == NW_OK

    def last_message(self) -> str:
        """Status and message of the last batch that failed ("" while none has)."""
        buf = ctypes.create_string_buffer(1024)
        n = load().nw_server_last_message(self.handle, buf, len(buf))
        return buf.value.decode(errors="replace") if n > 0 else ""

    def stats(self) -> dict:
        out = (ctypes.c_uint64 * 8)()
        load().nw_server_stats(self.handle, out, 8)
        keys = ["submitted", "completed", "waiting", "running", "cells", "reserved", "batches", "budget"]
        return {k: int(v) for k, v in zip(keys, out)}

    def close(self):
        if getattr(self, "handle", None):
            load().nw_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nw_score_all_pairs(ctx: Context, pool2b, off, lens, scoring=DEFAULT_SCORING, flags: int = 0, out=None):
    """All-vs-all score matrix.  Host mode returns an (n, n) int32 array."""
    L = load()
    nseq = len(lens)
    oo, oop = _u64(off)
    ll, llp = _u32(lens)
    if _is_host(pool2b):
        flags |= NW_HOST_IO
        res = np.zeros((nseq, nseq), np.int32)
        _check(ctx, L.nw_score_all_pairs(ctx.handle, _ptr(pool2b), oop, llp, nseq, _sc(scoring), flags, _ptr(res)))
        return res
    _check(ctx, L.nw_score_all_pairs(ctx.handle, _ptr(pool2b), oop, llp, nseq, _sc(scoring), flags, _ptr(out)))
    return out


def _center_cigar_offsets(lens) -> np.ndarray:
    """CIGAR offsets for nw_center_star: 2*(len[k] + max len) + 1 bytes per
    sequence (at least nw_cigar_bound against any center)."""
    L = np.asarray(lens, np.uint64)
    caps = np.uint64(2) * (L + (L.max() if L.size else np.uint64(0))) + np.uint64(1)
    out = np.zeros(L.size + 1, np.uint64)
    np.cumsum(caps, out=out[1:])
    return out


def nw_center_star(ctx: Context, pool2b, off, lens, scoring=DEFAULT_SCORING, flags: int = 0, row_sums=None,
                   scores=None, cigar_pool=None, cigar_off=None, cigar_len=None, msa=None, msa_ld: int = 0):
    """Center-star multiple alignment (Sec. 3.2).

    Host mode (pool2b numpy): returns a dict with the center, the row sums,
    each sequence's score and CIGAR against the center and the merged rows
    (strings over 'ACGT-'); the rows come from nw_msa_merge once the column
    count is known.  Device mode: writes into the given CUDA tensors
    (row_sums int64[nseq] or None, scores int32[nseq], cigar_pool uint8,
    cigar_len int64[nseq], msa uint8[nseq * msa_ld] or None) and returns
    (center, msa_cols)."""
    L = load()
    nseq = len(lens)
    oo, oop = _u64(off)
    ll, llp = _u32(lens)
    if cigar_off is None:
        cigar_off = _center_cigar_offsets(ll)
    co, cop = _u64(cigar_off)
    center = ctypes.c_uint32(0)
    cols = ctypes.c_uint64(0)
    if _is_host(pool2b):
        sums = np.zeros(max(nseq, 1), np.int64)
        sc_out = np.zeros(max(nseq, 1), np.int32)
        cpool = np.zeros(max(int(co[-1]), 1), np.uint8)
        clen = np.zeros(max(nseq, 1), np.uint64)
        rc = L.nw_center_star(ctx.handle, _ptr(pool2b), oop, llp, nseq, _sc(scoring), flags | NW_HOST_IO,
                              ctypes.byref(center), _ptr(sums), _ptr(sc_out), _ptr(cpool), cop, _ptr(clen), None, 0,
                              ctypes.byref(cols))
        _check(ctx, rc)
        ld = int(cols.value) + 1
        rows = np.zeros(max(nseq * ld, 1), np.uint8)
        c0, c0p = _u64(co[:nseq])
        rc = L.nw_msa_merge(ctx.handle, _ptr(pool2b), oop, llp, nseq, center.value, NW_HOST_IO, _ptr(cpool), c0p,
                            _ptr(clen), _ptr(rows), ld, ctypes.byref(cols))
        _check(ctx, rc)
        ncols = int(cols.value)
        text = rows[: nseq * ld].reshape(nseq, ld)[:, :ncols] if nseq else rows[:0]
        return {"center": int(center.value), "row_sums": sums[:nseq], "scores": sc_out[:nseq],
                "cigars": _cigars(ctx, cpool, co, clen, nseq), "rows": [bytes(r).decode() for r in text],
                "columns": ncols}
    rc = L.nw_center_star(ctx.handle, _ptr(pool2b), oop, llp, nseq, _sc(scoring), flags, ctypes.byref(center),
                          _ptr(row_sums), _ptr(scores), _ptr(cigar_pool), cop, _ptr(cigar_len), _ptr(msa), msa_ld,
                          ctypes.byref(cols))
    if rc == NW_ERR_CIGAR_TRUNC:
        return int(center.value), int(cols.value), False
    _check(ctx, rc)
    return int(center.value), int(cols.value), True


def nw_msa_merge(ctx: Context, pool2b, off, lens, center: int, cigar_pool, cigar_off, cigar_len, msa=None,
                 msa_ld: int = 0, flags: int = 0) -> int:
    """Merge given alignments against sequence `center` (the last stage of
    nw_center_star); returns the column count.  Device tensors, or numpy
    arrays with NW_HOST_IO."""
    L = load()
    oo, oop = _u64(off)
    ll, llp = _u32(lens)
    co, cop = _u64(np.asarray(cigar_off)[: len(lens)])
    cols = ctypes.c_uint64(0)
    if _is_host(pool2b):
        flags |= NW_HOST_IO
    rc = L.nw_msa_merge(ctx.handle, _ptr(pool2b), oop, llp, len(lens), center, flags, _ptr(cigar_pool), cop,
                        _ptr(cigar_len), _ptr(msa), msa_ld, ctypes.byref(cols))
    _check(ctx, rc)
    return int(cols.value)


def nw_align_score_noalloc(a2b, m: int, b2b, n: int, scoring=DEFAULT_SCORING, score=None, stream=None) -> int:
    """Score of one pair with no allocation inside the library (device
    tensors in, device int32[1] out; waits for completion).  Returns the
    status code (NW_OK, NW_ERR_ARG beyond the static scratch, ...)."""
    import torch
    dev = torch.cuda.current_device()
    for name, t in (("a2b", a2b), ("b2b", b2b), ("score", score)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == dev):
            raise ValueError(f"nw_align_score_noalloc: {name} must be a CUDA tensor on the current device (cuda:{dev})")
    if score.dtype != torch.int32 or score.numel() < 1:
        raise ValueError("nw_align_score_noalloc: score must be an int32 tensor with at least one element")
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return int(load().nw_align_score_noalloc(_ptr(a2b), m, _ptr(b2b), n, _sc(scoring), _ptr(score), s))


def nw_peak_int(ctx: Context, kind: int, iters: int = 1 << 16) -> float:
    """Measured integer-pipe rate (1e9 lane-ops/s) for one instruction kind."""
    v = ctypes.c_double(0.0)
    _check(ctx, load().nw_peak_int(ctx.handle, kind, iters, ctypes.byref(v)))
    return float(v.value)


def pool_of(seqs) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Pack sequences (code arrays) into one pool with the library's
    nw_pack_pool; returns (pool, byte offsets, lengths).  Each sequence
    starts on a 16-byte boundary (at least 16 bytes each)."""
    seqs = [np.ascontiguousarray(s, dtype=np.uint8) for s in seqs]
    lens = np.array([s.size for s in seqs], np.uint32)
    if not seqs:
        return np.zeros(16, np.uint8), np.zeros(0, np.uint64), lens
    slot = np.maximum((lens.astype(np.uint64) + 3) // 4 + 15, 16) // 16 * 16   # bytes per sequence, 16-aligned
    offs = np.zeros(len(seqs), np.uint64)
    np.cumsum(slot[:-1], out=offs[1:])
    codes = np.concatenate(seqs) if lens.sum() else np.zeros(1, np.uint8)
    code_off = np.zeros(len(seqs), np.uint64)
    np.cumsum(lens[:-1].astype(np.uint64), out=code_off[1:])
    pool = np.zeros(int(offs[-1] + slot[-1]), np.uint8)
    co, cop = _u64(code_off)
    ll, llp = _u32(lens)
    po, pop = _u64(offs)
    rc = load().nw_pack_pool(_ptr(codes), cop, llp, len(seqs), _ptr(pool), pop)
    if rc != NW_OK:
        raise NWError(rc, load().nw_strerror(rc).decode())
    return pool, offs, lens
