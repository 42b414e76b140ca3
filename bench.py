"""Benchmark of the Needleman-Wunsch hot path on one GB300 (or N replicas).

Default workload (`band`): 20,000 pairs of lengths log-uniform in [2,000,
20,000] at 1-25% divergence with indel bursts, aligned with score + CIGAR by
the certified learned band (a BF16 network trained on the GPU picks each
pair's band; the closed-form certificate accepts a banded result only when
it provably equals full NW; the rest widen or fall back to the full batched
kernel).  One step = features, network, banded rounds, fallback, traceback,
CIGARs.  Metric: effective GCUPS = full-matrix cells / step time; the line
also carries the plain full-matrix batch on the same pairs and the number of
score and CIGAR mismatches between the two.

Other workloads: pair32k (one 32,768 x 32,768 pair), pair1k (one 1,000 x
1,000 pair), allpairs (512 sequences, all 130,816 pairwise scores),
centerstar (the center-star multiple alignment of the same 512 sequences),
local (local alignment of 4,000 query/reference pairs), affine (affine-gap
global alignment of 2,000 pairs), serve (Poisson request stream into the continuous-batching server).

    python bench.py [--gpus N] [--steps K] [--warmup W]
                    [--workload band|pair32k|pair1k|allpairs|centerstar|local|affine|serve]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

Prints one JSON line.  The path does not shard: with --gpus N under
torchrun every rank runs an independent replica and `value` counts the
cells of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import seqgen  # noqa: E402

METRIC = "GCUPS on 1 GB300 and % of int/DPX roofline; learned-band+batched vs plain NW, exact"
SCORING = (1, -1, -1)
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2
HERE = os.path.dirname(os.path.abspath(__file__))
OPS_PER_CELL = 4             # algorithmic work of the textbook cell: s select, D+s, max(E_up, E_left), add-max
W_OPS_PER_CELL = 3           # what the W-domain kernels issue for it: prmt + add-max + max
PEAK_KINDS = (0, 2, 4)       # nw_peak_int kinds: DPX add-max, max, prmt (lane-ops/s each)
CELL_KINDS = (5, 6, 7)       # nw_peak_int kinds: score-only cells in three instruction mixes (cells/s)
# The bit-sliced kernels (bits_score, bband_*) update 32 cells of an anti-diagonal
# with whole-word operations.  Their algorithmic work per 32 cells: 14 logic
# ops of the difference update (match word 2, T = max(s', a, b) 6, dV 3, dH 3)
# and 2 funnel shifts that bring the upper neighbour's difference into line;
# the pointer planes add 2 (L, Hb).
BITS_OPS_PER_32 = 16
BITS_PTR_OPS_PER_32 = 18
BITS_PEAK_KINDS = (8, 10)    # nw_peak_int kinds: 3-input logic op, funnel shift (lane-ops/s)
BITS_CELL_KIND = 11          # nw_peak_int kind: one bit-sliced step, 32 cells (cells/s)
BITS_KERNELS = ("bits_score", "bband_fill_ptr", "bband_score", "bpair_fill_ptr")
# The single-pair kernel (bpair_fill_ptr) keeps 31 rows per word (bit 31 is a
# spare row) and runs one anti-diagonal step of a stripe after another: its
# time is the wavefront's chain of m + n + m/31 steps, each 24 logic ops of
# one warp (the 16-lane logic pipe of one scheduler: 2 cycles each).
PAIR_ROWS = 31
PAIR_ALU_OPS_PER_STEP = 24
HBM_PEAK_FALLBACK = 6800.0   # GB/s, when MEASURED_PEAKS.json is absent
STEPS_DEFAULT = {"pair32k": 100, "pair1k": 200, "allpairs": 20, "centerstar": 20, "local": 10, "affine": 10, "band": 3}


def code_only(text: str) -> str:
    """C/C++/CUDA source without its comments and trailing blanks (string
    and character literals kept): what the compiler sees of the code."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(ln.rstrip() for ln in "".join(out).splitlines() if ln.strip())


def source_region(text: str, spec: str) -> str:
    """The part of a source that a record covers: the whole text, or for a
    spec `from..to` the lines from the first one holding `from` up to (not
    including) the next one holding `to` (empty when either is missing)."""
    if not spec:
        return text
    start, _, end = spec.partition("..")
    lines = text.splitlines()
    try:
        i = next(k for k, ln in enumerate(lines) if start in ln)
        j = next(k for k in range(i + 1, len(lines)) if end in lines[k])
    except StopIteration:
        return ""
    return "\n".join(lines[i:j])


def sources_sha(files, read=None) -> str:
    """First 16 hex digits of the sha256 over the code (comments removed) of
    the given sources, in name order.  A source is a file path, or
    `path#from..to` for one region of it (source_region); `read(path)` gives
    a file's text (default: the file in this tree)."""
    import hashlib
    read = read or (lambda f: open(os.path.join(HERE, f), encoding="utf-8").read())
    h = hashlib.sha256()
    for src in sorted(files):
        f, _, spec = src.partition("#")
        h.update(os.path.basename(src).encode())
        h.update(code_only(source_region(read(f), spec)).encode())
    return h.hexdigest()[:16]


def dram_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    record, or None when there is none or the kernel's code changed since
    (comments do not count)."""
    path = os.path.join(HERE, "profiles", "dram_traffic.json")
    try:
        rec = json.load(open(path))["entries"][f"{kernel}@{workload}"]
        if sources_sha(rec["sources"]) != rec["sha"]:
            return None
        return rec["dram_read"] + rec["dram_write"]
    except (OSError, KeyError, ValueError):
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default per workload: pair32k 100, pair1k 200, allpairs 20, band 3)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="band",
                    choices=["band", "pair32k", "pair1k", "allpairs", "centerstar", "local", "affine", "serve"])
    ap.add_argument("--rate", type=float, default=50000.0, help="serve: Poisson arrival rate (requests/s)")
    ap.add_argument("--duration", type=float, default=3.0, help="serve: seconds of arrivals")
    ap.add_argument("--serve-pool", type=int, default=1500, help="serve: distinct requests the stream cycles through")
    ap.add_argument("--serve-workers", type=int, default=8, help="serve: worker threads (contexts, streams)")
    ap.add_argument("--serve-batch", type=int, default=1024, help="serve: most requests one admission takes")
    ap.add_argument("--npairs", type=int, default=None,
                    help="pairs of the band / local / affine workloads (full: 20,000 / 4,000 / 2,000)")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="leave out the CPU oracle leg (outside the timed region; for profiling runs)")
    ap.add_argument("--nseq", type=int, default=512, help="allpairs: number of sequences (512 = the full workload)")
    ap.add_argument("--m", type=int, default=32768, help="pair32k: query length (32,768 = the full workload)")
    return ap.parse_args()


def slowest_rank_ms(ms: float, device=None) -> float:
    """The largest of each rank's time over the default process group (the
    rank's own time when there is none): a multi-rank job is as fast as its
    slowest rank.  `device` is where the reduction tensor lives (a CUDA
    device for NCCL, None = CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gcups(cells_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the cells every rank aligned over the slowest
    rank's time."""
    return world * cells_per_rank / (ms * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


WL_ARGS = {"nseq": 512, "m": 32768, "npairs": None}
NPAIRS_FULL = {"band": 20000, "local": 4000, "affine": 2000}
LABELS = os.path.join(ROOT, "tests", "golden", "band_labels_seed9004.npz")


def workload(name: str):
    npairs = WL_ARGS["npairs"] or NPAIRS_FULL.get(name, 0)
    if name == "band":
        pairs = seqgen.band_pairs(1004, npairs=npairs)
        return pairs, (f"learned certified band, {npairs:,} pairs: lengths log-uniform [2,000, 20,000], divergence "
                       "U[0.01,0.25], geometric indels, indel bursts 50-500 bp w.p. 0.3 (seed 1004); score + CIGAR; "
                       "model trained on the GPU from oracle labels of 4,000 pairs of seed 9004")
    if name == "allpairs":
        nseq = WL_ARGS["nseq"]
        seqs = seqgen.all_vs_all_family(1003, nseq=nseq)
        return seqs, (f"all-vs-all scores of {nseq} mutants of one random 1,500-base root (lengths U{{500..1500}}, "
                      f"divergence U[0.05,0.30], 20% of mutations 1-bp indels), {nseq * (nseq - 1) // 2:,} pairs, int32 matrix "
                      "(seed 1003)")
    if name == "centerstar":
        nseq = WL_ARGS["nseq"]
        seqs = seqgen.all_vs_all_family(1003, nseq=nseq)
        return seqs, (f"center-star multiple alignment of {nseq} mutants of one random 1,500-base root (lengths "
                      f"U{{500..1500}}, divergence U[0.05,0.30], 20% of mutations 1-bp indels; seed 1003): "
                      f"{nseq * (nseq - 1) // 2:,} scored pairs, center, {nseq} alignments with CIGAR, merged rows")
    if name == "local":
        pairs = seqgen.local_pairs(1006, npairs=npairs)
        return pairs, (f"local alignment (Smith-Waterman), {npairs:,} pairs: a reference of U[2,000, 10,000] random bases "
                       "against a query made of a mutated window of it (U[200, 2,000] bases, divergence U[0.01,0.20], "
                       "geometric indels) between random flanks of up to 500 bases (seed 1006); score, start, end "
                       "and CIGAR")
    if name == "affine":
        pairs = seqgen.band_pairs(1007, npairs=npairs, lmin=1000, lmax=5000)
        return pairs, (f"affine-gap global alignment (Gotoh), {npairs:,} pairs: lengths log-uniform [1,000, 5,000], "
                       "divergence U[0.01,0.25], geometric indels, indel bursts 50-500 bp w.p. 0.3 (seed 1007); "
                       "match 2, mismatch -3, gap open -5, gap extend -2; score + CIGAR")
    if name == "pair1k":
        p = seqgen.random_pair(1001, 1000, 1000)
        return p, "single pair 1,000 x 1,000 i.i.d. uniform ACGT, score + CIGAR (seed 1001)"
    p = seqgen.long_mutated_pair(1002, m=WL_ARGS["m"])
    return p, (f"single long pair {p.a.size:,} x {p.b.size:,}: B = A with 10% substitutions and 2% geometric "
               f"indels (mean 3), score + CIGAR (seed 1002)")


class ClockSampler:
    """nvidia-smi clock samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.perf_counter(), ln.strip()))

    def window(self, t0: float, t1: float):
        """The timed region; only samples taken inside it count."""
        self.t0, self.t1 = t0, t1

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if self.t0 is not None and not (self.t0 <= ts <= self.t1 + 0.15):
                continue  # (a sample reaches us up to one period after it was taken)
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- reference arm
def oracle_gcups(pair, budget_s: float = 12.0, threads: int | None = None):
    """The CPU oracle, as it stands, on diagonal sub-blocks of the pair
    (score + alignment), one block per host thread."""
    import oracle
    threads = threads or len(os.sched_getaffinity(0))
    blk = 4096
    nblk = max(1, min(pair.a.size, pair.b.size) // blk)
    jobs = [(pair.a[k * blk:(k + 1) * blk], pair.b[k * blk:(k + 1) * blk]) for k in range(nblk)]
    cells = 0
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < budget_s and done < 64:
        batch = jobs[: max(1, threads)]
        oracle.align_many(batch, *SCORING, threads=threads)
        cells += sum(x.size * y.size for x, y in batch)
        done += 1
    dt = time.perf_counter() - t0
    used = min(threads, len(jobs))
    return cells / dt / 1e9, used, f"{done} rounds of {min(threads, len(jobs))} diagonal {blk}x{blk} blocks " \
                                   f"of the pair ({cells:.3g} cells, {dt:.1f} s)"


def allpairs_oracle_gcups(seqs, budget_s: float = 12.0):
    """The CPU oracle, as it stands, on random pairs of the family (score
    only), spread over the host threads."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    rs = seqgen.Stream(4242)
    idx = rs.integers(0, len(seqs) - 1, 4000).reshape(-1, 2)
    pairs = [(seqs[int(i)], seqs[int(j)]) for i, j in idx if i != j]
    t0 = time.perf_counter()
    done, cells = 0, 0
    while time.perf_counter() - t0 < budget_s and done < len(pairs):
        chunk = pairs[done: done + 64]
        oracle.score_many(chunk, *SCORING, threads=threads)
        cells += sum(a.size * b.size for a, b in chunk)
        done += len(chunk)
    dt = time.perf_counter() - t0
    return cells / dt / 1e9, threads, f"{done} random pairs of the family, score only ({cells:.3g} cells, {dt:.1f} s)"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    data, desc = workload(args.workload)
    import oracle
    oracle.build()
    sample_fn = {"allpairs": allpairs_oracle_gcups, "centerstar": allpairs_oracle_gcups,
                 "local": lambda d, budget_s: local_oracle_gcups([(p.a, p.b) for p in d[:400]], budget_s),
                 "affine": lambda d, budget_s: affine_oracle_gcups([(p.a, p.b) for p in d[:400]], budget_s),
                 "band": lambda d, budget_s: oracle_gcups_pairs([(p.a, p.b) for p in d[:400]], budget_s)}.get(
        args.workload, oracle_gcups)
    vals = []
    for _ in range(args.warmup):
        sample_fn(data, budget_s=1.0)
    for _ in range(args.steps):
        g, cores, sample = sample_fn(data, budget_s=max(0.5, 60.0 / max(args.steps, 1)))
        vals.append(g)
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GCUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc, "scoring": list(SCORING)},
            "cpu_baseline": {"value": v, "unit": "GCUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
class PairWork:
    """One pair: pack both sequences on the device, fill with pointers,
    trace back, build the CIGAR."""
    dominant = "bpair_fill_ptr"

    def __init__(self, nw, ctx, dev, name):
        import torch
        self.nw, self.ctx = nw, ctx
        pair, self.desc = workload(name)
        self.pair = pair
        m, n = pair.a.size, pair.b.size
        self.m, self.n, self.cells = m, n, m * n
        self.a_ascii = torch.tensor(np.frombuffer(seqgen.to_ascii(pair.a).encode(), np.uint8), device=dev)
        self.b_ascii = torch.tensor(np.frombuffer(seqgen.to_ascii(pair.b).encode(), np.uint8), device=dev)
        self.a2b = torch.zeros((m + 3) // 4, dtype=torch.uint8, device=dev)
        self.b2b = torch.zeros((n + 3) // 4, dtype=torch.uint8, device=dev)
        self.score = torch.zeros(1, dtype=torch.int32, device=dev)
        self.cigar = torch.zeros(nw.nw_cigar_bound(m, n), dtype=torch.uint8, device=dev)
        self.clen = torch.zeros(1, dtype=torch.int64, device=dev)
        self.a_host = torch.from_numpy(nw.pack_codes(pair.a)).pin_memory().numpy()
        self.b_host = torch.from_numpy(nw.pack_codes(pair.b)).pin_memory().numpy()
        self.config = {"m": m, "n": n}

    def step(self):
        nw = self.nw
        nw.nw_pack_device(self.ctx, self.a_ascii, self.m, self.a2b)
        nw.nw_pack_device(self.ctx, self.b_ascii, self.n, self.b2b)
        nw.nw_align(self.ctx, self.a2b, self.m, self.b2b, self.n, SCORING, nw.NW_CIGAR, self.score, self.cigar,
                    self.clen)

    def e2e(self):
        res = self.nw.nw_align(self.ctx, self.a_host, self.m, self.b_host, self.n, SCORING, self.nw.NW_CIGAR)
        return self.a_host.nbytes + self.b_host.nbytes, 16 + len(res[1]) + 1

    def result(self):
        return {"score": int(self.score.item())}

    def oracle_sample(self):
        return oracle_gcups(self.pair, budget_s=12.0)


class AllPairsWork:
    """All-vs-all int32 score matrix of 512 sequences (130,816 pairs)."""
    dominant = "bits_score"

    def __init__(self, nw, ctx, dev, name):
        import torch
        self.nw, self.ctx = nw, ctx
        seqs, self.desc = workload(name)
        self.seqs = seqs
        pool, off, lens = nw.pool_of(seqs)
        self.pool_host = torch.from_numpy(pool).pin_memory().numpy()
        self.off, self.lens = off, lens
        self.pool = torch.from_numpy(pool).to(dev)
        n = len(seqs)
        self.out = torch.zeros((n, n), dtype=torch.int32, device=dev)
        L = lens.astype(np.float64)
        self.cells = int((np.outer(L, L).sum() - (L * L).sum()) / 2)
        self.config = {"nseq": n, "pairs": n * (n - 1) // 2}

    def step(self):
        # replays the CUDA graph captured on the first (warm-up) call
        self.nw.nw_score_all_pairs(self.ctx, self.pool, self.off, self.lens, SCORING, self.nw.NW_GRAPH, self.out)

    def e2e(self):
        # host pool in, host matrix out; repeated calls replay the captured launches
        res = self.nw.nw_score_all_pairs(self.ctx, self.pool_host, self.off, self.lens, SCORING, self.nw.NW_GRAPH)
        return self.pool_host.nbytes, res.nbytes

    def result(self):
        return {"matrix_checksum": int(self.out.sum().item())}

    def oracle_sample(self):
        return allpairs_oracle_gcups(self.seqs)


class LocalWork:
    """Local alignment of many pairs (score, start, end, CIGAR)."""
    dominant = "local_fill_ptr"

    def __init__(self, nw, ctx, dev, name):
        import torch
        self.nw, self.ctx = nw, ctx
        pairs, self.desc = workload(name)
        self.pairs = pairs
        seqs = []
        for p in pairs:
            seqs += [p.a, p.b]
        pool, off, lens = nw.pool_of(seqs)
        self.pool_host = torch.from_numpy(pool).pin_memory().numpy()
        self.pool = torch.from_numpy(pool).to(dev)
        self.ao, self.al, self.bo, self.bl = off[0::2], lens[0::2], off[1::2], lens[1::2]
        n = len(pairs)
        self.coff = nw._cigar_offsets(self.al, self.bl)
        self.scores = torch.zeros(n, dtype=torch.int32, device=dev)
        self.ends = torch.zeros((n, 4), dtype=torch.int32, device=dev)
        self.cpool = torch.zeros(int(self.coff[-1]), dtype=torch.uint8, device=dev)
        self.clen = torch.zeros(n, dtype=torch.int64, device=dev)
        self.cells = int(sum(int(x) * int(y) for x, y in zip(self.al, self.bl)))
        self.config = {"npairs": n}

    def step(self):
        self.nw.nw_local_align_batch(self.ctx, self.pool, self.ao, self.al, self.bo, self.bl, SCORING,
                                     self.nw.NW_CIGAR, self.scores, self.ends, self.cpool, self.coff, self.clen)

    def e2e(self):
        sc, ends, cig = self.nw.nw_local_align_batch(self.ctx, self.pool_host, self.ao, self.al, self.bo, self.bl,
                                                     SCORING, self.nw.NW_CIGAR)
        return self.pool_host.nbytes, sc.nbytes + ends.nbytes + cig.nbytes() + 8 * len(cig)

    def result(self):
        return {"score_checksum": int(self.scores.sum().item())}

    def oracle_sample(self):
        return local_oracle_gcups([(p.a, p.b) for p in self.pairs[:400]])


AFFINE_SCORING = (2, -3, -5, -2)


class AffineWork:
    """Affine-gap global alignment of many pairs (score + CIGAR)."""
    dominant = "affine_fill_ptr"
    scoring = AFFINE_SCORING

    def __init__(self, nw, ctx, dev, name):
        import torch
        self.nw, self.ctx = nw, ctx
        pairs, self.desc = workload(name)
        self.pairs = pairs
        seqs = []
        for p in pairs:
            seqs += [p.a, p.b]
        pool, off, lens = nw.pool_of(seqs)
        self.pool_host = torch.from_numpy(pool).pin_memory().numpy()
        self.pool = torch.from_numpy(pool).to(dev)
        self.ao, self.al, self.bo, self.bl = off[0::2], lens[0::2], off[1::2], lens[1::2]
        n = len(pairs)
        self.coff = nw._cigar_offsets(self.al, self.bl)
        self.scores = torch.zeros(n, dtype=torch.int32, device=dev)
        self.cpool = torch.zeros(int(self.coff[-1]), dtype=torch.uint8, device=dev)
        self.clen = torch.zeros(n, dtype=torch.int64, device=dev)
        self.cells = int(sum(int(x) * int(y) for x, y in zip(self.al, self.bl)))
        self.config = {"npairs": n}

    def step(self):
        self.nw.nw_affine_align_batch(self.ctx, self.pool, self.ao, self.al, self.bo, self.bl, AFFINE_SCORING,
                                      self.nw.NW_CIGAR, self.scores, self.cpool, self.coff, self.clen)

    def e2e(self):
        sc, cig = self.nw.nw_affine_align_batch(self.ctx, self.pool_host, self.ao, self.al, self.bo, self.bl,
                                                AFFINE_SCORING, self.nw.NW_CIGAR)
        return self.pool_host.nbytes, sc.nbytes + cig.nbytes() + 8 * len(cig)

    def result(self):
        return {"score_checksum": int(self.scores.sum().item())}

    def oracle_sample(self):
        return affine_oracle_gcups([(p.a, p.b) for p in self.pairs[:400]])


def affine_oracle_gcups(pairs, budget_s: float = 12.0):
    """The CPU oracle, as it stands, on affine-gap alignments (score +
    traceback) of pairs of the workload, on all host threads."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    done, cells = 0, 0
    while time.perf_counter() - t0 < budget_s and done < len(pairs):
        chunk = pairs[done: done + threads]
        oracle.affine_align_many(chunk, *AFFINE_SCORING, threads=threads)
        cells += sum(a.size * b.size for a, b in chunk)
        done += len(chunk)
    dt = time.perf_counter() - t0
    return cells / dt / 1e9, threads, f"{done} pairs of the workload, affine score + traceback ({cells:.3g} " \
                                      f"cells, {dt:.1f} s)"


def local_oracle_gcups(pairs, budget_s: float = 12.0):
    """The CPU oracle, as it stands, on local alignments (score, ends and
    traceback) of pairs of the workload, on all host threads."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    done, cells = 0, 0
    while time.perf_counter() - t0 < budget_s and done < len(pairs):
        chunk = pairs[done: done + threads]
        oracle.local_align_many(chunk, *SCORING, threads=threads)
        cells += sum(a.size * b.size for a, b in chunk)
        done += len(chunk)
    dt = time.perf_counter() - t0
    return cells / dt / 1e9, threads, f"{done} pairs of the workload, local score + traceback ({cells:.3g} cells, " \
                                      f"{dt:.1f} s)"


class CenterStarWork:
    """Center-star multiple alignment (Sec. 3.2): scoring matrix, center,
    alignments with the center, merged rows -- all on the device."""
    dominant = "bits_score"

    def __init__(self, nw, ctx, dev, name):
        import torch
        self.nw, self.ctx = nw, ctx
        seqs, self.desc = workload(name)
        self.seqs = seqs
        pool, off, lens = nw.pool_of(seqs)
        self.pool_host = torch.from_numpy(pool).pin_memory().numpy()
        self.off, self.lens = off, lens
        self.pool = torch.from_numpy(pool).to(dev)
        n = len(seqs)
        self.coff = nw._center_cigar_offsets(lens)
        self.sums = torch.zeros(n, dtype=torch.int64, device=dev)
        self.scores = torch.zeros(n, dtype=torch.int32, device=dev)
        self.cpool = torch.zeros(int(self.coff[-1]), dtype=torch.uint8, device=dev)
        self.clen = torch.zeros(n, dtype=torch.int64, device=dev)
        L = lens.astype(np.float64)
        self.pair_cells = int((np.outer(L, L).sum() - (L * L).sum()) / 2)
        # the merged column count first (no rows), then rows of that stride
        self.center, self.cols, ok = nw.nw_center_star(ctx, self.pool, off, lens, SCORING, 0, self.sums, self.scores,
                                                       self.cpool, self.coff, self.clen, None, 0)
        self.ld = self.cols + 1
        self.msa = torch.zeros(n * self.ld, dtype=torch.uint8, device=dev)
        self.cells = self.pair_cells + int((L * L[self.center]).sum())
        self.config = {"nseq": n, "pairs": n * (n - 1) // 2, "center": self.center, "msa_columns": self.cols}

    def step(self):
        # the scoring stage replays the CUDA graph captured on the first call
        self.nw.nw_center_star(self.ctx, self.pool, self.off, self.lens, SCORING, self.nw.NW_GRAPH, self.sums,
                               self.scores, self.cpool, self.coff, self.clen, self.msa, self.ld)

    def e2e(self):
        # host pool in, host results out; repeated calls replay the scoring stage's graph
        res = self.nw.nw_center_star(self.ctx, self.pool_host, self.off, self.lens, SCORING, self.nw.NW_GRAPH)
        out = res["scores"].nbytes + res["row_sums"].nbytes + res["cigars"].nbytes() + \
            sum(len(r) for r in res["rows"])
        return self.pool_host.nbytes, out

    def result(self):
        return {"score_checksum": int(self.scores.sum().item())}

    def oracle_sample(self):
        return allpairs_oracle_gcups(self.seqs)


def train_band_model(nw, ctx, dev, epochs: int = 60, batch: int = 512, lr: float = 2e-3, seed: int = 0):
    """Train the band-width network on the GPU from the committed oracle
    labels (tests/golden/band_labels_seed9004.npz); features of the training
    pairs come from the library's feature kernel.  Returns the final loss."""
    import torch
    lab = np.load(LABELS)
    count = int(lab["label"].size)
    pairs = seqgen.band_pairs(int(lab["seed"]), npairs=count)
    seqs = []
    for p in pairs:
        seqs += [p.a, p.b]
    pool, off, lens = nw.pool_of(seqs)
    feat = nw.nw_band_features(ctx, torch.from_numpy(pool).to(dev), off[0::2], lens[0::2], off[1::2], lens[1::2])
    target = torch.from_numpy(np.log(np.maximum(lab["label"], 1)).astype(np.float32)).to(dev)
    nw.nw_band_model_init(ctx, seed)
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = None
    for _ in range(epochs):
        perm = torch.randperm(count, generator=g).to(dev)
        for k in range(0, count - batch + 1, batch):
            idx = perm[k:k + batch]
            loss = nw.nw_band_model_train_step(ctx, feat[idx].contiguous(), target[idx].contiguous(), lr)
    return float(loss.item()) if loss is not None else None


class BandWork:
    """Certified learned band over many pairs (score + CIGAR); the plain
    full-grid batch runs on the same pairs for comparison."""
    dominant = "bband_fill_ptr"

    def __init__(self, nw, ctx, dev, name):
        import torch
        self.nw, self.ctx, self.dev = nw, ctx, dev
        pairs, self.desc = workload(name)
        self.pairs = pairs
        seqs = []
        for p in pairs:
            seqs += [p.a, p.b]
        pool, off, lens = nw.pool_of(seqs)
        self.pool_host = torch.from_numpy(pool).pin_memory().numpy()
        self.pool = torch.from_numpy(pool).to(dev)
        self.ao, self.al, self.bo, self.bl = off[0::2], lens[0::2], off[1::2], lens[1::2]
        n = len(pairs)
        caps = [nw.nw_cigar_bound(int(x), int(y)) for x, y in zip(self.al, self.bl)]
        self.coff = np.concatenate([[0], np.cumsum(caps)]).astype(np.uint64)
        self.scores = torch.zeros(n, dtype=torch.int32, device=dev)
        self.cpool = torch.zeros(int(self.coff[-1]), dtype=torch.uint8, device=dev)
        self.clen = torch.zeros(n, dtype=torch.int64, device=dev)
        self.cells = int(sum(int(x) * int(y) for x, y in zip(self.al, self.bl)))
        t0 = time.perf_counter()
        self.train_loss = train_band_model(nw, ctx, dev)
        self.train_s = time.perf_counter() - t0
        self.config = {"npairs": n, "train_loss": self.train_loss, "train_seconds": self.train_s}
        self.flags = nw.NW_CIGAR | nw.NW_LEARNED_BAND

    def step(self):
        self.nw.nw_align_batch(self.ctx, self.pool, self.ao, self.al, self.bo, self.bl, SCORING, self.flags,
                               self.scores, self.cpool, self.coff, self.clen)

    def e2e(self):
        sc, cig = self.nw.nw_align_batch(self.ctx, self.pool_host, self.ao, self.al, self.bo, self.bl, SCORING,
                                         self.flags)
        return self.pool_host.nbytes, sc.nbytes + cig.nbytes() + 8 * len(cig)

    def result(self):
        """Plain full-grid batch on the same pairs: time, and score mismatches."""
        import torch
        nw = self.nw
        plain = torch.zeros_like(self.scores)
        cp = torch.zeros_like(self.cpool)
        cl = torch.zeros_like(self.clen)
        nw.nw_align_batch(self.ctx, self.pool, self.ao, self.al, self.bo, self.bl, SCORING, nw.NW_CIGAR, plain, cp,
                          self.coff, cl)
        self.ctx.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nw.nw_align_batch(self.ctx, self.pool, self.ao, self.al, self.bo, self.bl, SCORING, nw.NW_CIGAR, plain, cp,
                          self.coff, cl)
        self.ctx.sync()
        plain_s = time.perf_counter() - t0
        mism = int((plain != self.scores).sum().item())
        cig_len_mism = int((cl != self.clen).sum().item())
        # CIGAR bytes: per pair, mismatching bytes inside [off, off + length)
        # of the two pools (a prefix sum over the byte-wise difference)
        diff = torch.zeros(cp.numel() + 1, dtype=torch.int64, device=cp.device)
        torch.cumsum((cp != self.cpool).to(torch.int32), 0, out=diff[1:])
        start = torch.from_numpy(self.coff[:-1].astype(np.int64)).to(cp.device)
        per_pair = diff[start + self.clen] - diff[start]
        cig_mism = int(((per_pair != 0) | (cl != self.clen)).sum().item())
        del diff
        st = nw.nw_ctx_band_stats(self.ctx)
        # the same certified band without the network (fixed start): what the
        # trained network gains, on the same context (same memory budget and
        # warm scratch) with its model taken out for these calls
        nonet = torch.zeros_like(self.scores)
        params = nw.nw_band_model_get(self.ctx)
        nw.nw_band_model_clear(self.ctx)
        times = []
        for k in range(4):  # (the median of the last three)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nw.nw_align_batch(self.ctx, self.pool, self.ao, self.al, self.bo, self.bl, SCORING, self.flags, nonet, cp,
                              self.coff, cl)
            self.ctx.sync()
            times.append(time.perf_counter() - t0)
        nonet_s = statistics.median(times[1:])
        nw.nw_band_model_set(self.ctx, params)
        nonet_mism = int((nonet != self.scores).sum().item())
        return {"plain_full_gcups": self.cells / plain_s / 1e9, "plain_full_s": plain_s,
                "score_mismatches_vs_plain": mism, "cigar_mismatches_vs_plain": cig_mism,
                "cigar_length_mismatches_vs_plain": cig_len_mism,
                "no_network_gcups": self.cells / nonet_s / 1e9, "no_network_score_mismatches": nonet_mism,
                "band_stats_cumulative": st}

    def oracle_sample(self):
        return oracle_gcups_pairs([(p.a, p.b) for p in self.pairs[:400]])


def oracle_gcups_pairs(pairs, budget_s: float = 12.0):
    """The CPU oracle, as it stands, aligning pairs (score + traceback) on
    all host threads until the budget is spent."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    done, cells = 0, 0
    while time.perf_counter() - t0 < budget_s and done < len(pairs):
        chunk = pairs[done: done + threads]
        oracle.align_many(chunk, *SCORING, threads=threads)
        cells += sum(a.size * b.size for a, b in chunk)
        done += len(chunk)
    dt = time.perf_counter() - t0
    return cells / dt / 1e9, threads, f"{done} pairs of the workload, score + traceback ({cells:.3g} cells, {dt:.1f} s)"


def run_serve(args):
    """Poisson request stream into the continuous-batching server."""
    import torch

    import paper_2412_21103_gb300 as nw

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = nw.Context(local, torch.cuda.current_stream(dev))
    reqs = list(seqgen.serving_stream(1005, rate=args.rate, limit=args.serve_pool))
    seqs = []
    for r in reqs:
        seqs += [r.pair.a, r.pair.b]
    pool, off, lens = nw.pool_of(seqs)
    ao, al, bo, bl = off[0::2], lens[0::2], off[1::2], lens[1::2]
    want = np.array([r.want_cigar for r in reqs], np.uint8)
    cells_of = al.astype(np.float64) * bl.astype(np.float64)
    train_loss = train_band_model(nw, ctx, dev)
    srv = nw.Server(ctx, workers=args.serve_workers, max_batch=args.serve_batch, trace_budget=64 << 30,
                    flags=nw.NW_LEARNED_BAND)
    # warm-up: a few requests through every worker
    srv.submit_many(pool, ao[:16], al[:16], bo[:16], bl[:16], want[:16])
    srv.drain(300.0)
    srv.poll_all()
    arrivals = np.cumsum(-np.log1p(-seqgen.Stream(1005, 77).uniform(int(args.rate * args.duration) + 1)) / args.rate)
    arrivals = arrivals[arrivals < args.duration]
    idx = np.arange(arrivals.size) % len(reqs)
    t0 = time.perf_counter()
    k = 0
    ticket_req = {}
    ticket_lag = {}  # submission minus scheduled arrival (the server's intake can push back)
    done = []
    while k < arrivals.size:
        now = time.perf_counter() - t0
        j = int(np.searchsorted(arrivals, now, side="right"))
        if j > k:
            sel = idx[k:j]
            tick = srv.submit_many(pool, ao[sel], al[sel], bo[sel], bl[sel], want[sel])
            for tt, q, arr in zip(tick, sel, arrivals[k:j]):
                ticket_req[int(tt)] = int(q)
                ticket_lag[int(tt)] = now - float(arr)
            k = j
        else:
            time.sleep(0.0005)
        done += srv.poll_all()
    submit_end = time.perf_counter() - t0
    backlog = srv.stats()
    drained = srv.drain(600.0)
    done += srv.poll_all()
    wall = time.perf_counter() - t0
    lat = np.array([d[4] for d in done]) if done else np.zeros(1)
    # from the scheduled arrival: the server's latency plus the time the
    # request waited to be submitted
    lat_arr = np.array([d[4] + ticket_lag.get(d[0], 0.0) for d in done]) if done else np.zeros(1)
    cells = float(sum(cells_of[ticket_req[d[0]]] for d in done if d[0] in ticket_req))
    ok = sum(1 for d in done if d[1] == nw.NW_OK)
    failed = {}
    for d in done:
        if d[1] != nw.NW_OK:
            failed[int(d[1])] = failed.get(int(d[1]), 0) + 1
    offered = float(cells_of[idx].sum()) / args.duration
    line = {
        "metric": METRIC, "value": cells / wall / 1e9, "unit": "GCUPS", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": (f"serving: Poisson arrivals at {args.rate:,.0f} req/s for {args.duration} s, pair "
                                "lengths log-uniform [50, 50,000], divergence U[0.01,0.30], half score-only / half "
                                f"score+CIGAR, requests cycled from {len(reqs)} drawn from seed 1005; certified learned "
                                f"band, {args.serve_workers} workers, batches of at most {args.serve_batch}, "
                                "64 GiB traceback budget"),
                   "requests": int(arrivals.size), "completed": len(done), "ok": ok, "failed_by_status": failed,
                   "last_failure": srv.last_message(),
                   "drained": drained,
                   "offered_gcups": offered / 1e9, "backlog_at_end_of_arrivals": backlog["waiting"] + backlog["running"],
                   "arrival_window_s": submit_end, "train_loss": train_loss},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max()), "from": "submission"},
        "latency_from_arrival_s": {"p50": float(np.percentile(lat_arr, 50)), "p99": float(np.percentile(lat_arr, 99)),
                                   "max": float(lat_arr.max())},
        "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)
    srv.close()
    ctx.close()


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2412_21103_gb300 as nw

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = nw.Context(local, stream)
    ctx.set_autotune(True)  # the warm-up steps time the candidate shapes
    work = {"allpairs": AllPairsWork, "band": BandWork, "centerstar": CenterStarWork,
            "local": LocalWork, "affine": AffineWork}.get(args.workload, PairWork)(
        nw, ctx, dev, args.workload)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # clock samples: nvidia-smi starts now (it takes a while to print its
    # first line); only the samples inside the timed region are kept
    clk = ClockSampler(local) if not args.no_clocks else _Null()
    clk.__enter__()
    for _ in range(max(args.warmup, 3)):
        work.step()
    ctx.sync()

    # integer-pipe peak (roofline denominator), measured live: the instructions of the cell update, each alone on every SM; the slowest
    # of them bounds the cell rate (3 of them per cell)
    peak_ops = min(nw.nw_peak_int(ctx, kind, 1 << 15) for kind in PEAK_KINDS)
    # measured score-only cell rates (GCUPS) of three instruction mixes of the
    # cell update on every SM: the cell roofline as a measured number
    cell_rates = {f"kind{k}": nw.nw_peak_int(ctx, k, 1 << 15) for k in CELL_KINDS}
    bits_kernel = work.dominant in BITS_KERNELS
    if bits_kernel:
        # the bit-sliced kernels' instructions (LOP3, funnel shift) and their
        # step on independent chains, measured the same way
        bits_rates = {f"kind{k}": nw.nw_peak_int(ctx, k, 1 << 15) for k in BITS_PEAK_KINDS}
        bits_peak = min(bits_rates.values())
        bits_cell_peak = nw.nw_peak_int(ctx, BITS_CELL_KIND, 1 << 13)

    band0 = nw.nw_ctx_band_stats(ctx)["band_cells"]
    ctx.reset_stats()
    ctx.set_profiling(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")     # lets a profiler select the timed steps' launches
    for k in range(args.steps):
        flush.zero_()                       # evict L2 between timed steps
        evs[k][0].record(stream)
        work.step()
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_pop()
    wall1 = time.perf_counter()
    wall = wall1 - wall0
    clk.window(wall0, wall1)
    time.sleep(0.2)                         # the last in-window sample arrives
    clk.__exit__(None, None, None)
    ctx.set_profiling(False)
    ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)
    ctx.sync()
    stats = ctx.kernel_stats()
    band_cells = nw.nw_ctx_band_stats(ctx)["band_cells"] - band0  # the timed steps' banded cells
    if world > 1:
        ms = slowest_rank_ms(ms, dev)
        dist.barrier()

    # end to end through the public API with host buffers, copies inside
    e2e_ms = []
    h2d = d2h = 0
    for k in range(4):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h2d, d2h = work.e2e()
        t1 = time.perf_counter()
        if k:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_val = job_gcups(work.cells, world, slowest_rank_ms(statistics.mean(e2e_ms), dev))

    dl, dms = stats.get(work.dominant, (0, 0.0))
    dom_avg_ms = dms / max(dl, 1)
    # cells the dominant kernel computed per launch: the full grid, or for
    # the banded kernels the band (window) cells they actually swept
    kcells = (band_cells / max(dl, 1)) if "band" in work.dominant else work.cells
    achieved = kcells * OPS_PER_CELL / (dom_avg_ms * 1e-3) / 1e9 if dom_avg_ms else None
    kernel_gcups = kcells / (dom_avg_ms * 1e-3) / 1e9 if dom_avg_ms else None
    cell_peak = max(cell_rates.values())
    launches = sum(v[0] for k_, v in stats.items() if k_ != "peak" and not k_.startswith("host:"))

    line = {
        "metric": METRIC, "value": job_gcups(work.cells, world, ms), "unit": "GCUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": dict(workload=work.desc, scoring=list(getattr(work, "scoring", SCORING)),
                       parallelism=f"replicas{world}",
                       tuning=ctx.tuning(), graphs=ctx.graph_stats(),
                       l2="flushed between timed steps (256 MB device write)", cells=work.cells,
                       **work.config, **work.result()),
        "roofline": {"bound": "alu", "kernel": work.dominant, "achieved": achieved, "peak": peak_ops,
                     "unit": "Gop/s", "frac": (achieved / peak_ops) if achieved else None,
                     "traffic": dram_traffic(work.dominant, args.workload),
                     "traffic_note": "DRAM bytes per launch (ncu, profiles/dram_traffic.json); "
                                     "algorithmic: 0.25 B/cell of pointers for *_ptr kernels, ~0 for score-only",
                     "ops_per_cell": OPS_PER_CELL, "kernel_ms": dom_avg_ms, "cells_per_launch": kcells,
                     "peak_source": "measured live: slowest of nw_peak_int kinds 0/2/4 (DPX add-max, max, prmt; "
                                    "independent chains on every SM)",
                     "w_domain": {"ops_per_cell": W_OPS_PER_CELL,
                                  "achieved": kernel_gcups * W_OPS_PER_CELL if kernel_gcups else None,
                                  "frac": kernel_gcups * W_OPS_PER_CELL / peak_ops if kernel_gcups else None,
                                  "note": "instructions the W-domain cell issues (prmt, add-max, max) against the "
                                          "same peak"},
                     "cell_peak": {"unit": "GCUPS", "value": cell_peak, "kernel_gcups": kernel_gcups,
                                   "frac": kernel_gcups / cell_peak if kernel_gcups else None,
                                   "rates": cell_rates,
                                   "source": "measured live: nw_peak_int kinds 5-7, score-only cells of three "
                                             "instruction mixes, independent chains on every SM; the best"}},
        "kernels": {k_: {"launches": v[0], "ms_total": v[1]} for k_, v in stats.items()},
        "gpu_launches": launches,
        "e2e": {"value": e2e_val, "unit": "GCUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms)},
        "wall_s_timed": wall,
    }
    if bits_kernel:
        line["roofline"] = bits_roofline(work.dominant, args.workload, kcells, dom_avg_ms, bits_peak, bits_cell_peak,
                                         peak_ops)
        line["roofline"].setdefault("alu", {}).setdefault("rates", bits_rates)
        if line["roofline"]["bound"] == "alu":
            line["roofline"]["rates"] = bits_rates
            line["roofline"].pop("alu")
    if not args.no_clocks:
        line["clocks"] = clk.summary()
    if work.dominant == "bpair_fill_ptr" and dom_avg_ms:
        line["roofline"]["chain"] = pair_chain(work.m, work.n, dom_avg_ms, line.get("clocks", {}).get("sm_mhz"))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, cores, sample = work.oracle_sample()
        line["cpu_baseline"] = {"value": g, "unit": "GCUPS", "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def pair_chain(m, n, kernel_ms, sm_mhz):
    """The single-pair kernel against its own bound: the steps on its
    critical path (stripes of 31 rows, one per lane, 32 steps behind the
    previous one; the next warp's first lane 34 chunks of 32 steps behind a
    warp's), the time per step, and the floor of a step (its logic ops on
    one scheduler's 16-lane pipe, 2 cycles each, at the sampled SM clock)."""
    S = -(-m // PAIR_ROWS)
    C = -(-(n + PAIR_ROWS - 1) // 32)
    nwarps = -(-S // 32)
    steps = 32 * ((nwarps - 1) * 34 + C + min(31, S - 1 - 32 * (nwarps - 1)))
    ns = kernel_ms * 1e6 / steps
    out = {"critical_steps": steps, "ns_per_step": ns, "warps": nwarps,
           "alu_ops_per_step": PAIR_ALU_OPS_PER_STEP,
           "note": "a wavefront: each anti-diagonal step of a stripe waits for the previous one; the whole-GPU "
                   "ALU fraction above is small because only one warp per scheduler on ~m/992 schedulers can "
                   "work at a time"}
    if sm_mhz:
        cyc = ns * sm_mhz / 1e3
        floor = 2.0 * PAIR_ALU_OPS_PER_STEP
        out.update({"cycles_per_step": cyc, "floor_cycles_per_step": floor, "frac": floor / cyc})
    return out


def measured_hbm_gbs():
    """The driver's measured copy bandwidth (GB/s) and where it came from."""
    try:
        v = float(json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))["hbm_gbs"])
        return v, "MEASURED_PEAKS.json hbm_gbs (STREAM-style copy, measured on this pool's GB300)"
    except (OSError, KeyError, ValueError):
        return HBM_PEAK_FALLBACK, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def bits_roofline(kernel, workload, cells, kernel_ms, bits_peak, bits_cell_peak, scalar_peak):
    """Roofline of a bit-sliced kernel.  Score-only (bits_score): bound by the
    ALU issue of its word operations, 16 per 32 cells, against the slowest of
    the measured LOP3 / funnel-shift rates.  With pointers (bband_fill_ptr): it
    also writes 0.25 B per window cell, so the line reports the HBM side as
    the bound (pointer bytes per launch over the kernel's time against the
    measured copy bandwidth) with the ALU side beside it."""
    if not kernel_ms or not cells:
        return {"bound": "alu", "kernel": kernel, "achieved": None, "peak": bits_peak, "unit": "Gop/s",
                "frac": None, "traffic": dram_traffic(kernel, workload)}
    sec = kernel_ms * 1e-3
    ptr = kernel in ("bband_fill_ptr", "bpair_fill_ptr")
    ops32 = BITS_PTR_OPS_PER_32 if ptr else BITS_OPS_PER_32
    rows = PAIR_ROWS if kernel == "bpair_fill_ptr" else 32  # grid cells per word step
    alu_achieved = cells * ops32 / rows / sec / 1e9
    gcups = cells / sec / 1e9
    alu = {"bound": "alu", "achieved": alu_achieved, "peak": bits_peak, "unit": "Gop/s",
           "frac": alu_achieved / bits_peak, "ops_per_32_cells": ops32,
           "peak_source": "measured live: slowest of nw_peak_int kinds 8/10 (LOP3, funnel shift; independent "
                          "chains on every SM)"}
    cell = {"unit": "GCUPS", "value": bits_cell_peak, "kernel_gcups": gcups, "frac": gcups / bits_cell_peak,
            "source": "measured live: nw_peak_int kind 11, one bit-sliced anti-diagonal step (32 cells) on "
                      "independent chains on every SM"}
    scalar = {"ops_per_cell": OPS_PER_CELL, "achieved": gcups * OPS_PER_CELL, "peak": scalar_peak,
              "frac": gcups * OPS_PER_CELL / scalar_peak,
              "note": "the scalar unit (4 int32 ops per cell against the DPX/max/prmt peak): above 1 because one "
                      "word op here updates a bit of 32 cells"}
    base = {"kernel": kernel, "kernel_ms": kernel_ms, "cells_per_launch": cells,
            "traffic": dram_traffic(kernel, workload),
            "traffic_note": "DRAM bytes per launch (ncu, profiles/dram_traffic.json); algorithmic: 0.25 B per "
                            "window cell of pointers for bband_fill_ptr, ~0 for score-only"}
    if not ptr:
        return {**alu, **base, "cell_peak": cell, "scalar_unit": scalar}
    if kernel == "bpair_fill_ptr":
        return {**alu, **base, "cell_peak": cell, "scalar_unit": scalar}
    hbm, src = measured_hbm_gbs()
    bytes_ = cells * 0.25
    achieved = bytes_ / sec / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "bytes_per_launch": bytes_, "peak_source": src, **base, "alu": alu, "cell_peak": cell,
            "scalar_unit": scalar}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def window(self, t0, t1):
        pass

    def summary(self):
        return {}


def main():
    args = parse()
    if args.steps is None:
        args.steps = STEPS_DEFAULT.get(args.workload, 10)
    WL_ARGS.update(nseq=args.nseq, m=args.m, npairs=args.npairs)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
