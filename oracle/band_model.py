"""CPU reference of the learned band's features and network -- TEST
INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``: only tests, the
smoke check and the benchmark's CPU-baseline leg use it).

Not in the paper: the band predictor is an addition around the method.
Definitions (written from the library's documented contract, not from its
code):

features(a, b): K = min(256, m-3) anchors i_k = floor(k*(m-4)/(K-1)) in A;
  e(i) = round-half-even(delta*i/m), delta = n - m; window half-width
  W = max(1, max(m,n)//8); every j in [max(0, i+e(i)-W), min(n-4, i+e(i)+W)]
  whose 4-mer B[j:j+4] equals A[i:i+4] adds 1 to bin
  floor((j - i - e(i) + W) * 64 / (2W+1)); f[b] = log1p(count_b)/log1p(K),
  f[64] = delta / max(m,n).  m < 4 or n < 4: zero histogram.

network: y = W3b . H2 + b3, H2 = bf16(relu(W2b H1 + b2)),
  H1 = bf16(relu(W1b bf16(x) + b1)), where Xb denotes round-to-nearest-even
  BF16 of the FP32 value; loss 0.5*mean((y - t)^2); gradients by the chain
  rule through the same rounded values (the rounding itself is treated as
  identity, as the GPU kernels do).  Computed in float64.
  Parameter layout: W1[128][65], b1[128], W2[128][128], b2[128], W3[128], b3.
"""
from __future__ import annotations

import numpy as np

F, H = 65, 128
SIZES = [("W1", H * F), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H), ("b3", 1)]
NPARAMS = sum(s for _, s in SIZES)


def bf16(x):
    """Round to float32, then to BF16 with round-to-nearest-even; float64 out."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    out = {}
    k = 0
    for name, size in SIZES:
        out[name] = p[k:k + size]
        k += size
    out["W1"] = out["W1"].reshape(H, F)
    out["W2"] = out["W2"].reshape(H, H)
    return out


def kmer(codes, i):
    return int(codes[i]) | int(codes[i + 1]) << 2 | int(codes[i + 2]) << 4 | int(codes[i + 3]) << 6


def features(a, b) -> np.ndarray:
    a = np.asarray(a, dtype=np.uint8)
    b = np.asarray(b, dtype=np.uint8)
    m, n = a.size, b.size
    L = max(m, n)
    delta = n - m
    hist = np.zeros(64, dtype=np.int64)
    K = min(256, m - 3) if (m >= 4 and n >= 4) else 0
    if K:
        bk = [kmer(b, j) for j in range(n - 3)]
        W = max(1, L // 8)
        for k in range(K):
            i = (k * (m - 4)) // (K - 1) if K > 1 else 0
            ak = kmer(a, i)
            e = int(round(delta * i / m))          # Python rounds halves to even
            c0 = i + e
            for j in range(max(0, c0 - W), min(n - 4, c0 + W) + 1):
                if bk[j] == ak:
                    hist[min(max(((j - c0 + W) * 64) // (2 * W + 1), 0), 63)] += 1
    f = np.zeros(F)
    f[:64] = np.log1p(hist) / (np.log1p(K) if K else 1.0)
    f[64] = delta / L if L else 0.0
    return f


def forward(params, X):
    P = unpack(params)
    Xb = bf16(X)
    a1 = Xb @ bf16(P["W1"]).T + P["b1"]
    H1 = bf16(np.maximum(a1, 0.0))
    a2 = H1 @ bf16(P["W2"]).T + P["b2"]
    H2 = bf16(np.maximum(a2, 0.0))
    y = H2 @ bf16(P["W3"]) + P["b3"][0]
    return y, (Xb, H1, H2)


def loss_and_grad(params, X, t):
    P = unpack(params)
    y, (Xb, H1, H2) = forward(params, X)
    B = X.shape[0]
    e = y - t
    loss = 0.5 * float(np.mean(e * e))
    dy = e / B
    gW3 = dy @ H2
    gb3 = np.array([dy.sum()])
    dH2 = np.outer(dy, bf16(P["W3"])) * (H2 > 0)
    gW2 = dH2.T @ H1
    gb2 = dH2.sum(0)
    dH1 = (dH2 @ bf16(P["W2"])) * (H1 > 0)
    gW1 = dH1.T @ Xb
    gb1 = dH1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return loss, g


def forward_exact(params, X):
    """The same network with no rounding (for finite differences)."""
    P = unpack(params)
    H1 = np.maximum(X @ P["W1"].T + P["b1"], 0.0)
    H2 = np.maximum(H1 @ P["W2"].T + P["b2"], 0.0)
    return H2 @ P["W3"] + P["b3"][0]


def loss_and_grad_exact(params, X, t):
    P = unpack(params)
    a1 = X @ P["W1"].T + P["b1"]
    H1 = np.maximum(a1, 0.0)
    a2 = H1 @ P["W2"].T + P["b2"]
    H2 = np.maximum(a2, 0.0)
    y = H2 @ P["W3"] + P["b3"][0]
    B = X.shape[0]
    e = y - t
    dy = e / B
    dH2 = np.outer(dy, P["W3"]) * (a2 > 0)
    dH1 = (dH2 @ P["W2"]) * (a1 > 0)
    g = np.concatenate([(dH1.T @ X).ravel(), dH1.sum(0), (dH2.T @ H1).ravel(), dH2.sum(0), dy @ H2,
                        np.array([dy.sum()])])
    return 0.5 * float(np.mean(e * e)), g


def start_width(y: float, m: int, n: int, margin: float = 0.75) -> int:
    """The first banded round's half-width for a pair whose network output is
    y = log of the predicted half-width: ceil(margin * e^y), at least 8 and at
    most max(m, n).  (y is the FP32 output, widened to float64.)"""
    import math
    y = float(np.float32(y))
    if y > 700.0:  # e^y overflows a double; the clamp gives max(m, n)
        return max(m, n)
    return int(min(max(m, n), max(8, math.ceil(math.exp(y) * margin))))


def band_label(m: int, n: int, score: int, excursion: int, match: int = 1, gap: int = -1) -> int:
    """Training label of a pair: the smallest half-width w whose closed-form
    exit bound lies strictly below the full score (so the certificate accepts
    and the optimal path is inside the band), and at least the traceback's
    excursion from the [min(0,n-m), max(0,n-m)] diagonal range."""
    from . import exit_bound
    lo_w, hi_w = max(0, excursion), max(m, n) + 1
    while lo_w < hi_w:
        mid = (lo_w + hi_w) // 2
        U = exit_bound(m, n, mid, match, gap)
        if U is None or score > U:
            hi_w = mid
        else:
            lo_w = mid + 1
    return max(lo_w, excursion)


def excursion(ops: str, m: int, n: int) -> int:
    """How far the alignment path strays outside the diagonals between 0 and n-m."""
    d_lo, d_hi = min(0, n - m), max(0, n - m)
    i = j = 0
    worst = 0
    for o in ops:
        if o in "=XM":
            i += 1
            j += 1
        elif o == "I":
            i += 1
        else:
            j += 1
        d = j - i
        worst = max(worst, d_lo - d, d - d_hi)
    return worst
