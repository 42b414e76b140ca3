"""Pins for the CPU reference of the learned band (features, BF16 network,
labels): closed forms, brute force, finite differences."""
import itertools

import numpy as np
import pytest

import oracle
import seqgen
from oracle import band_model as bm


def de_bruijn_4():
    """Order-4 de Bruijn sequence over {0,1,2,3} (every 4-mer once in 259
    bases), by the standard Lyndon-word concatenation."""
    k, n = 4, 4
    a = [0] * (k * n)
    seq = []

    def db(t, p):
        if t > n:
            if n % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            db(t + 1, p)
            for j in range(a[t - p] + 1, k):
                a[t] = j
                db(t + 1, t)
    db(1, 1)
    s = np.array(seq + seq[:3], dtype=np.uint8)
    return s


def test_de_bruijn_has_every_4mer_once():
    s = de_bruijn_4()
    assert s.size == 259
    kms = [bm.kmer(s, i) for i in range(256)]
    assert sorted(kms) == list(range(256))


def test_features_identity_is_one_hot():
    """A == B with all 4-mers distinct: every anchor hits only itself, at
    offset 0, which falls in bin floor(64W/(2W+1)) = 31."""
    s = de_bruijn_4()
    f = bm.features(s, s)
    want = np.zeros(65)
    want[31] = 1.0
    assert np.allclose(f, want)


def test_features_no_common_letter():
    f = bm.features(np.zeros(300, np.uint8), np.full(280, 1, np.uint8))
    assert np.all(f[:64] == 0) and f[64] == pytest.approx(-20 / 300)


def test_features_hit_count_brute_force():
    """Total hits = number of (anchor, j) with equal 4-mers inside the
    window, counted here over all index pairs with numpy."""
    rs = seqgen.Stream(3)
    for m, n in [(40, 55), (300, 260), (9, 9)]:
        a, b = rs.bases(m), rs.bases(n)
        f = bm.features(a, b)
        K = min(256, m - 3)
        counts = np.expm1(f[:64] * np.log1p(K))
        L, delta = max(m, n), n - m
        W = max(1, L // 8)
        ak = np.array([bm.kmer(a, i) for i in range(m - 3)])
        bk = np.array([bm.kmer(b, j) for j in range(n - 3)])
        anchors = [(k * (m - 4)) // (K - 1) for k in range(K)]
        total = 0
        for i in anchors:
            c0 = i + int(round(delta * i / m))
            js = np.arange(n - 3)
            total += int(np.sum((bk == ak[i]) & (np.abs(js - c0) <= W)))
        assert round(counts.sum()) == total


def test_bf16_rounding():
    assert bm.bf16(1.0) == 1.0
    assert bm.bf16(1.0 + 2 ** -8) == 1.0                 # tie -> even
    assert bm.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6   # tie -> even (up)
    assert bm.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7       # representable
    assert bm.bf16(-3.14159) == -3.140625


def _params(seed):
    rs = np.random.default_rng(seed)
    p = rs.normal(0, 0.1, bm.NPARAMS)
    return p


def test_exact_gradient_against_finite_differences():
    p = _params(1)
    X = np.random.default_rng(2).uniform(0, 1, (7, 65))
    t = np.random.default_rng(3).normal(0, 1, 7)
    loss, g = bm.loss_and_grad_exact(p, X, t)
    rs = np.random.default_rng(4)
    for idx in rs.choice(bm.NPARAMS, 40, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[idx] += h
        pm[idx] -= h
        lp = 0.5 * np.mean((bm.forward_exact(pp, X) - t) ** 2)
        lm = 0.5 * np.mean((bm.forward_exact(pm, X) - t) ** 2)
        assert g[idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-4, abs=1e-9)


def test_rounded_gradient_close_to_exact():
    """With BF16 rounding the gradient stays within a few percent of the
    exact one (BF16 keeps 8 significant bits)."""
    p = _params(5)
    X = np.random.default_rng(6).uniform(0, 1, (32, 65))
    t = np.random.default_rng(7).normal(0, 1, 32)
    _, g = bm.loss_and_grad(p, X, t)
    _, ge = bm.loss_and_grad_exact(p, X, t)
    assert np.linalg.norm(g - ge) / np.linalg.norm(ge) < 0.05


def test_band_label_is_minimal_certifying_width():
    for (m, n, s, ex) in [(100, 100, 80, 0), (1000, 950, 600, 12), (500, 800, 100, 300), (10, 10, 10, 0)]:
        w = bm.band_label(m, n, s, ex)
        U = oracle.exit_bound(m, n, w)
        assert U is None or s > U or w == ex
        assert w >= ex
        if w > ex and w > 0:
            U1 = oracle.exit_bound(m, n, w - 1)
            assert U1 is not None and s <= U1


def test_excursion_of_a_path():
    assert bm.excursion("====", 4, 4) == 0
    assert bm.excursion("D=I", 2, 2) == 1
    assert bm.excursion("III====", 7, 4) == 0      # n - m = -3: diagonals -3..0 allowed
    assert bm.excursion("DD==II", 4, 4) == 2


# ------------------------------------------------ features: offsets != 0 ----
ROTATION_BINS = {-32: 0, -31: 0, -20: 11, -7: 24, -1: 30, 1: 32, 5: 36, 13: 44, 31: 62, 32: 63}


@pytest.mark.parametrize("k", sorted(ROTATION_BINS))
def test_features_rotation_lands_in_the_bin_of_its_offset(k):
    """B = the cyclic de Bruijn sequence rotated by k, A unrotated, m = n =
    259 (so the expected diagonal is the main one).  Anchor i (0..255, one per
    position) finds its 4-mer in B only at j = i + k (mod 256), so exactly the
    256 - |k| anchors with 0 <= i + k <= 255 hit, all at offset +k; the other
    occurrence lies 256 - |k| > W = 259 // 8 = 32 diagonals away, outside the
    window.  Hand values of the bin floor((k + 32) * 64 / 65): k = 5 gives
    floor(37 * 64 / 65) = floor(36.43) = 36, k = -7 gives floor(25 * 64 / 65)
    = 24, and so on; a sign flip of the offset or a 2W denominator moves the
    count to another bin."""
    s = de_bruijn_4()
    cyc = s[:256]
    b = np.array([cyc[(j - k) % 256] for j in range(259)], np.uint8)
    f = bm.features(s, b)
    want = np.zeros(65)
    want[ROTATION_BINS[k]] = np.log1p(256 - abs(k)) / np.log1p(256)
    assert np.allclose(f, want, rtol=0, atol=1e-12)


def test_features_expected_diagonal_rounds_the_length_slope():
    """m = 5, n = 9 (delta = 4), A = ACGTG, B = TTTCGTGTT, worked by hand.
    K = min(256, 5 - 3) = 2 anchors at i = floor(k * 1 / 1) = 0, 1 with
    4-mers ACGT and CGTG; W = max(1, 9 // 8) = 1.  e(0) = 0 and e(1) =
    round(4 / 5) = 1, so anchor 1 searches j in [1, 3]; CGTG sits in B at j =
    3 only (B's 4-mers: TTTC TTCG TCGT CGTG GTGT TGTT), offset 3 - 1 - 1 = +1,
    bin floor(2 * 64 / 3) = 42.  ACGT does not occur in B.  So f[42] =
    log1p(1) / log1p(2) and f[64] = 4 / 9.  Flooring e(1) to 0 (window
    [0, 2]) loses the hit; a sign flip puts it in bin 0."""
    lut = {"A": 0, "C": 1, "G": 2, "T": 3}
    a = np.array([lut[x] for x in "ACGTG"], np.uint8)
    b = np.array([lut[x] for x in "TTTCGTGTT"], np.uint8)
    want = np.zeros(65)
    want[42] = np.log(2) / np.log(3)
    want[64] = 4 / 9
    assert np.allclose(bm.features(a, b), want, rtol=0, atol=1e-12)


# -------------------------------------------------------- start width ------
@pytest.mark.parametrize("y,m,n,want", [
    (float(np.log(100.5)), 5000, 6000, 76),   # 0.75 * 100.5 = 75.375 -> 76
    (float(np.log(13.0)), 5000, 5000, 10),    # 0.75 * 13 = 9.75 -> 10
    (float(np.log(9.0)), 5000, 5000, 8),      # 6.75 -> 7, raised to the floor 8
    (0.0, 5000, 5000, 8),                     # 0.75 -> 1 -> 8
    (-50.0, 300, 200, 8),
    (20.0, 3000, 7000, 7000),                 # e^20 * 0.75 far above max(m, n)
    (800.0, 3000, 7000, 7000),                # e^800 overflows a double: still max(m, n)
    (10.0, 5, 3, 5),                          # max(m, n) below the floor: max(m, n) wins
    (-3.0, 5, 3, 5),
])
def test_start_width_hand_values(y, m, n, want):
    assert bm.start_width(y, m, n) == want


# ------------------------------------------- forward: BF16 placements ------
def _index():
    off, k = {}, 0
    for name, size in bm.SIZES:
        off[name] = k
        k += size
    return off


def _hand_network():
    """A network with two live units per layer, worked by hand in exact
    binary fractions.  BF16 keeps 8 significant bits, so on [1, 2) it
    rounds to multiples of 2^-7, ties to an even last bit.

    x0 = 1 + 2^-7 + 2^-9           -> bf16 1 + 2^-7
    W1[0][0] = 1 + 2^-9            -> bf16 1;  b1[0] = 2^-9 (FP32 master, not rounded)
      a1[0] = (1 + 2^-7) + 2^-9     -> H1[0] = bf16 = 1 + 2^-7
    W1[1][0] = -1                   -> a1[1] < 0, H1[1] = 0 (ReLU)
    W2[0][0] = 1 + 2^-9 -> bf16 1;  W2[0][1] = 7 (meets H1[1] = 0);  b2[0] = 2^-9
      a2[0] = (1 + 2^-7) + 2^-9     -> H2[0] = 1 + 2^-7
    W2[1][0] = -1                   -> H2[1] = 0 (ReLU)
    W3[0] = 1 + 2^-8 + 2^-10        -> bf16 1 + 2^-7 (nearer than 1);  W3[1] = 3;  b3 = 0
      y = (1 + 2^-7)^2 = 1 + 2^-6 + 2^-14

    Each rounding step matters: without bf16(x) a1[0] = 1 + 2^-7 + 2^-8 is a
    tie that rounds to 1 + 2^-6; without bf16(W1) a1[0] = 1 + 2^-7 + 2^-8 +
    2^-16 rounds up to 1 + 2^-6; without bf16 on H1 or H2 the value keeps its
    2^-9; without bf16(W3) y gains W3's low bits; without either ReLU the
    weights 7 and 3 meet negative values."""
    off = _index()
    F, H = bm.F, bm.H
    p = np.zeros(bm.NPARAMS)
    p[off["W1"] + 0 * F + 0] = 1 + 2 ** -9
    p[off["b1"] + 0] = 2 ** -9
    p[off["W1"] + 1 * F + 0] = -1.0
    p[off["W2"] + 0 * H + 0] = 1 + 2 ** -9
    p[off["W2"] + 0 * H + 1] = 7.0
    p[off["b2"] + 0] = 2 ** -9
    p[off["W2"] + 1 * H + 0] = -1.0
    p[off["W3"] + 0] = 1 + 2 ** -8 + 2 ** -10
    p[off["W3"] + 1] = 3.0
    x = np.zeros((1, F))
    x[0, 0] = 1 + 2 ** -7 + 2 ** -9
    return p, x


def test_forward_hand_network_rounds_at_every_stage():
    p, x = _hand_network()
    y, _ = bm.forward(p, x)
    assert y[0] == 1 + 2 ** -6 + 2 ** -14


def test_forward_parameter_layout_row_major():
    """W1 is [128][65] and W2 [128][128], row = output unit.  Flat W1 index
    65 + 1 is W1[1][1] (input 1 -> hidden unit 1) and flat W2 index 1 is
    W2[0][1] (hidden unit 1 -> second-layer unit 0); with W3[0] = 3 and
    input 1 = 2, y = 2 * 1 * 1 * 3 = 6.  Read as W1[65][128] the same flat
    index is input 0 -> hidden unit 66, and with W2 transposed it is hidden
    unit 0 -> unit 1: both meet zeros and give y = 0."""
    off = _index()
    F, H = bm.F, bm.H
    p = np.zeros(bm.NPARAMS)
    p[off["W1"] + 1 * F + 1] = 1.0      # hidden unit 1 <- input 1
    p[off["W2"] + 0 * H + 1] = 1.0      # layer-2 unit 0 <- hidden unit 1
    p[off["W3"] + 0] = 3.0
    x = np.zeros((1, F))
    x[0, 1] = 2.0
    y, _ = bm.forward(p, x)
    assert y[0] == 6.0
