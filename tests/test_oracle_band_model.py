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
