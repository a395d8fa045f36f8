"""Pins of the proposal-network oracle against what mathematics and independent library routines
fix: cross-correlation (scipy), adjoint identities, finite differences, closed forms of the loss
and of the optimiser, round-to-nearest-even bf16 (torch's conversion), brute-force image binning,
mass conservation of the tile proposals, and the published first output of splitmix64."""
import math

import numpy as np
import pytest
import scipy.signal
import torch

from oracle import cnn_oracle as C
from paper_1810_09784_gb300 import synth


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: the first output is the finaliser of 0 + golden gamma
    assert int(synth.mix64(np.uint64(0))) == 0xE220A8397B1DCDAF


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -0.0, 0.0, 65504.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(C.bf16_bits(x), ref.view(np.uint16))
    assert C.bf16_bits(1.0 + 2 ** -8) == 0x3F80          # tie to even
    assert C.bf16_bits(1.0 + 3 * 2 ** -8) == 0x3F82


@pytest.mark.parametrize("S", [1, 2])
def test_conv3x3_is_cross_correlation(S):
    rng = np.random.default_rng(S)
    x = rng.standard_normal((2, 12, 12, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    out = C.conv3x3(x, W, S)
    for b in range(2):
        for o in range(4):
            ref = sum(scipy.signal.correlate2d(x[b, :, :, c], W[o, :, :, c], mode="same")
                      for c in range(3))
            np.testing.assert_allclose(out[b, :, :, o], ref[::S, ::S], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("S", [1, 2])
def test_conv3x3_adjoints(S):
    rng = np.random.default_rng(10 + S)
    x = rng.standard_normal((2, 16, 16, 5))
    W = rng.standard_normal((6, 3, 3, 5))
    G = rng.standard_normal((2, 16 // S, 16 // S, 6))
    y = C.conv3x3(x, W, S)
    lhs = float((y * G).sum())
    assert math.isclose(lhs, float((x * C.conv3x3_input_grad(G, W, S, 16)).sum()), rel_tol=1e-11)
    assert math.isclose(lhs, float((W * C.conv3x3_weight_grad(G, x, S)).sum()), rel_tol=1e-11)


def test_softmax_ce_closed_forms():
    logits = np.zeros((3, 257))
    loss, d = C.softmax_ce(logits, np.array([0, 5, 256]))
    np.testing.assert_allclose(loss, math.log(257), rtol=1e-14)
    np.testing.assert_allclose(d.sum(axis=1), 0.0, atol=1e-15)
    assert math.isclose(d[1, 5], (1 / 257 - 1) / 3, rel_tol=1e-12)


def test_head_against_loops():
    rng = np.random.default_rng(3)
    pooled = rng.standard_normal((2, 5, 64))
    WH = rng.standard_normal((64, 3, 64))
    bH = rng.standard_normal(64)
    out = C.head(pooled, WH, bH, 0.25)
    for b in range(2):
        for kt in (0, 17, 63):
            for f in range(5):
                s = bH[kt]
                for d in range(3):
                    if 0 <= f + d - 1 < 5:
                        s += WH[kt, d] @ pooled[b, f + d - 1]
                assert math.isclose(out[b, kt * 5 + f], s, rel_tol=1e-12, abs_tol=1e-12)
    assert np.all(out[:, -1] == 0.25)


def _small_params(seed):
    off, total = C.layout()
    rng = np.random.default_rng(seed)
    p = np.zeros(total)
    for l in range(5):
        o, sh = off[f"W{l + 1}"]
        p[o:o + np.prod(sh)] = rng.uniform(-1, 1, np.prod(sh)) * math.sqrt(6.0 / (9 * C.CIN[l]))
        o, sh = off[f"b{l + 1}"]
        p[o:o + np.prod(sh)] = rng.uniform(0.0, 0.1, np.prod(sh))
    o, sh = off["WH"]
    p[o:o + np.prod(sh)] = rng.uniform(-1, 1, np.prod(sh)) * 0.1
    return p


def test_network_gradient_finite_differences():
    """Directional derivative of the exact (fp64) loss against the oracle's backward pass."""
    rng = np.random.default_rng(5)
    params = _small_params(5)
    images = rng.uniform(0, 2, (2, 16, 16, 2))
    labels = np.array([3 * 4 + 1, 64 * 4])
    cache = C.forward(params, images, mirror=False)
    loss, g = C.backward(cache, labels)
    for trial in range(3):
        v = rng.standard_normal(params.size)
        eps = 1e-6
        lp, _ = C.softmax_ce(C.forward(params + eps * v, images, mirror=False)["logits"], labels)
        lm, _ = C.softmax_ce(C.forward(params - eps * v, images, mirror=False)["logits"], labels)
        fd = (lp.mean() - lm.mean()) / (2 * eps)
        assert math.isclose(fd, float(g @ v), rel_tol=1e-6, abs_tol=1e-9)
    # each block on its own (a wrong index in one layer's gradient cannot hide behind the others)
    off, _ = C.layout()
    for name, (o, sh) in off.items():
        v = np.zeros(params.size)
        v[o:o + np.prod(sh)] = rng.standard_normal(np.prod(sh))
        eps = 1e-6
        lp, _ = C.softmax_ce(C.forward(params + eps * v, images, mirror=False)["logits"], labels)
        lm, _ = C.softmax_ce(C.forward(params - eps * v, images, mirror=False)["logits"], labels)
        fd = (lp.mean() - lm.mean()) / (2 * eps)
        assert math.isclose(fd, float(g @ v), rel_tol=1e-5, abs_tol=1e-9), name


def test_adamw_first_step_closed_form():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    w1, m, v = C.adamw(w, g, np.zeros(3), np.zeros(3), 1, lr=0.01, wd=0.0)
    # bias-corrected first step: m/c1 = g, sqrt(v/c2) = |g|
    np.testing.assert_allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    w2, _, _ = C.adamw(w, np.zeros(3), np.zeros(3), np.zeros(3), 1, lr=0.01, wd=0.1)
    np.testing.assert_allclose(w2, w * (1 - 0.001), rtol=1e-12)


def test_image_counts_brute_force():
    n_fft, lo, hi = 300, 40, 339       # 300 FFTs, 300 bins over 256 pixels: uneven ranges
    f, b = synth.hashed_peaklist(7, 3, n_fft, lo, hi, int(0.05 * 2 ** 24))
    counts = C.image_counts(f, b, n_fft, lo, hi)
    ref = np.zeros((256, 256), np.int64)
    for fi, bj in zip(f.tolist(), b.tolist()):
        tb = next(t for t in range(256) if t * n_fft // 256 <= fi < (t + 1) * n_fft // 256)
        fb = next(x for x in range(256) if x * 300 // 256 <= bj - lo < (x + 1) * 300 // 256)
        ref[tb, fb] += 1
    assert np.array_equal(counts, ref)
    assert counts.sum() == f.size
    bits = C.image_bits(counts, 0.6)
    assert np.all(bits[..., 1] == C.bf16_bits(np.float32(0.6)))
    assert np.all(C.bf16_value(bits[..., 0])[counts == 0] == 0.0)


def test_hashed_peaklist_density_and_track():
    p24 = int(0.0755 * 2 ** 24)
    f, b = synth.hashed_peaklist(1, 0, 1799, 200, 799, p24)
    cells = 1799 * 600
    p = p24 / 2 ** 24
    assert abs(f.size - cells * p) < 5 * math.sqrt(cells * p * (1 - p))
    assert np.all(np.diff(b.astype(np.int64) * 1799 + f) > 0)      # sorted by (bin, fft), unique
    track = np.full(1799, -1)
    track[::2] = 500
    f2, b2 = synth.hashed_peaklist(1, 0, 1799, 200, 799, p24, 1 << 24, track)
    on = (b2 == 500) & (f2 % 2 == 0)
    assert on.sum() == 900                                           # p_track = 1: every cell


def test_proposal_mass_and_identity_gain():
    rng = np.random.default_rng(2)
    logits = rng.standard_normal(4097) * 3
    gain = np.stack([np.linspace(3.0, 1.0, 64), np.linspace(2.5, 0.9, 64)], axis=1)
    sc, pnull = C.tile_scores(logits, gain)
    assert math.isclose(sc.sum() + pnull, 1.0, rel_tol=1e-12)
    # ga = gb = 1: class (d, xt) is k tile d of x0 tile xt
    sc1, _ = C.tile_scores(logits, np.ones((64, 2)))
    p = np.exp(logits - logits.max())
    p /= p.sum()
    np.testing.assert_allclose(sc1, p[:4096], rtol=1e-12)
    top, resid, full = C.propose(logits, np.ones((64, 2)), 32)
    order = np.argsort(-p[:4096], kind="stable")
    assert list(top) == list(order[:32]) and not full
    assert math.isclose(resid, max(0.0, 1 - p[4096] - p[top].sum()), rel_tol=1e-9, abs_tol=1e-12)
    # a threshold cuts the list at the first prefix whose leftover is within it
    cut = 1 - p[4096] - np.cumsum(p[order[:32]])
    n = int(np.argmax(cut <= cut[9])) + 1
    top2, resid2, full2 = C.propose(logits, np.ones((64, 2)), 32, tau=float(cut[9]))
    assert list(top2[:n]) == list(order[:n]) and np.all(top2[n:] == -1) and not full2
    _, _, full3 = C.propose(logits, np.ones((64, 2)), 32, tau=float(cut[31]) / 2)
    assert full3


def test_labels_follow_the_drift_and_gains_cover_the_true_row():
    """The proposer's labels against the physics of the grid: the drift class is the first-order
    drift k f0^n T_obs (Eq. diff_powlaws) in units of K/64 bins, which bounds the power law's actual
    drift from above (the spin-down slows as f falls) and matches it while the drift is small; and
    the k-tile range that the proposal assigns to the label's class holds the true row's k tile."""
    from paper_1810_09784_gb300 import proposer as PR
    spec = PR.ProposerSpec()
    smp = PR.draw(spec, np.arange(0, 400))
    checked = 0
    for b in np.nonzero(smp.signal)[0]:
        n, f0, r = smp.n[b], smp.f0[b], smp.row[b]
        d, xt = divmod(int(smp.labels[b]), 64)
        ga, gb = smp.gain[b, xt]
        kt = r * 64 // spec.n_k
        lo = min(63, math.floor(d * gb))
        hi = min(63, max(lo, math.ceil((d + 1) * ga) - 1))
        assert lo <= kt <= hi, (b, d, xt, kt, lo, hi)
        lin = smp.k[b] * f0 ** n * spec.t_obs / spec.df * 64 / spec.n_k
        if d < 63:
            assert d <= lin < d + 1 + 1e-9, (b, d, lin)
        # actual drift from f(t0) to f(t_obs) in bins, in units of K/64 bins (Eq. powlaws)
        f_end = f0 / (1 + (n - 1) * smp.k[b] * f0 ** (n - 1) * spec.t_obs) ** (1 / (n - 1))
        drift = (f0 - f_end) / spec.df * 64 / spec.n_k
        assert drift <= lin * (1 + 1e-12)
        # second order: 1 - (1 + (n-1) u)^(-1/(n-1)) >= u - n u^2 / 2 with u = k f0^(n-1) T_obs
        u = smp.k[b] * f0 ** (n - 1) * spec.t_obs
        assert drift >= lin * (1 - n * u / 2) - 1e-9, (b, lin, drift, u)
        checked += 1
    assert checked > 150


def test_head_grads_and_pool_grad_are_adjoints():
    """The head is bilinear in (weights, input) plus biases, and the pool is linear: their
    gradients are fixed by <L x, y> = <x, L* y> for each argument on its own.  A transposed tap,
    a dropped bias or a wrong 1/T would break one of these identities."""
    rng = np.random.default_rng(21)
    B, F = 3, 7
    pooled = rng.standard_normal((B, F, 64))
    WH = rng.standard_normal((64, 3, 64))
    bH = rng.standard_normal(64)
    dl = rng.standard_normal((B, 64 * F + 1))
    dWH, dbH, dbnull, dpooled = C.head_grads(dl, pooled, WH)
    z = np.zeros(64)
    lin_in = C.head(pooled, WH, z, 0.0)                    # linear in pooled for fixed WH
    assert math.isclose(float((lin_in * dl).sum()), float((pooled * dpooled).sum()), rel_tol=1e-11)
    assert math.isclose(float((lin_in * dl).sum()), float((WH * dWH).sum()), rel_tol=1e-11)
    only_b = C.head(np.zeros_like(pooled), WH, bH, 0.7)
    assert math.isclose(float((only_b[:, :-1] * dl[:, :-1]).sum()), float(bH @ dbH), rel_tol=1e-11)
    assert math.isclose(float(only_b[:, -1] @ dl[:, -1]), 0.7 * float(dbnull[0]), rel_tol=1e-11)
    # edge taps: logit f = 0 reads no row -1, logit F - 1 no row F
    one = np.zeros_like(dl)
    one[0, 5 * F + 0] = 1.0
    _, _, _, dp = C.head_grads(one, pooled, WH)
    assert np.array_equal(dp[0, 0], WH[5, 1]) and np.array_equal(dp[0, 1], WH[5, 2])
    assert np.all(dp[0, 2:] == 0) and np.all(dp[1:] == 0)
    a = rng.standard_normal((B, 11, F, 64))
    dp2 = rng.standard_normal((B, F, 64))
    assert math.isclose(float((C.pool(a) * dp2).sum()), float((a * C.pool_grad(dp2, 11)).sum()),
                        rel_tol=1e-11)
    np.testing.assert_allclose(C.pool(a), a.sum(axis=1) / 11, rtol=1e-13)


def test_line_scores_against_loops_and_a_planted_track():
    """The non-learned proposer's line sums: against a loop that places each time bin's pixel from
    the drift in floating point (no exact halves occur for K = 500, nb = 600: (2d+1)(2tb+1) 10 is
    never a multiple of 4 plus 1536 mod 3072), and a straight track drawn into an empty image
    scores 256 x its value in its own class, more than in any other class."""
    rng = np.random.default_rng(4)
    K, nb = 500, 600
    img = C.bf16(np.log1p(rng.poisson(1.2, (256, 256))))
    sc = C.line_scores(img, K, nb)
    for d, xt in ((0, 0), (5, 17), (63, 63), (30, 2), (12, 40)):
        best = None
        for c0 in range(4 * xt, 4 * xt + 4):
            s = 0.0
            for tb in range(256):
                off = math.floor((d + 0.5) * K / 64 * 256 / nb * (tb + 0.5) / 256 + 0.5)
                if c0 - off >= 0:
                    s += img[tb, c0 - off]
            best = s if best is None else max(best, s)
        assert math.isclose(sc[d * 64 + xt], best, rel_tol=1e-12), (d, xt)
    empty = np.zeros((256, 256))
    d, xt, c0 = 10, 40, 161
    for tb in range(256):
        empty[tb, c0 - ((2 * d + 1) * (2 * tb + 1) * K + 128 * nb) // (256 * nb)] = 1.0
    s2 = C.line_scores(empty, K, nb)
    assert s2[d * 64 + xt] == 256.0 and np.argmax(s2) == d * 64 + xt
    assert np.sort(s2)[-2] < 256.0
    lg = C.heuristic_logits(s2, 2.0, 0.7, -1.5)
    assert lg.size == 4097
    z = (s2 - s2.mean()) / s2.std()
    np.testing.assert_allclose(lg[:-1], 2.0 * z, rtol=1e-13)
    # the no-signal probability is the logistic function of 0.7 max(z) + 1.5
    p = np.exp(lg - lg.max())
    p /= p.sum()
    assert math.isclose(p[-1], 1.0 / (1.0 + math.exp(0.7 * z.max() + 1.5)), rel_tol=1e-10)
    flat = C.heuristic_logits(np.ones(4096), 3.0, 1.0, 0.0)
    assert np.all(flat[:-1] == 0.0) and math.isclose(flat[-1], math.log(4096), rel_tol=1e-12)
