"""Pins of the oracle's peakmap (Sec. III): peak test, equaliser, full chain statistics."""
import math

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth


def test_peak_test_density_is_p0_on_iid_exponential():
    """On an equalised spectrum of iid exp(1) bins, strict local maxima above theta occur with
    probability p0 = e^-t - e^-2t + e^-3t/3 (a one-sided test would give e^-t - e^-2t/2)."""
    rng = np.random.default_rng(3)
    R = rng.exponential(size=(3000, 1202)).astype(np.float32)
    fi, bj = O.peaks_from_equalised(R, 1000, 2.5)
    cells = 3000 * 1200
    p0 = O.p0_local_max(2.5)
    assert abs(len(fi) / cells - p0) < 4 * math.sqrt(p0 / cells)


def test_peak_test_brute_force_and_order():
    rng = np.random.default_rng(4)
    R = rng.exponential(size=(7, 30)).astype(np.float32) * 2
    fi, bj = O.peaks_from_equalised(R, 500, 2.5)
    ref = []
    for j in range(500, 528):
        for i in range(7):
            c = j - 499
            if R[i, c] > 2.5 and R[i, c] > R[i, c - 1] and R[i, c] > R[i, c + 1]:
                ref.append((j, i))
    assert list(zip(bj.tolist(), fi.tolist())) == ref


def test_equaliser_exceedances_follow_its_own_mean():
    """R_j = P_j / S_(j-1) with S independent of P_j: for iid exp(1) power the expected number of
    exceedances of theta is exactly sum_j exp(-theta S_(j-1))."""
    rng = np.random.default_rng(5)
    P = rng.exponential(size=(3000, 1000)).astype(np.float32)
    R, S = O.equalise(P, 300, 899, return_mean=True)
    assert R.dtype == np.float32
    cnt = int((R > 2.5).sum())
    expect = float(np.exp(-2.5 * S.astype(np.float64)).sum())
    assert abs(cnt - expect) < 5 * math.sqrt(expect)


def test_equaliser_is_unbiased_tracks_and_ignores_lines():
    rng = np.random.default_rng(6)
    P = rng.exponential(size=(2000, 2000)).astype(np.float32)
    P[:, 700:] *= 4.0                                  # noise level steps up x4
    P[:, 400] = 1e6                                    # a strong line
    R, S = O.equalise(P, 200, 1997, return_mean=True)
    col = lambda j: j - 199
    # mean level: the clip gain makes the clipped AR mean unbiased (without it S ~ 0.89)
    assert S[:, col(300):col(390)].mean() == pytest.approx(1.0, abs=0.01)
    # tracking: the clip slows the rise (at most 2^-7 (2.5 G - 1) per bin), then the level
    # converges to 4 with a time constant of ~1/(2^-7 (1 - 2.5 G e^-2.5)) ~ 165 bins
    assert S[:, col(1800):col(1890)].mean() == pytest.approx(4.0, rel=0.01)
    # a line moves S by at most one clipped update: 2^-7 (2.5 G - 1) S
    jump = S[:, col(401)] / S[:, col(400)]
    assert jump.max() <= 1 + (2.72356367 - 1) / 128 + 1e-6


def test_noise_only_peakmap_density():
    """Full chain on white noise: density p0 plus the small excess theta^2 var(S)/2 ~ 1.5% that
    any estimated mean adds (Jensen)."""
    x = synth.strain_series(1800 * 1024, 1024.0, seed=11)
    fi, bj = O.peakmap(x, 1024.0, 2.0, 200, 799)
    d = len(fi) / (1799 * 600)
    p0 = O.p0_local_max(2.5)
    assert p0 <= d <= 1.03 * p0
    assert np.all(np.diff(bj.astype(np.int64)) >= 0)


def test_injection_appears_in_peakmap():
    """A strong power-law injection gives a peak at the bin of f(t_i) in most FFTs."""
    f0, n = 350.0, 5.0
    k = 300 * 2.7296915853696254e-17
    inj = synth.Injection(f0=f0, k=k, n=n, amp=synth.amplitude_for_snr(30.0, 1.0, 2048))
    x = synth.strain_series(1800 * 1024, 1024.0, seed=12, injections=(inj,))
    fi, bj = O.peakmap(x, 1024.0, 2.0, 200, 799)
    have = set(zip(fi.tolist(), bj.tolist()))
    hits = 0
    for i in range(1799):
        f = float(O.powerlaw_f(1.0 + i, f0, k, n))
        j = int(math.floor(f / 0.5 + 0.5))
        hits += ((i, j) in have) or ((i, j - 1) in have) or ((i, j + 1) in have)
    assert hits > 0.9 * 1799
