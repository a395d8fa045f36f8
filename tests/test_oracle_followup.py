"""Pins of the oracle's follow-up stage (Sec. V): the residual phase of Eq. phcor against numerical
quadrature of Eq. powlaws, the heterodyne against its special cases and against a noise-free power
law (which it must turn into one line), the complex spectra against the real-series spectra and
Parseval, and the bin-shift projection against a brute-force loop and a straight track (no GPU)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth


def f_of_t(t, f0, k, n):
    # Eq. powlaws written out here: f = f0 / (1 + k (n-1) f0^(n-1) t)^(1/(n-1))
    return f0 / (1.0 + k * (n - 1.0) * f0 ** (n - 1.0) * t) ** (1.0 / (n - 1.0))


@pytest.mark.parametrize("n,f0,fdot0,t", [(5.0, 300.0, 0.04, 1700.0), (2.0, 812.5, 0.9, 900.0),
                                           (7.0, 95.3, 0.002, 9000.0), (2.5, 1500.0, 0.06, 10000.0),
                                           (3.0, 440.0, 1e-9, 50.0)])
def test_residual_phase_equals_quadrature(n, f0, fdot0, t):
    k = O.k_from_spindown(f0, fdot0, n)
    got = float(O.spindown_cycles(t, f0, k, n))
    want, err = integrate.quad(lambda u: f_of_t(u, f0, k, n) - f0, 0.0, t, epsabs=1e-10,
                               epsrel=1e-13, limit=400)
    assert abs(got - want) <= 1e-9 * max(1.0, abs(want)) + 10 * err
    # the leading term: -fdot0 t^2 / 2 for small t
    ts = min(t, 1e-4 * f0 / fdot0)
    assert float(O.spindown_cycles(ts, f0, k, n)) == pytest.approx(-0.5 * fdot0 * ts * ts, rel=1e-3)


def test_braking_index_two_is_the_limit_of_its_neighbours():
    f0, fdot0, t = 612.0, 0.3, 5000.0
    k = O.k_from_spindown(f0, fdot0, 2.0)
    c2 = float(O.spindown_cycles(t, f0, k, 2.0))
    for eps in (1e-6, -1e-6):
        ke = O.k_from_spindown(f0, fdot0, 2.0 + eps)
        assert float(O.spindown_cycles(t, f0, ke, 2.0 + eps)) == pytest.approx(c2, rel=1e-4)


def test_heterodyne_special_cases():
    rng = np.random.default_rng(3)
    h = rng.standard_normal(5000).astype(np.float32)
    z = O.heterodyne(h, 4096.0, 12.5, 300.0, 0.0, 5.0)            # k = 0: nothing to correct
    assert np.array_equal(z.real, h.astype(np.float64)) and not np.any(z.imag)
    z = O.heterodyne(h, 4096.0, 12.5, 300.0, 1e-12, 5.0)
    assert np.allclose(np.abs(z), np.abs(h.astype(np.float64)), rtol=1e-14, atol=0)
    # the correction of sample s depends on its time only: a later start shifts the phases
    za = O.heterodyne(h[1000:], 4096.0, 12.5 + 1000 / 4096.0, 300.0, 1e-12, 5.0)
    assert np.allclose(za, z[1000:], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("n,f0,fdot0", [(5.0, 300.0, 0.5), (3.0, 151.0, 0.3), (2.0, 410.0, 1.0)])
def test_heterodyne_turns_the_power_law_into_one_line(n, f0, fdot0):
    """A noise-free power law sampled at 1024 Hz for 64 s sweeps over many bins; corrected with its
    own (f0, k, n) nearly all of its positive-frequency power sits in the bin of f0 (and the half
    bins beside it), and with a k off by 30% it does not."""
    fs, T = 1024.0, 64.0
    k = O.k_from_spindown(f0, fdot0, n)
    t = np.arange(int(fs * T)) / fs
    h = np.cos(synth.powerlaw_phase(t, f0, k, n))
    f_end = float(f_of_t(T, f0, k, n))
    assert f0 - f_end > 10.0                                   # the raw signal sweeps > 10 Hz

    def line_fraction(kk):
        Z = np.fft.fft(O.heterodyne(h, fs, 0.0, f0, kk, n))
        P = np.abs(Z) ** 2
        j0 = int(round(f0 * T))
        pos = P[1:Z.size // 2].sum()
        return P[j0 - 1:j0 + 2].sum() / pos
    assert line_fraction(k) > 0.98
    assert line_fraction(1.3 * k) < 0.2


def test_complex_spectra_of_a_real_series_and_parseval():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(8192 * 3)
    fs, t_fft = 1024.0, 4.0
    Pc = O.complex_power_spectra(x.astype(np.complex128), fs, t_fft)
    Pr = O.short_power_spectra(x, fs, t_fft)
    N = int(fs * t_fft)
    assert Pc.shape == (Pr.shape[0], N)
    assert np.allclose(Pc[:, :N // 2 + 1], Pr, rtol=2e-6, atol=1e-6 * Pr.max())
    assert np.allclose(Pc[:, 1:N // 2], Pc[:, N - 1:N // 2:-1], rtol=2e-6, atol=1e-6 * Pr.max())
    z = (rng.standard_normal(x.size) + 1j * rng.standard_normal(x.size))
    P = O.complex_power_spectra(z, fs, t_fft)
    hop = N // 2
    for i in (0, 3):
        frame = z[i * hop:i * hop + N]
        assert P[i].astype(np.float64).sum() == pytest.approx(N * np.sum(np.abs(frame) ** 2), rel=1e-6)


def test_projection_equals_a_loop_and_collects_a_straight_track():
    rng = np.random.default_rng(9)
    n_fft, lo, hi, df = 40, 500, 560, 0.25
    fi = rng.integers(0, n_fft, 300)
    bj = rng.integers(lo - 20, hi + 20, 300)
    t_first, t_hop, fdot = 2.0, 4.0, -0.0173
    got = O.project_peaks(fi, bj, t_first, t_hop, df, fdot, lo, hi)
    want = np.zeros(hi - lo + 1, np.int64)
    for i, j in zip(fi.tolist(), bj.tolist()):
        s = math.floor(fdot * (t_first + i * t_hop) / df + 0.5)
        if lo <= j - s <= hi:
            want[j - s - lo] += 1
    assert np.array_equal(got, want)
    # a straight track f0 + fdot t (f0 on a bin centre) lands in the bin of f0
    j0 = 530
    tfi = np.arange(n_fft)
    tbj = np.floor((j0 * df + fdot * (t_first + tfi * t_hop)) / df + 0.5).astype(np.int64)
    c = O.project_peaks(tfi, tbj, t_first, t_hop, df, fdot, lo, hi)
    assert c[j0 - lo] == n_fft and c.sum() == n_fft
    assert O.projection_cr(c + 1, j0 - lo) == 0.0          # no noise spread: CR undefined, 0
    counts = np.array([3, 5, 4, 20, 4, 6, 2], np.int64)
    rest = np.array([3, 5, 4, 4, 6, 2], float)
    assert O.projection_cr(counts, 3) == pytest.approx((20 - rest.mean()) / rest.std(), rel=1e-15)
