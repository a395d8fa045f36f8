"""Pins of the oracle's closed forms against mathematics the paper fixes (no GPU)."""
import math
import pathlib

import numpy as np
import pytest
from scipy import integrate

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth

CASES = [(350.0, 8.19e-15, 5.0), (993.25, 0.199 / 993.25 ** 7, 7.0), (600.0, 1e-6, 2.0),
         (1200.0, 3e-10, 3.0), (800.0, 2e-9, 2.5)]


@pytest.mark.parametrize("f0,k,n", CASES)
def test_power_law_is_a_line_in_x(f0, k, n):
    """Sec. IV: with x = f^(1-n), Eq. powlaws becomes x = x0 + (n-1) k t exactly."""
    t = np.linspace(0.0, 5000.0, 257)
    x = O.x_of_f(O.powerlaw_f(t, f0, k, n), n)
    line = O.x_of_f(f0, n) + (n - 1.0) * k * t
    assert np.max(np.abs(x / line - 1.0)) < 1e-12


@pytest.mark.parametrize("f0,k,n", CASES)
def test_spindown_law(f0, k, n):
    """Sec. II: Eq. powlaws solves fdot = -k f^n, and k = |fdot0| / f0^n recovers k."""
    t = np.array([10.0, 100.0, 1000.0])
    h = 1e-3
    fd = (O.powerlaw_f(t + h, f0, k, n) - O.powerlaw_f(t - h, f0, k, n)) / (2 * h)
    assert np.allclose(fd, -k * O.powerlaw_f(t, f0, k, n) ** n, rtol=1e-6)
    assert O.k_from_spindown(f0, -k * f0 ** n, n) == pytest.approx(k, rel=1e-14)


@pytest.mark.parametrize("n", [2.0, 3.3, 5.0, 7.0])
def test_inverse_transform(n):
    f = np.array([50.0, 333.3, 1999.75])
    assert np.allclose(O.f_of_x(O.x_of_f(f, n), n), f, rtol=1e-13)


@pytest.mark.parametrize("n", [2.5, 5.0, 7.0])
def test_dk_step_matches_its_taylor_form(n):
    """Sec. VI.B: dk = k((1 + df/f0max)^(-n) - 1) ~ -n k df/f0max for df << f0max."""
    k, f = 3e-15, 1000.0
    for df in (0.5, 0.25, 0.125):
        exact = O.dk_step(k, df, f, n)
        taylor = -n * k * df / f
        assert exact < 0
        # next Taylor term is +n(n+1)/2 (df/f)^2 k
        assert abs(exact / taylor - 1.0) <= (n + 1) / 2 * df / f * 1.01


def test_p0_closed_form():
    """Noise-only peak probability of a strict local maximum above theta for iid exp(1) power."""
    for th in (1.0, 2.5, 4.0):
        q, _ = integrate.quad(lambda x: math.exp(-x) * (1 - math.exp(-x)) ** 2, th, np.inf)
        assert O.p0_local_max(th) == pytest.approx(q, rel=1e-12)
    assert O.p0_local_max(2.5) == pytest.approx(0.0755314, abs=1e-7)


def test_p0_monte_carlo():
    rng = np.random.default_rng(7)
    R = rng.exponential(size=(2000, 2002))
    mid = R[:, 1:-1]
    sel = (mid > 2.5) & (mid > R[:, :-2]) & (mid > R[:, 2:])
    p0 = O.p0_local_max(2.5)
    n = sel.size
    assert abs(sel.mean() - p0) < 4 * math.sqrt(p0 * (1 - p0) / n)


def test_coincidence_distance():
    """Sec. IV: d = sqrt((dx0 bins)^2 + (dk bins)^2)."""
    assert O.coincidence_distance(1.0, 2.0, 1.0 + 3 * 0.1, 2.0 + 4 * 0.01, 0.1, 0.01) == pytest.approx(5.0)


def test_fig_pm_printed_ratio():
    """Fig. pm caption (Sec. IV): the printed x0 and k are both scaled by the same factor relative
    to Eq. transform and k = |fdot0|/f0^n, so their ratio still matches x0/k = f0/|fdot0|."""
    vals = {}
    for line in (pathlib.Path(__file__).parent / "golden" / "fig_pm_example.txt").read_text().splitlines():
        line = line.split("#")[0].strip()
        if line:
            key, val = line.split("=")
            vals[key.strip()] = float(val)
    f0, fdot0, n = vals["f0"], vals["fdot0"], vals["n"]
    x0 = float(O.x_of_f(f0, n))
    k = O.k_from_spindown(f0, fdot0, n)
    assert x0 / k == pytest.approx(f0 / abs(fdot0), rel=1e-12)
    assert vals["x0_printed"] / vals["k_printed"] == pytest.approx(f0 / abs(fdot0), rel=5e-3)
    # the printed values themselves are not reproducible (both off by the same factor ~0.452)
    assert vals["x0_printed"] / x0 == pytest.approx(vals["k_printed"] / k, rel=5e-3)


@pytest.mark.parametrize("f0,k,n", CASES)
def test_injection_phase_is_the_integral_of_f(f0, k, n):
    """The generator's phase is 2 pi times the integral of Eq. powlaws (Sec. V Eq. phcor)."""
    for T in (1.0, 700.0, 3000.0):
        q, _ = integrate.quad(lambda s: float(O.powerlaw_f(s, f0, k, n)), 0.0, T, epsabs=0, epsrel=1e-13, limit=200)
        ph = synth.powerlaw_phase(np.array([T]), f0, k, n)[0]
        assert ph / (2 * np.pi) == pytest.approx(q, rel=1e-10)


def test_amplitude_for_snr():
    """A bin-centred sinusoid of the generator's amplitude has |X|^2 = snr * N sigma^2."""
    N, snr = 2048, 4.0
    A = synth.amplitude_for_snr(snr, 1.0, N)
    t = np.arange(N)
    X = np.fft.rfft(A * np.sin(2 * np.pi * 100 * t / N))
    assert abs(X[100]) ** 2 == pytest.approx(snr * N, rel=1e-9)


# ---- Sec. VI grids on n (Eq. dn_powlaws) and k (Eq. dkeqn) ---------------------------------------

def test_powlaw_ratio_is_the_power_law():
    # f(t) / f0 of Eq. powlaws with k = fdot0 / f0^n, against the formula written in f0, k, t
    for n, f0, fdot0, t in ((2.5, 300.0, 1e-2, 1000.0), (7.0, 120.0, 3e-3, 5000.0), (4.0, 50.0, 1e-4, 10.0)):
        k = fdot0 / f0 ** n
        ref = O.powerlaw_f(t, f0, k, n) / f0
        assert abs(float(O.powlaw_ratio(n, fdot0 * t / f0)) - ref) < 1e-14


def test_n_grid_small_spindown_closed_form():
    """For u = fdot0 t / f0 << 1 the two power laws differ by dn u^2 f0 / 2 (second order of
    Eq. powlaws in n), largest at f_min: the first step is dn = 2 df f_min / (fdot T)^2."""
    df, fmin, fmax, fdot, T = 5e-5, 100.0, 400.0, 1e-5, 1e4      # u <= 1e-3, dn ~ 1
    grid = O.n_grid(3.0, 7.0, df, fmin, fmax, fdot, T)
    dn0 = grid[1] - grid[0]
    ref = 2 * df * fmin / (fdot * T) ** 2
    assert abs(dn0 / ref - 1) < 0.01


def test_n_grid_steps_are_maximal():
    df, fmin, fmax, fdot, T = 0.5, 100.0, 400.0, 0.02, 1800.0
    grid = O.n_grid(2.5, 7.0, df, fmin, fmax, fdot, T)
    assert grid[0] == 2.5 and grid[-1] == 7.0
    assert all(b > a for a, b in zip(grid, grid[1:]))
    for a, b in list(zip(grid, grid[1:]))[:-1][:6]:
        assert O.dn_max_df(a, b, fmin, fmax, fdot, T) <= df * (1 + 1e-9)
        assert O.dn_max_df(a, a + (b - a) * 1.01, fmin, fmax, fdot, T) > df
        # a denser evaluation does not find a larger difference than 1 % above df
        assert O.dn_max_df(a, b, fmin, fmax, fdot, T, n_f=257, n_u=1025) <= df * 1.01
    # steps grow with n (higher n decelerates faster: fewer points, Sec. VI.A)
    steps = np.diff(grid[:-1])
    assert steps[-1] > steps[0]


def test_k_segments_reproduce_eq_dkeqn():
    n, df, fmin, fmax = 5.0, 0.5, 100.0, 400.0
    fdot_lo, fdot_hi = 1e-6, 1e-3
    c = 1 - (1 + df / fmax) ** (-n)
    # growth 1: one row per segment, k_{r+1} = k_r + |dk(k_r)| = k_r (2 - (1 + df/f_max)^-n)
    seg = O.k_segments(n, df, fmin, fmax, fdot_lo, fdot_hi, growth=1.0)
    ks = np.array([s[0] for s in seg])
    assert all(s[2] == 1 for s in seg)
    assert np.allclose(ks[1:] / ks[:-1], 2 - (1 + df / fmax) ** (-n), rtol=1e-12, atol=0)
    assert ks[0] == fdot_lo / fmax ** n and ks[-1] >= fdot_hi / fmin ** n > ks[-2]
    # Taylor form of Eq. dkeqn: |dk| ~ n k df / f_max
    assert abs(seg[0][1] / (n * ks[0] * df / fmax) - 1) < n * df / fmax
    # growth 2: uniform segments never coarser than Eq. dkeqn, contiguous, covering k_hi
    seg2 = O.k_segments(n, df, fmin, fmax, fdot_lo, fdot_hi, growth=2.0)
    for (k0, dk, rows), nxt in zip(seg2, seg2[1:] + [None]):
        assert dk == k0 * c
        last = k0 + (rows - 1) * dk
        assert last * c <= 2.0 * dk * (1 + 1e-12)       # every row's Eq. dkeqn step >= dk / 1
        if nxt is not None:
            assert nxt[0] == k0 + rows * dk
    assert seg2[-1][0] + (seg2[-1][2] - 1) * seg2[-1][1] >= fdot_hi / fmin ** n
    assert sum(r for _, _, r in seg2) < 1.5 * len(seg)
