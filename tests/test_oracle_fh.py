"""Pins of the oracle's original FrequencyHough form (n = 0; Sec. III Eq. fdotslope) against what
the equation fixes without the x-transform: a direct count in the (f0, fdot) plane, a straight
track with fdot on a grid row (spin-down and spin-up), the grid constants and the covering
(no GPU)."""
import math

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth

ONE = 1 << 32


def fh_grid(bin_lo=300, bin_hi=339, n_fft=24, n_k=9, k_min=0.0, dk=0.0, df=0.37, t_first=0.83,
            t_hop=1.31, band_hz=1.0):
    f_lo, f_hi = bin_lo * df, (bin_hi + 1) * df
    return O.make_grid(O.Grid(n=0.0, df=df, bin_lo=bin_lo, bin_hi=bin_hi, n_fft=n_fft,
                              t_first=t_first, t_hop=t_hop, t_obs=t_first + n_fft * t_hop,
                              n_k=n_k, k_min=k_min, dk=dk, ana_lo=f_lo, ana_hi=f_hi,
                              band_hz=band_hz))


def direct_fdot_plane(g, fi, bj):
    """Count per (k row r, column m) by Eq. fdotslope alone: peak (i, j) covers the frequencies
    f in (f_j - df/2, f_j + df/2] and on row r (fdot = -k_r) the initial frequencies
    f0 = f - fdot t_i; column m holds f0 in (F - (m+1) dx0, F - m dx0] with F = -x0_min.  Cells with
    an interval end within 1e-6 column of the column's ends are returned in `near` (there the
    oracle's 2^-32 lattice decides)."""
    F = -g.x0_min
    cnt = np.zeros((g.n_k, g.n_x0), np.int64)
    near = np.zeros((g.n_k, g.n_x0), bool)
    eps = 1e-6 * g.dx0
    for r in range(g.n_k):
        k = g.k_min + r * g.dk
        for i, j in zip(fi.tolist(), bj.tolist()):
            if not g.bin_lo <= j <= g.bin_hi:
                continue
            t = g.t_first + i * g.t_hop
            lo = (j - 0.5) * g.df + k * t
            hi = (j + 0.5) * g.df + k * t
            for m in range(g.n_x0):
                c_lo, c_hi = F - (m + 1) * g.dx0, F - m * g.dx0
                if lo < c_hi and c_lo < hi:
                    cnt[r, m] += 1
                if min(abs(lo - c_hi), abs(hi - c_lo), abs(lo - c_lo), abs(hi - c_hi)) < eps:
                    near[r, m] = True
    return cnt, near


def test_grid_constants_are_the_classic_resolutions():
    """n = 0: one frequency bin per f0 column, fdot step df / T_obs (one column of drift over the
    observation), candidates' fdot0 = -k."""
    g = fh_grid()
    assert g.dx0 == g.df
    assert g.dk == pytest.approx(g.df / g.t_obs, rel=1e-15)
    assert O.slope(0.0) == 1.0 and O.slope(5.0) == 4.0
    assert float(O.x_of_f(12.5, 0.0)) == -12.5 and float(O.f_of_x(-12.5, 0.0)) == 12.5
    U = np.array(O.edge_positions(g), dtype=np.int64)
    widths = (U[:-1] - U[1:]) / ONE
    assert np.allclose(widths, 1.0, atol=1e-6)        # every bin is one column wide


@pytest.mark.parametrize("k_min_cols", [0.0, -4.0, -9.5])
def test_map_covers_every_strip_both_signs(k_min_cols):
    g0 = fh_grid(n_k=12)
    g = fh_grid(n_k=12, k_min=k_min_cols * g0.dk)
    U = np.array(O.edge_positions(g), dtype=np.int64)
    B, S = (np.array(v, dtype=np.int64) for v in O.fft_shifts(g))
    lo_min = min(((U[-1] - B[i] - r * S[i]) >> 32) for i in range(g.n_fft) for r in (0, g.n_k - 1))
    hi_max = max(((U[0] - B[i] - r * S[i] - 1) >> 32) for i in range(g.n_fft) for r in (0, g.n_k - 1))
    assert 0 <= lo_min <= 2
    assert g.n_x0 - 3 <= hi_max <= g.n_x0 - 1


@pytest.mark.parametrize("seed", range(6))
def test_map_equals_direct_count_in_the_fdot_plane(seed):
    rng = np.random.default_rng(seed)
    bin_lo = int(rng.integers(200, 400))
    g0 = fh_grid(bin_lo=bin_lo, bin_hi=bin_lo + int(rng.integers(3, 9)), n_fft=int(rng.integers(2, 8)),
                 n_k=int(rng.integers(2, 7)), df=float(rng.uniform(0.2, 0.6)))
    k_min = float(rng.choice([0.0, -3.3, -1.7])) * g0.dk
    dk = g0.dk * float(rng.choice([1.0, 0.41, 2.7]))
    g = fh_grid(bin_lo=g0.bin_lo, bin_hi=g0.bin_hi, n_fft=g0.n_fft, n_k=g0.n_k, df=g0.df,
                k_min=k_min, dk=dk)
    fi, bj = synth.random_peaklist(g.n_fft, g.bin_lo - 1, g.bin_hi + 1, 0.35, seed)
    hm = O.hough_map(g, fi, bj)
    assert np.array_equal(hm, O.hough_map_bruteforce(g, fi, bj))
    want, near = direct_fdot_plane(g, fi.astype(np.int64), bj.astype(np.int64))
    # the grid is aligned to the extreme line (x0_min from k_max t_max), so the cells that line
    # touches sit exactly on column ends: there the lattice decides; everywhere else the counts
    # are those of the fdot plane
    assert near.mean() < 0.3
    assert np.array_equal(hm[~near], want[~near])


@pytest.mark.parametrize("fdot_rows,f0", [(5, 118.4), (0, 121.0), (-6, 116.9)])
def test_straight_track_lands_in_one_cell(fdot_rows, f0):
    """Peaks of f(t) = f0 + fdot t with -fdot on a k row put every FFT's line through the cell of
    (f0, k): it counts n_fft, is the global maximum, and its candidate gives f0 within one column
    and fdot0 = -k (Sec. III Eq. fdotslope)."""
    g0 = fh_grid(bin_lo=280, bin_hi=360, n_fft=64, n_k=16)
    g = fh_grid(bin_lo=280, bin_hi=360, n_fft=64, n_k=16, k_min=-8 * g0.dk)
    row = 8 + fdot_rows
    k = g.k_min + row * g.dk
    fi, bj = [], []
    for i in range(g.n_fft):
        t = g.t_first + i * g.t_hop
        j = int(math.floor((f0 - k * t) / g.df + 0.5))
        fi.append(i)
        bj.append(j)
    order = np.lexsort((fi, bj))
    fi = np.array(fi)[order].astype(np.uint32)
    bj = np.array(bj)[order].astype(np.uint32)
    hm = O.hough_map(g, fi, bj)
    m = int(math.floor((-f0 - g.x0_min) / g.dx0))
    assert hm[row, m] == g.n_fft
    assert hm.max() == g.n_fft
    # a strip is one column wide, so a neighbouring k row can reach the full count too (ties go to
    # the lowest row): the candidate is within one row and one column of the track
    cands, _ = O.select_candidates(g, hm)
    best = max(cands, key=lambda c: c["count"])
    assert best["count"] == g.n_fft and abs(best["row"] - row) <= 1
    assert abs(best["f0"] - f0) <= 1.5 * g.dx0
    assert best["fdot0"] == -(g.k_min + best["row"] * g.dk)
    assert best["x0"] == pytest.approx(-best["f0"], rel=1e-15)


def test_generalized_grids_are_unchanged_by_the_n0_form():
    """The n > 1 grids keep their derived fields (k_min >= 0: the k < 0 extension adds nothing)."""
    g = O.make_grid(O.Grid(n=5.0, df=0.5, bin_lo=200, bin_hi=239, n_fft=40, t_first=1.0, t_hop=1.0,
                           t_obs=41.0, n_k=12, ana_lo=100.0, ana_hi=120.0))
    x_top = math.pow(239.5 * 0.5, -4.0)
    x_bot = math.pow(199.5 * 0.5, -4.0)
    k_max = 11 * g.dk
    assert g.x0_min == x_top - 4.0 * k_max * 40.0 - g.dx0
    assert g.n_x0 == int(math.ceil((x_bot - g.x0_min) / g.dx0)) + 1
    with pytest.raises(ValueError):
        O.make_grid(O.Grid(n=5.0, df=0.5, bin_lo=200, bin_hi=239, n_fft=40, t_first=1.0,
                           t_hop=1.0, t_obs=41.0, n_k=12, k_min=-1e-20, ana_lo=100.0, ana_hi=120.0))
