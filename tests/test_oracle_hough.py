"""Pins of the oracle's grid, Hough map and candidate selection (no GPU)."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth

ONE = 1 << 32


def small_grid(n=5.0, bin_lo=200, bin_hi=239, n_fft=40, n_k=12, k_min=0.0, dk=0.0, df=0.5,
               ana=None, band_hz=1.0):
    f_lo, f_hi = bin_lo * df, (bin_hi + 1) * df
    ana_lo, ana_hi = ana if ana else (f_lo, f_hi)
    return O.make_grid(O.Grid(n=n, df=df, bin_lo=bin_lo, bin_hi=bin_hi, n_fft=n_fft, t_first=1.0,
                              t_hop=1.0, t_obs=float(n_fft + 1), n_k=n_k, k_min=k_min, dk=dk,
                              ana_lo=ana_lo, ana_hi=ana_hi, band_hz=band_hz))


def noise_free_track(g: O.Grid, f0: float, row: int):
    """Peaks of a power law with k on grid row `row`: in each FFT, the bin holding f(t_i)."""
    k = g.k_min + row * g.dk
    fi, bj = [], []
    for i in range(g.n_fft):
        t = g.t_first + i * g.t_hop
        f = float(O.powerlaw_f(t, f0, k, g.n))
        j = int(math.floor(f / g.df + 0.5))
        if g.bin_lo <= j <= g.bin_hi:
            fi.append(i)
            bj.append(j)
    order = np.lexsort((fi, bj))
    return np.array(fi)[order].astype(np.uint32), np.array(bj)[order].astype(np.uint32), k


# ---- grid (Sec. VI) ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2.0, 3.0, 5.0, 7.0])
def test_finest_bin_is_one_column(n):
    """Sec. VI.C: dx0 is taken at f_max, so the narrowest bin (the top one) spans just over one
    column and every other bin spans more."""
    g = small_grid(n=n, bin_lo=200, bin_hi=799, n_fft=100)
    U = np.array(O.edge_positions(g), dtype=np.int64)
    widths = (U[:-1] - U[1:]) / ONE
    assert widths.min() >= 1.0 - 1e-9
    assert widths[-1] == pytest.approx(widths.min())
    assert widths[-1] < 1.0 + 1e-3
    # bin widths scale as (f_max / f)^n (derivative of Eq. transform)
    assert widths[0] == pytest.approx((799 / 200) ** n, rel=2e-2)


@pytest.mark.parametrize("n,k_min", [(5.0, 0.0), (7.0, 1e-17), (2.0, 0.0)])
def test_map_covers_every_strip(n, k_min):
    """x0_min and n_x0 bound every peak's interval on every row, with one spare column each side."""
    g = small_grid(n=n, bin_lo=300, bin_hi=340, n_fft=50, n_k=30, k_min=k_min)
    U = np.array(O.edge_positions(g), dtype=np.int64)
    B, S = (np.array(v, dtype=np.int64) for v in O.fft_shifts(g))
    lo_min = min(((U[-1] - B[i] - r * S[i]) >> 32) for i in (0, g.n_fft - 1) for r in (0, g.n_k - 1))
    hi_max = max(((U[0] - B[i] - r * S[i] - 1) >> 32) for i in (0, g.n_fft - 1) for r in (0, g.n_k - 1))
    assert 0 <= lo_min <= 2
    assert g.n_x0 - 3 <= hi_max <= g.n_x0 - 1


def test_default_k_step_is_one_column_over_tobs():
    """dk = dx0/((n-1) T_obs): the last FFT's line moves t/T_obs columns per k row."""
    g = small_grid(n_fft=200)
    _, S = O.fft_shifts(g)
    t_last = g.t_first + (g.n_fft - 1) * g.t_hop
    assert S[-1] / ONE == pytest.approx(t_last / g.t_obs, rel=1e-9)


# ---- Hough map (Sec. IV) ----------------------------------------------------------------------

def random_case(seed):
    rng = np.random.default_rng(seed)
    n = float(rng.choice([2.0, 2.5, 4.0, 5.0, 7.0]))
    bin_lo = int(rng.integers(150, 400))
    nb = int(rng.integers(3, 12))
    n_fft = int(rng.integers(2, 9))
    n_k = int(rng.integers(1, 6))
    g = small_grid(n=n, bin_lo=bin_lo, bin_hi=bin_lo + nb - 1, n_fft=n_fft, n_k=n_k,
                   k_min=float(rng.choice([0.0, 1e-18])))
    if rng.random() < 0.5:   # steep k grid: several columns of drift per row
        g = dataclasses.replace(g, dk=g.dk * float(rng.uniform(2.0, 30.0)))
        g = O.make_grid(dataclasses.replace(g, dx0=0.0, x0_min=0.0, n_x0=0))
    if rng.random() < 0.3:   # clipped map: columns cut on both sides
        g = dataclasses.replace(g, x0_min=g.x0_min + 3 * g.dx0, n_x0=max(1, g.n_x0 // 2))
    fi, bj = synth.random_peaklist(n_fft, g.bin_lo - 1, g.bin_hi + 1, 0.3, seed)
    return g, fi, bj


@pytest.mark.parametrize("seed", range(12))
def test_differential_equals_brute_force(seed):
    """Differential counting + running sum == direct per-cell overlap count on tiny maps."""
    g, fi, bj = random_case(seed)
    a = O.hough_map(g, fi, bj)
    b = O.hough_map_bruteforce(g, fi, bj)
    assert a.shape == (g.n_k, g.n_x0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("n,k_min", [(2.0, 0.0), (4.0, 0.0), (5.0, 3e-9), (7.0, 0.0)])
def test_fft_window_is_exactly_the_meeting_peaks(n, k_min):
    """With k_min >= 0 the shift B_i + r S_i does not fall as i grows (Sec. IV: x0 = x - (n-1) k
    t_i with t_i growing), so the FFTs of one bin whose interval meets a block of rows and columns
    are one contiguous window: those whose right edge on the block's first row is at or right of
    its first column (a prefix of the FFTs) and whose left edge on its last row is left of its
    last column + 1 (a suffix).  Checked against a direct test of every row of the block, the
    window the coarse-tile search walks instead of the bin's whole peak list."""
    g = small_grid(n=n, bin_lo=200, bin_hi=279, n_fft=90, n_k=60, k_min=k_min)
    U = np.array(O.edge_positions(g), dtype=np.int64)
    B, S = (np.array(v, dtype=np.int64) for v in O.fft_shifts(g))
    assert np.all(np.diff(B) >= 0) and np.all(np.diff(S) >= 0)
    rng = np.random.default_rng(int(n * 10))
    for _ in range(40):
        R = int(rng.choice([4, 8, 16]))
        row0 = int(rng.integers(0, g.n_k - R + 1))
        c0 = int(rng.integers(0, g.n_x0))
        ub = min(g.n_x0 - 1, c0 + int(rng.integers(0, 40)))
        for jl in range(g.bin_hi - g.bin_lo + 1):
            # the window: last FFT whose shift on row0 is <= U[jl] - 1 - c0 2^32, first FFT whose
            # shift on the last row exceeds U[jl+1] - (ub + 1) 2^32
            last = int(np.searchsorted(B + row0 * S, U[jl] - 1 - (c0 << 32), side="right")) - 1
            first = int(np.searchsorted(B + (row0 + R - 1) * S, U[jl + 1] - ((ub + 1) << 32),
                                        side="right"))
            window = set(range(first, last + 1))
            # direct: the interval [U[jl+1] - shift, U[jl] - shift) covers a column c0..ub on a row
            direct = set()
            for i in range(g.n_fft):
                for r in range(row0, row0 + R):
                    sh = B[i] + r * S[i]
                    lo, hi = (U[jl + 1] - sh) >> 32, (U[jl] - sh - 1) >> 32
                    if lo <= ub and hi >= c0 and lo <= hi:
                        direct.add(i)
                        break
            assert direct <= window, (jl, row0, R, c0, ub)
            # and the window is exactly the per-peak test of the extreme edges (right edge on
            # the first row, left edge on the last) that every drawn peak passes
            edge_test = {i for i in range(g.n_fft)
                         if ((U[jl] - B[i] - row0 * S[i] - 1) >> 32) >= c0
                         and ((U[jl + 1] - B[i] - (row0 + R - 1) * S[i]) >> 32) <= ub}
            assert edge_test == window, (jl, row0, R, c0, ub)


@pytest.mark.parametrize("seed", range(4))
def test_row_sums_equal_covered_columns(seed):
    """Each row of the map sums to the total number of columns the peaks' intervals overlap,
    computed here from the real-valued interval ends."""
    g, fi, bj = random_case(100 + seed)
    hm = O.hough_map(g, fi, bj)
    a_lo, a_hi, S = O._peak_intervals(g, fi, bj)
    for r in range(g.n_k):
        a = (a_lo - r * S).astype(np.float64) / ONE
        b = (a_hi - r * S).astype(np.float64) / ONE
        lo = np.maximum(np.floor(a), 0)
        hi = np.minimum(np.ceil(b) - 1, g.n_x0 - 1)
        assert hm[r].sum() == int(np.maximum(hi - lo + 1, 0).sum())


def test_sampled_cells_and_rows_agree():
    g, fi, bj = random_case(7)
    hm = O.hough_map(g, fi, bj)
    rng = np.random.default_rng(0)
    rows = rng.integers(0, g.n_k, 50)
    cols = rng.integers(0, g.n_x0, 50)
    assert np.array_equal(O.hough_cells(g, fi, bj, rows, cols), hm[rows, cols])
    for r in range(g.n_k):
        assert np.array_equal(O.hough_row(g, fi, bj, r), hm[r])


@pytest.mark.parametrize("n,f0,row", [(5.0, 380.0, 7), (7.0, 395.0, 3), (2.5, 370.0, 10)])
def test_noise_free_injection_peaks_in_one_cell(n, f0, row):
    """A noise-free power-law track whose k lies on a grid row puts one line per FFT through the
    cell of (x0(f0), k): that cell counts every FFT and is the global maximum (Sec. IV, Fig. hm)."""
    g = small_grid(n=n, bin_lo=300, bin_hi=799, n_fft=300, n_k=16)
    fi, bj, k = noise_free_track(g, f0, row)
    assert len(fi) == g.n_fft
    hm = O.hough_map(g, fi, bj)
    m = int(math.floor((float(O.x_of_f(f0, n)) - g.x0_min) / g.dx0))
    assert hm[row, m] == g.n_fft
    assert hm.max() == g.n_fft


def test_peaks_outside_band_ignored_and_bad_fft_rejected():
    g = small_grid()
    fi = np.array([0, 1, 2], np.uint32)
    bj = np.array([g.bin_lo - 1, g.bin_lo, g.bin_hi + 1], np.uint32)
    hm = O.hough_map(g, fi, bj)
    only = O.hough_map(g, fi[1:2], bj[1:2])
    assert np.array_equal(hm, only)
    with pytest.raises(ValueError):
        O.hough_map(g, np.array([g.n_fft], np.uint32), np.array([g.bin_lo], np.uint32))


# ---- candidates (Sec. IV) ---------------------------------------------------------------------

def brute_select(g, hm):
    f0c, f0n, band = O.column_bands(g)
    out = {}
    for b in range(O.n_bands(g)):
        best = None
        for r in range(g.n_k):
            for m in range(g.n_x0):
                if band[m] == b and (best is None or hm[r, m] > best[0]):
                    best = (int(hm[r, m]), r, m)
        if best:
            out[b] = best
    cells = hm[:, band >= 0].astype(np.float64)
    return out, cells.mean(), cells.std()


@pytest.mark.parametrize("seed", range(6))
def test_select_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    g = small_grid(n=float(rng.choice([3.0, 5.0])), bin_lo=400, bin_hi=419, n_fft=6, n_k=5,
                   ana=(200.5, 207.5), band_hz=float(rng.choice([0.5, 1.0, 2.0])))
    hm = rng.integers(0, 4, size=(g.n_k, g.n_x0)).astype(np.int32)
    cands, (s1, s2, cells) = O.select_candidates(g, hm)
    ref, mu, sd = brute_select(g, hm)
    assert {c["band"]: (c["count"], c["row"], c["col"]) for c in cands} == ref
    for c in cands:
        assert c["cr"] == pytest.approx((c["count"] - mu) / sd, rel=1e-12)
    assert s1 == int(hm[:, O.column_bands(g)[2] >= 0].sum())


def test_select_ties_and_extension():
    """Ties go to the lowest row then column; columns whose f0 is outside the analysis band
    (the peakmap extension of Sec. IV) never give candidates."""
    g = small_grid(n=5.0, bin_lo=400, bin_hi=439, n_fft=6, n_k=4, ana=(200.0, 210.0))
    f0c, _, band = O.column_bands(g)
    assert np.all(band[f0c >= 210.0] == -1) and np.all(band[(f0c < 210.0) & (f0c >= 200.0)] >= 0)
    assert np.all(np.diff(band[band >= 0]) <= 0)          # f0 decreases along x0
    hm = np.zeros((g.n_k, g.n_x0), np.int32)
    cols = np.nonzero(band == 3)[0]
    hm[2, cols[1]] = 9
    hm[1, cols[-1]] = 9
    hm[1, cols[0]] = 9
    ext = np.nonzero(band == -1)[0][0]
    hm[0, ext] = 50
    cands, _ = O.select_candidates(g, hm)
    c3 = [c for c in cands if c["band"] == 3][0]
    assert (c3["row"], c3["col"], c3["count"]) == (1, int(cols[0]), 9)
    assert max(c["count"] for c in cands) == 9


def test_candidate_recovers_injection():
    """The candidate of the injection's band is the injection's cell; its f0, fdot0 come back
    through the inverse of Eq. transform and fdot = -k f^n."""
    n, f0, row = 5.0, 381.3, 9
    g = small_grid(n=n, bin_lo=300, bin_hi=799, n_fft=300, n_k=16, ana=(150.0, 399.0))
    fi, bj, k = noise_free_track(g, f0, row)
    hm = O.hough_map(g, fi, bj)
    cands, _ = O.select_candidates(g, hm)
    best = max(cands, key=lambda c: (c["count"], -c["row"]))
    assert best["count"] == g.n_fft and best["row"] == row
    assert best["band"] == int(f0 - 150.0)
    assert best["f0"] == pytest.approx(f0, abs=g.df)
    assert best["fdot0"] == pytest.approx(-k * f0 ** n, rel=1e-2)
    assert best["cr"] > 10


# ---- squares (Sec. IV) and coincidences ------------------------------------------------------------

def _tiny_map(seed=3, n_k=11):
    from paper_1810_09784_gb300 import synth
    g = O.make_grid(O.Grid(n=4.0, df=0.5, bin_lo=100, bin_hi=140, n_fft=30, t_first=1.0,
                           t_hop=1.0, t_obs=31.0, n_k=n_k, ana_lo=51.0, ana_hi=69.0, band_hz=1.0))
    fi, bj = synth.random_peaklist(30, 98, 142, 0.2, seed)
    return g, O.hough_map(g, fi, bj)


def test_squares_brute_force():
    g, hm = _tiny_map()
    out, (s1, s2, n) = O.select_squares(g, hm, 3, 2, min_dk=3)
    _, _, band = O.column_bands(g)
    cols = [m for m in range(g.n_x0) if band[m] >= 0]
    wa = len(cols)
    for j in range(2):
        rows = list(range(j * g.n_k // 2, (j + 1) * g.n_k // 2))
        for i in range(3):
            cs = cols[i * wa // 3:(i + 1) * wa // 3]
            sq = j * 3 + i
            best = None
            for r in rows:                      # row-major scan: first maximum wins
                for m in cs:
                    if best is None or hm[r, m] > hm[best[0], best[1]]:
                        best = (r, m)
            rec = out[(sq, 0)]
            assert (rec["row"], rec["col"], rec["count"]) == (best[0], best[1], int(hm[best]))
            best2 = None
            for r in rows:
                if abs(r - best[0]) < 3:
                    continue
                for m in cs:
                    if best2 is None or hm[r, m] > hm[best2[0], best2[1]]:
                        best2 = (r, m)
            if best2 is None:
                assert (sq, 1) not in out
            else:
                rec2 = out[(sq, 1)]
                assert (rec2["row"], rec2["col"]) == best2 and rec2["count"] <= rec["count"]
                assert abs(rec2["row"] - rec["row"]) >= 3


def test_one_square_is_the_global_maximum_of_the_band_candidates():
    g, hm = _tiny_map(seed=8)
    out, stats = O.select_squares(g, hm, 1, 1)
    bands, stats_b = O.select_candidates(g, hm)
    assert stats == stats_b
    top = max(bands, key=lambda c: (c["count"], -c["row"], -c["col"]))
    rec = out[(0, 0)]
    assert (rec["count"], rec["row"], rec["col"], rec["cr"]) == (top["count"], top["row"], top["col"], top["cr"])


def test_coincidence_distance_and_radius():
    a = [dict(x0=1.0, k=2.0), dict(x0=10.0, k=5.0), dict(x0=-4.0, k=0.0)]
    b = [dict(x0=1.0 + 3 * 0.5, k=2.0 + 4 * 0.25), dict(x0=10.0, k=5.0 + 2.9 * 0.25),
         dict(x0=1.0 - 3 * 0.5, k=2.0 - 4 * 0.25)]
    match, dist = O.coincidences(a, b, dx0=0.5, dk=0.25, radius=3.0)
    assert dist[0] == 5.0 and match[0] == -1             # 3-4-5 triangle, beyond 3 bins; tie -> index 0
    assert match[1] == 1 and abs(dist[1] - 2.9) < 1e-12
    assert match[2] == -1
    match2, dist2 = O.coincidences(a, b, dx0=0.5, dk=0.25, radius=5.0)
    assert match2[0] == 0 and dist2[0] == 5.0             # equal distances: the lower index
    assert O.coincidences(a, [], 0.5, 0.25) == ([-1, -1, -1], [-1.0, -1.0, -1.0])
