"""CPU oracle of the generalized FrequencyHough hot path (Miller et al., arXiv:1810.09784).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check of the build entry module and the
benchmark's CPU-baseline / reference leg may import or call this module.  The library in
`paper_1810_09784_gb300/` never imports it, and it imports nothing from that library: the two paths
share no code, tables or constants.  Everything here is plain, slow fp64 numpy (pure-Python loops
only for the brute-force checks on tiny inputs), written from the paper's equations:

  Sec. II   Eq. diff_powlaws  fdot = -k f^n;  Eq. powlaws  f(t) = f0 / (1 + k (n-1) f0^(n-1) (t-t0))^(1/(n-1))
  Sec. II   k = |fdot0| / f0^n
  Sec. III  peakmap: equalised spectra, peaks above a threshold that are local maxima
  Sec. IV   Eq. transform  x = 1/f^(n-1), x0 = 1/f0^(n-1);  line x = x0 + (n-1) k (t - t0)
  Sec. III  Eq. fdotslope  (original FrequencyHough, n = 0 here) f0 = f - fdot (t - t0): taken as
            x = -f, x0 = -f0, k = -fdot, so that x0 = x - k (t - t0) has the orientation of
            Eq. transform's x0 = x - (n-1) k (t - t0) with (n-1) replaced by 1
  Sec. IV   each peak is a line in the (x0, k) plane; the Hough map is the histogram of lines
  Sec. IV   candidates per region of the map, critical ratio CR = (y - mu)/sigma, distance d
  Sec. VI.B Eq. dkeqn  dk = k((1 + df/f0max)^(-n) - 1)
  Sec. VI.C dx0 = (n-1) df / f^n taken at the highest frequency f_max
  Sec. VI.D Eq. dot_tfft  fdot <= 1/T_FFT^2 keeps a signal in one bin; T_FFT doubles once the
            spin-down has fallen by 4 (portions of the data)
  Sec. V    Eq. phcor heterodyne correction; complex-series peakmap; bin-shift projection and its CR

Where the paper is silent the readings are fixed here and listed in the design notes:
  * time stamp of FFT i = its centre; t0 = start of the data (Sec. IV, Fig. hm caption)
  * equaliser = clipped auto-regressive mean along frequency with an unbiasing gain (Sec. III
    names only "an auto-regressive mean ... not sensitive to peaks"); boxcar window
  * peak test: R > theta strictly and R strictly above both frequency neighbours, theta = 2.5 (Sec. VII)
  * a peak of bin j covers x in [x(f_j + df/2), x(f_j - df/2)); it counts in every x0 column its
    shifted interval overlaps (positions on a lattice of 2^-32 columns, rounded down)
  * uniform k grid k_r = k_min + r dk; the shift of FFT i on row r is B_i + r S_i on that lattice
  * one candidate per band of `band_hz` in f0: the maximum count, ties to the lowest (row, column);
    columns whose centre f0 lies outside the analysis band are not candidates (Sec. IV, extended band)
  * CR uses the population mean / std over all analysis-band cells of the map

Parity status: every function below is pinned by the CPU tests (closed forms, brute force on tiny
maps, invariants, the noise-only peak density p0; for n = 0 a direct count in the (f0, fdot) plane;
for the heterodyne numerical quadrature of Eq. powlaws; for the portion planner a brute-force
maximum over power laws) except the equaliser's constants, whose values the paper does not give
("parity unpinned" beyond the p0 statistic).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FRAC_BITS = 32                  # fixed-point fraction bits of x0-column positions
THETA = 2.5                     # peak threshold on the equalised spectrum (Sec. VII, Fig. h0mincompar)

# Equaliser reading (Sec. III).  S is an AR(1) mean along frequency with weight 2^-7.  Each bin
# enters as GAIN * P, clipped at CLIP * GAIN * S; GAIN = 1/(1 - exp(-CLIP)) makes the clipped update
# unbiased for exponentially distributed noise power (E[min(P, CLIP mu)] = mu (1 - e^-CLIP)).  The
# estimate starts as the plain mean of WARMUP bins below the first bin that is equalised.  The paper
# fixes no precision; the peak decision is taken in float32 (IEEE-rounded per operation), the
# precision of the GPU kernel, so the constants are float32 values.
AR_WEIGHT = np.float32(0.0078125)       # 2^-7
CLIP = 2.5
GAIN = np.float32(1.08942544)           # float32(1 / (1 - exp(-2.5)))
CLIP_GAIN = np.float32(2.72356367)      # float32(2.5 / (1 - exp(-2.5)))
WARMUP = 128


# ----------------------------------------------------------------------------------------------
# Sec. II / IV closed forms
# ----------------------------------------------------------------------------------------------
def powerlaw_f(t, f0: float, k: float, n: float):
    """Sec. II Eq. powlaws: f(t) = f0 / (1 + k (n-1) f0^(n-1) t)^(1/(n-1)), t measured from t0."""
    return f0 / (1.0 + k * (n - 1.0) * f0 ** (n - 1.0) * np.asarray(t, dtype=np.float64)) ** (1.0 / (n - 1.0))


def k_from_spindown(f0: float, fdot0: float, n: float) -> float:
    """Sec. II: k = |fdot0| / f0^n."""
    return abs(fdot0) / f0 ** n


def x_of_f(f, n: float):
    """Sec. IV Eq. transform: x = 1 / f^(n-1); for n = 0 (original FrequencyHough, Sec. III
    Eq. fdotslope) x = -f."""
    f = np.asarray(f, dtype=np.float64)
    return -f if n == 0.0 else f ** (1.0 - n)


def f_of_x(x, n: float):
    """Inverse of Sec. IV Eq. transform: f = x^(-1/(n-1)); for n = 0, f = -x."""
    x = np.asarray(x, dtype=np.float64)
    return -x if n == 0.0 else x ** (-1.0 / (n - 1.0))


def slope(n: float) -> float:
    """Factor of k t in x0 = x - slope k t: n - 1 (Eq. transform), 1 for n = 0 (Eq. fdotslope)."""
    return 1.0 if n == 0.0 else n - 1.0


def _x_scalar(f: float, n: float) -> float:
    return -f if n == 0.0 else math.pow(f, 1.0 - n)


def dk_step(k: float, df: float, f0max: float, n: float) -> float:
    """Sec. VI.B Eq. dkeqn: dk = k((1 + df/f0max)^(-n) - 1) (negative; its magnitude is the step)."""
    return k * ((1.0 + df / f0max) ** (-n) - 1.0)


# ---- Sec. VI grids on n and k -------------------------------------------------------------------

def powlaw_ratio(n: float, u):
    """f(t)/f0 of Eq. powlaws as a function of u = |fdot0| t / f0 (k = |fdot0| / f0^n):
    (1 + (n-1) u)^(-1/(n-1))."""
    u = np.asarray(u, dtype=np.float64)
    return np.exp(-np.log1p((n - 1.0) * u) / (n - 1.0))


def dn_max_df(n1: float, n2: float, f_min: float, f_max: float, fdot_hi: float, t_obs: float,
              n_f: int = 64, n_u: int = 256) -> float:
    """Largest frequency difference (Eq. dn_powlaws) between the power laws of braking indices n1
    and n2 with the same f0 and fdot0, over f0 on n_f log-spaced values in [f_min, f_max] and u =
    |fdot0| t / f0 on n_u equal steps in [0, fdot_hi t_obs / f0]."""
    best = 0.0
    for a in range(n_f):
        f0 = f_min * (f_max / f_min) ** (a / (n_f - 1)) if n_f > 1 else f_min
        u = fdot_hi * t_obs / f0 * np.arange(n_u) / (n_u - 1)
        d = f0 * np.abs(powlaw_ratio(n2, u) - powlaw_ratio(n1, u))
        best = max(best, float(d.max()))
    return best


def n_grid(n_lo: float, n_hi: float, df: float, f_min: float, f_max: float, fdot_hi: float,
           t_obs: float, rel_tol: float = 1e-9, max_points: int = 100000):
    """Braking indices from n_lo: each step dn the largest (bisection) keeping the Eq. dn_powlaws
    frequency difference within df over the observation; the last point is n_hi or the first
    point beyond it."""
    out = [n_lo]
    n = n_lo
    while n < n_hi and len(out) < max_points:
        span = n_hi - n
        if dn_max_df(n, n + span, f_min, f_max, fdot_hi, t_obs) <= df:
            out.append(n_hi)
            break
        lo, hi = 0.0, span
        while hi - lo > rel_tol * hi:
            mid = 0.5 * (lo + hi)
            if dn_max_df(n, n + mid, f_min, f_max, fdot_hi, t_obs) <= df:
                lo = mid
            else:
                hi = mid
        if lo <= 0.0:
            raise ValueError("no braking-index step keeps the frequency difference within df")
        n = n + lo
        out.append(n)
    return out


def k_segments(n: float, df: float, f_min: float, f_max: float, fdot_lo: float, fdot_hi: float,
               growth: float = 1.0, max_rows: int = 1 << 30):
    """Eq. dkeqn k grid (Sec. VI.B) as uniform segments [(k_start, dk, rows)].  |dk(k)| =
    k (1 - (1 + df/f_max)^(-n)); a segment starting at k_s has step |dk(k_s)| and the rows m whose
    k_s + m dk_s keeps |dk| within growth dk_s (m <= (growth - 1) / c, at most max_rows); the next
    starts one step after its last row; the grid ends at the first row >= k_hi."""
    c = 1.0 - (1.0 + df / f_max) ** (-n)
    k_lo, k_hi = fdot_lo / f_max ** n, fdot_hi / f_min ** n
    rows_full = min(int(math.floor((growth - 1.0) / c)) + 1, max_rows)
    out, k = [], k_lo
    while True:
        dk = k * c
        rows = rows_full
        # stop at the first row >= k_hi
        need = int(math.ceil((k_hi - k) / dk)) + 1 if k < k_hi else 1
        rows = max(1, min(rows, need))
        out.append((k, dk, rows))
        last = k + (rows - 1) * dk
        if last >= k_hi:
            break
        k = k + rows * dk
    return out


def coincidence_distance(x0_a, k_a, x0_b, k_b, dx0: float, dk: float):
    """Sec. IV distance between two points of the (x0, k) plane in units of bins."""
    return np.sqrt(((np.asarray(x0_b) - x0_a) / dx0) ** 2 + ((np.asarray(k_b) - k_a) / dk) ** 2)


def p0_local_max(theta: float) -> float:
    """Probability that a bin of an iid exp(1) spectrum exceeds theta and both neighbours:
    integral_theta^inf e^-x (1 - e^-x)^2 dx = e^-theta - e^-2theta + e^-3theta / 3."""
    return math.exp(-theta) - math.exp(-2 * theta) + math.exp(-3 * theta) / 3.0


# ----------------------------------------------------------------------------------------------
# Sec. VI grids
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Grid:
    """One Hough map: braking index, peakmap band, time stamps, k grid, analysis band."""

    n: float
    df: float               # frequency bin width 1/T_FFT
    bin_lo: int             # peakmap band: bins bin_lo..bin_hi (f_j = j df)
    bin_hi: int
    n_fft: int
    t_first: float          # time of FFT 0 from t0 (its centre)
    t_hop: float            # time between FFTs
    t_obs: float            # observation time
    n_k: int                # k rows
    k_min: float = 0.0
    dk: float = 0.0         # 0: dx0 / ((n-1) T_obs), one x0 column of drift over T_obs per row
    f_max: float = 0.0      # 0: bin_hi * df, the highest frequency of the band (Sec. VI.C)
    ana_lo: float = 0.0     # analysis band [ana_lo, ana_hi) for candidates
    ana_hi: float = 0.0
    band_hz: float = 1.0    # candidate band width in f0
    # derived by make_grid
    dx0: float = 0.0
    x0_min: float = 0.0
    n_x0: int = 0


def make_grid(g: Grid) -> Grid:
    """Fill the derived fields: dx0 (Sec. VI.C, finest step at f_max), dk, x0_min, n_x0.

    x0_min is one column left of the lowest x0 any peak can reach, x(f_top edge) - (n-1) k_max t_max
    (no move for k_max <= 0); n_x0 reaches one column past the highest, x(f_bottom edge), moved by
    -(n-1) k_min t_max when k_min < 0.  n = 0 is the original FrequencyHough (x = -f, slope 1,
    dx0 = df, default dk = df / T_obs); only it takes k_min < 0 (spin-up).
    """
    g = dataclasses.replace(g)
    n = g.n
    if not (n > 1.0 or n == 0.0) or g.bin_lo < 1 or g.bin_hi < g.bin_lo or g.n_fft < 1 or g.n_k < 1:
        raise ValueError("invalid grid request")
    if g.k_min < 0.0 and n != 0.0:
        raise ValueError("k_min < 0 needs n = 0")
    m = slope(n)
    if g.f_max <= 0.0:
        g.f_max = g.bin_hi * g.df
    g.dx0 = m * g.df / math.pow(g.f_max, n)
    if g.dk <= 0.0:
        g.dk = g.dx0 / (m * g.t_obs)
    k_max = g.k_min + (g.n_k - 1) * g.dk
    t_max = g.t_first + (g.n_fft - 1) * g.t_hop
    x_top = _x_scalar((g.bin_hi + 0.5) * g.df, n)
    x_bot = _x_scalar((g.bin_lo - 0.5) * g.df, n)
    g.x0_min = x_top - m * max(k_max, 0.0) * t_max - g.dx0
    x0_hi = x_bot - m * g.k_min * t_max if g.k_min < 0.0 else x_bot
    g.n_x0 = int(math.ceil((x0_hi - g.x0_min) / g.dx0)) + 1
    return g


def fixed_floor(v: float) -> int:
    """floor(v * 2^32) as an exact integer."""
    return math.floor(math.ldexp(v, FRAC_BITS))


def edge_positions(g: Grid) -> list:
    """U_e, e = 0..J: x of the bin edge f = (bin_lo + e - 1/2) df (Sec. IV Eq. transform), as an
    x0-column position (x - x0_min)/dx0 on the 2^-32 lattice.  Bin j spans edges j-bin_lo
    (lower f, larger x) and j-bin_lo+1 (upper f, smaller x)."""
    J = g.bin_hi - g.bin_lo + 1
    out = []
    for e in range(J + 1):
        x = _x_scalar((g.bin_lo + e - 0.5) * g.df, g.n)
        out.append(fixed_floor((x - g.x0_min) / g.dx0))
    return out


def fft_shifts(g: Grid):
    """(B_i, S_i): the shift (n-1) k t_i / dx0 of Sec. IV's line (k t_i / dx0 for n = 0), for
    k = k_min (B) and per k row (S), on the 2^-32 column lattice.  t_i = t_first + i t_hop."""
    B, S = [], []
    m = slope(g.n)
    for i in range(g.n_fft):
        t = g.t_first + i * g.t_hop
        B.append(fixed_floor(m * g.k_min * t / g.dx0))
        S.append(fixed_floor(m * g.dk * t / g.dx0))
    return B, S


def _peak_intervals(g: Grid, fft_idx, bins):
    """Per in-band peak: (A_lo, A_hi, S) so that on row r its x0 interval is [A_lo - rS, A_hi - rS)."""
    fft_idx = np.asarray(fft_idx, dtype=np.int64)
    bins = np.asarray(bins, dtype=np.int64)
    if fft_idx.size and (fft_idx.min() < 0 or fft_idx.max() >= g.n_fft):
        raise ValueError("fft index out of range")
    keep = (bins >= g.bin_lo) & (bins <= g.bin_hi)
    fi, bj = fft_idx[keep], bins[keep] - g.bin_lo
    U = np.array(edge_positions(g), dtype=np.int64)
    B, S = (np.array(v, dtype=np.int64) for v in fft_shifts(g))
    a_lo = U[bj + 1] - B[fi]        # upper-f edge: smallest x
    a_hi = U[bj] - B[fi]            # lower-f edge: largest x
    return a_lo, a_hi, S[fi]


# ----------------------------------------------------------------------------------------------
# Sec. IV Hough map
# ----------------------------------------------------------------------------------------------
def hough_map(g: Grid, fft_idx, bins) -> np.ndarray:
    """Integer Hough map [n_k][n_x0] by differential counting: per row, +1 at the first column a
    peak's interval touches, -1 after the last, then a running sum along x0 (Sec. IV, Sec. VI.C)."""
    W, K = g.n_x0, g.n_k
    a_lo, a_hi, S = _peak_intervals(g, fft_idx, bins)
    out = np.zeros((K, W), dtype=np.int32)
    for r in range(K):
        lo = (a_lo - r * S) >> FRAC_BITS
        hi = ((a_hi - r * S) - 1) >> FRAC_BITS
        lo = np.maximum(lo, 0)
        hi = np.minimum(hi, W - 1)
        ok = lo <= hi
        d = np.bincount(lo[ok], minlength=W + 1) - np.bincount(hi[ok] + 1, minlength=W + 1)
        out[r] = np.cumsum(d[:W])
    return out


def hough_map_bruteforce(g: Grid, fft_idx, bins) -> np.ndarray:
    """Same map by direct definition, cell by cell: count(r, m) = number of peaks whose interval on
    row r overlaps column m, i.e. A_lo - rS < (m+1) 2^32 and A_hi - rS > m 2^32.  Tiny maps only."""
    a_lo, a_hi, S = _peak_intervals(g, fft_idx, bins)
    one = 1 << FRAC_BITS
    out = np.zeros((g.n_k, g.n_x0), dtype=np.int32)
    for r in range(g.n_k):
        for m in range(g.n_x0):
            c = 0
            for p in range(len(a_lo)):
                a = int(a_lo[p]) - r * int(S[p])
                b = int(a_hi[p]) - r * int(S[p])
                if a < (m + 1) * one and b > m * one:
                    c += 1
            out[r, m] = c
    return out


def hough_cells(g: Grid, fft_idx, bins, rows, cols) -> np.ndarray:
    """Counts of the listed cells (rows[q], cols[q]) by the direct definition, vectorised over peaks."""
    a_lo, a_hi, S = _peak_intervals(g, fft_idx, bins)
    one = np.int64(1 << FRAC_BITS)
    out = np.empty(len(rows), dtype=np.int64)
    for q, (r, m) in enumerate(zip(rows, cols)):
        a = a_lo - np.int64(r) * S
        b = a_hi - np.int64(r) * S
        out[q] = np.count_nonzero((a < (np.int64(m) + 1) * one) & (b > np.int64(m) * one))
    return out


def hough_row(g: Grid, fft_idx, bins, r: int) -> np.ndarray:
    """One row of the map (differential counting), for large maps where the full map is too slow."""
    W = g.n_x0
    a_lo, a_hi, S = _peak_intervals(g, fft_idx, bins)
    lo = np.maximum((a_lo - r * S) >> FRAC_BITS, 0)
    hi = np.minimum(((a_hi - r * S) - 1) >> FRAC_BITS, W - 1)
    ok = lo <= hi
    d = np.bincount(lo[ok], minlength=W + 1) - np.bincount(hi[ok] + 1, minlength=W + 1)
    return np.cumsum(d[:W]).astype(np.int32)


# ----------------------------------------------------------------------------------------------
# Sec. IV candidates
# ----------------------------------------------------------------------------------------------
def column_bands(g: Grid):
    """Per x0 column m: the f0 of its centre (inverse of Eq. transform), f0^n, and its candidate
    band index (floor((f0 - ana_lo)/band_hz), or -1 outside the analysis band)."""
    W = g.n_x0
    nb = n_bands(g)
    f0c = np.zeros(W)
    f0n = np.zeros(W)
    band = np.full(W, -1, dtype=np.int64)
    for m in range(W):
        x0c = g.x0_min + (m + 0.5) * g.dx0
        if g.n == 0.0:
            f = -x0c
        elif x0c > 0.0:
            f = math.pow(x0c, -1.0 / (g.n - 1.0))
        else:
            continue
        if f <= 0.0:
            continue
        f0c[m] = f
        f0n[m] = math.pow(f, g.n)
        if g.ana_lo <= f < g.ana_hi:
            band[m] = min(math.floor((f - g.ana_lo) / g.band_hz), nb - 1)
    return f0c, f0n, band


def n_bands(g: Grid) -> int:
    return int(math.ceil((g.ana_hi - g.ana_lo) / g.band_hz))


def select_candidates(g: Grid, hmap: np.ndarray):
    """One candidate per f0 band: the cell of highest count over all rows and the band's columns,
    ties to the lowest row then column; CR = (y - mu)/sigma over all analysis-band cells (Sec. IV).

    Returns a list of dicts (bands without any column give no record) and (sum_y, sum_y2, n_cells).
    """
    f0c, f0n, band = column_bands(g)
    K = g.n_k
    ana = band >= 0
    n_cells = K * int(np.count_nonzero(ana))
    sub = hmap[:, ana].astype(np.int64)
    s1 = int(sub.sum())
    s2 = int((sub * sub).sum())
    if n_cells > 0:
        mu = float(s1) / float(n_cells)
        var = float(s2) / float(n_cells) - mu * mu
        sigma = math.sqrt(var) if var > 0.0 else 0.0
    else:
        mu, sigma = 0.0, 0.0
    out = []
    for b in range(n_bands(g)):
        cols = np.nonzero(band == b)[0]
        if cols.size == 0:
            continue
        block = hmap[:, cols]
        flat = int(np.argmax(block))               # first maximum in (row, column) order
        r, c = divmod(flat, cols.size)
        m = int(cols[c])
        y = int(hmap[r, m])
        cr = (y - mu) / sigma if sigma > 0.0 else 0.0
        k = g.k_min + r * g.dk
        out.append(dict(band=b, row=r, col=m, count=y, cr=cr,
                        x0=g.x0_min + (m + 0.5) * g.dx0, k=k,
                        f0=float(f0c[m]), fdot0=-(k * float(f0n[m]))))
    return out, (s1, s2, n_cells)


def _record(g: Grid, hmap, r: int, m: int, mu: float, sigma: float, f0c, f0n, **extra):
    y = int(hmap[r, m])
    k = g.k_min + r * g.dk
    return dict(row=r, col=m, count=y, cr=(y - mu) / sigma if sigma > 0.0 else 0.0,
                x0=g.x0_min + (m + 0.5) * g.dx0, k=k, f0=float(f0c[m]),
                fdot0=-(k * float(f0n[m])), **extra)


def select_squares(g: Grid, hmap: np.ndarray, n_sx: int, n_sk: int, min_dk: int = 3):
    """Candidates per "square" (Sec. IV): the analysis columns and the k rows are each split into
    equal chunks (n_sx along x0, n_sk along k; chunk i of an axis of length L is [i L / n, (i+1) L / n)),
    and each square gives its highest count (ties to the lowest row, then column) and a second one:
    the highest count among its cells at least min_dk k rows away from the first.  The analysis
    columns are contiguous (f0 falls monotonically with the column).

    Returns {(square, which): record} for which = 0, 1 (squares without cells, or without cells far
    enough for a second candidate, give no record) and the CR statistics as in select_candidates.
    """
    f0c, f0n, band = column_bands(g)
    ana = np.nonzero(band >= 0)[0]
    K = g.n_k
    n_cells = K * ana.size
    sub = hmap[:, ana].astype(np.int64)
    s1, s2 = int(sub.sum()), int((sub * sub).sum())
    if n_cells > 0:
        mu = float(s1) / float(n_cells)
        var = float(s2) / float(n_cells) - mu * mu
        sigma = math.sqrt(var) if var > 0.0 else 0.0
    else:
        mu, sigma = 0.0, 0.0
    out = {}
    if ana.size == 0:
        return out, (s1, s2, n_cells)
    ca, wa = int(ana[0]), int(ana.size)
    assert ana[-1] - ana[0] + 1 == wa                  # contiguous
    for j in range(n_sk):
        r0, r1 = j * K // n_sk, (j + 1) * K // n_sk
        for i in range(n_sx):
            c0, c1 = ca + i * wa // n_sx, ca + (i + 1) * wa // n_sx
            if r1 <= r0 or c1 <= c0:
                continue
            sq = j * n_sx + i
            block = hmap[r0:r1, c0:c1]
            flat = int(np.argmax(block))
            rr, cc = divmod(flat, c1 - c0)
            out[(sq, 0)] = _record(g, hmap, r0 + rr, c0 + cc, mu, sigma, f0c, f0n, square=sq)
            far = np.abs(np.arange(r0, r1) - (r0 + rr)) >= min_dk
            if far.any():
                rows = np.arange(r0, r1)[far]
                blk2 = hmap[rows, c0:c1]
                flat2 = int(np.argmax(blk2))
                r2, c2 = divmod(flat2, c1 - c0)
                out[(sq, 1)] = _record(g, hmap, int(rows[r2]), c0 + c2, mu, sigma, f0c, f0n, square=sq)
    return out, (s1, s2, n_cells)


def coincidences(a: list, b: list, dx0: float, dk: float, radius: float = 3.0):
    """For each candidate of set a: the index of the nearest candidate of set b by the Sec. IV
    distance d = sqrt(((x0_b - x0_a)/dx0)^2 + ((k_b - k_a)/dk)^2) (ties to the lower index) and that
    distance; the index is -1 when the nearest lies farther than `radius` (coincidence within
    `radius` bins, Sec. IV uses 3) or when b is empty."""
    match, dist = [], []
    for ca in a:
        best, bj = math.inf, -1
        for j, cb in enumerate(b):
            dxn = (cb["x0"] - ca["x0"]) / dx0
            dkn = (cb["k"] - ca["k"]) / dk
            d = math.sqrt(dxn * dxn + dkn * dkn)
            if d < best:
                best, bj = d, j
        match.append(bj if best <= radius else -1)
        dist.append(best if bj >= 0 else -1.0)
    return match, dist


# ----------------------------------------------------------------------------------------------
# Sec. III peakmap
# ----------------------------------------------------------------------------------------------
def short_power_spectra(series, fs: float, t_fft: float):
    """Interlaced (50% overlap) boxcar FFTs of length N = fs T_FFT (fp64); returns |X|^2 rounded to
    float32, [n_fft][N/2+1]."""
    x = np.asarray(series, dtype=np.float64)
    N = int(round(fs * t_fft))
    hop = N // 2
    n_fft = (x.size - N) // hop + 1
    frames = np.lib.stride_tricks.as_strided(x, shape=(n_fft, N), strides=(hop * 8, 8))
    X = np.fft.rfft(frames, axis=1)
    return (X.real * X.real + X.imag * X.imag).astype(np.float32)


def equalise(P: np.ndarray, bin_lo: int, bin_hi: int, return_mean: bool = False):
    """Equalised spectra R_j = P_j / S_(j-1) for bins bin_lo-1 .. bin_hi+1 (column c of the result
    is bin bin_lo-1+c), in float32.  S is the clipped AR mean along frequency described at the top
    of this module, updated after each bin, so a bin never whitens itself:
        S <- sum of the WARMUP bins below bin_lo-1, times 2^-7;
        per bin: R = P/S;  u = min(GAIN P, CLIP_GAIN S);  S <- S + 2^-7 (u - S).
    With `return_mean` the estimate each bin was divided by is returned too."""
    P = np.asarray(P, dtype=np.float32)
    j0 = bin_lo - 1 - WARMUP
    if j0 < 1:
        raise ValueError("band too close to DC for the equaliser warm-up")
    S = np.zeros(P.shape[0], dtype=np.float32)
    for j in range(j0, j0 + WARMUP):
        S = S + P[:, j]
    S = S * np.float32(1.0 / WARMUP)
    R = np.empty((P.shape[0], bin_hi - bin_lo + 3), dtype=np.float32)
    used = np.empty_like(R)
    for c, j in enumerate(range(bin_lo - 1, bin_hi + 2)):
        p = P[:, j]
        R[:, c] = p / S
        used[:, c] = S
        u = np.minimum(p * GAIN, S * CLIP_GAIN)
        S = S + AR_WEIGHT * (u - S)
    return (R, used) if return_mean else R


def peaks_from_equalised(R: np.ndarray, bin_lo: int, theta: float = THETA):
    """Sec. III peak selection: bin j is a peak iff R_j > theta and R_j > R_(j-1) and R_j > R_(j+1).
    R's column c is bin bin_lo-1+c.  Returns (fft_idx, bin) sorted by bin, then FFT."""
    mid = R[:, 1:-1]
    sel = (mid > np.float32(theta)) & (mid > R[:, :-2]) & (mid > R[:, 2:])
    b_idx, f_idx = np.nonzero(sel.T)
    return f_idx.astype(np.uint32), (b_idx + bin_lo).astype(np.uint32)


def peaks_from_power(P: np.ndarray, bin_lo: int, bin_hi: int, theta: float = THETA):
    """Equalise power spectra P [n_fft][bins] and select peaks in bins bin_lo..bin_hi."""
    return peaks_from_equalised(equalise(P, bin_lo, bin_hi), bin_lo, theta)


def peakmap(series, fs: float, t_fft: float, bin_lo: int, bin_hi: int, theta: float = THETA):
    """Sec. III: time series -> interlaced FFTs -> equalised spectra -> thresholded local maxima."""
    return peaks_from_power(short_power_spectra(series, fs, t_fft), bin_lo, bin_hi, theta)


# ----------------------------------------------------------------------------------------------
# Sec. V follow-up: heterodyne correction, longer-FFT peakmap of the corrected series, original
# FrequencyHough on it (n = 0 grids above), projection of the corrected peakmap onto frequency
# ----------------------------------------------------------------------------------------------
def spindown_cycles(t, f0: float, k: float, n: float):
    """Residual phase of Sec. V Eq. phcor in cycles: integral from t0 to t of (f(t') - f0) dt' with
    f from Eq. powlaws, i.e. F(t) - f0 t where F is the integral of f.  With a = (n-1) k f0^(n-1):
    F(t) = f0 (n-1) / ((n-2) a) ((1 + a t)^((n-2)/(n-1)) - 1) for n != 2 and (f0 / a) ln(1 + a t)
    for n = 2 (t measured from t0)."""
    t = np.asarray(t, dtype=np.float64)
    a = (n - 1.0) * k * f0 ** (n - 1.0)
    if a == 0.0:
        return np.zeros_like(t)
    L = np.log1p(a * t)
    if n == 2.0:
        F = (f0 / a) * L
    else:
        F = f0 * (n - 1.0) / ((n - 2.0) * a) * np.expm1((n - 2.0) / (n - 1.0) * L)
    return F - f0 * t


def heterodyne(series, fs: float, t_start: float, f0: float, k: float, n: float):
    """Sec. V: h'(t) = h(t) exp(-2 pi j (F(t) - f0 t)) at t = t_start + s / fs, so that the power
    law of (f0, k, n) becomes a constant line at f0 (complex128).  The sign makes the positive-
    frequency part of a real signal monochromatic (the paper writes e^{j phi_sd} with its own
    convention)."""
    h = np.asarray(series, dtype=np.float64)
    t = t_start + np.arange(h.size, dtype=np.float64) / fs
    c = spindown_cycles(t, f0, k, n)
    return h * np.exp(-2j * np.pi * c)


def complex_power_spectra(z, fs: float, t_fft: float):
    """Interlaced (50% overlap) boxcar FFTs of length N = fs T_FFT of a complex series (fp64,
    numpy's complex FFT); |X|^2 rounded to float32, [n_fft][N] (bin j = frequency j / T_FFT for
    j < N/2)."""
    z = np.asarray(z, dtype=np.complex128)
    N = int(round(fs * t_fft))
    hop = N // 2
    n_fft = (z.size - N) // hop + 1
    frames = np.lib.stride_tricks.as_strided(z, shape=(n_fft, N), strides=(hop * 16, 16))
    X = np.fft.fft(frames, axis=1)
    return (X.real * X.real + X.imag * X.imag).astype(np.float32)


def peakmap_complex(z, fs: float, t_fft: float, bin_lo: int, bin_hi: int, theta: float = THETA):
    """Sec. III peakmap of a complex (heterodyned) series: complex FFTs, then the same equaliser and
    peak test as the real series."""
    return peaks_from_power(complex_power_spectra(z, fs, t_fft), bin_lo, bin_hi, theta)


def bin_shift(i, t_first: float, t_hop: float, df: float, fdot: float):
    """Sec. V correction of a peakmap by shifting bins: FFT i (time t_i = t_first + i t_hop) moves
    by floor(fdot t_i / df + 1/2) bins, the rounded drift of the line f0 + fdot t."""
    t = t_first + np.asarray(i, dtype=np.float64) * t_hop
    return np.floor(fdot * t / df + 0.5).astype(np.int64)


def project_peaks(fft_idx, bins, t_first: float, t_hop: float, df: float, fdot: float, bin_lo: int,
                  bin_hi: int):
    """Sec. V projection: every peak (i, j) is moved to bin j - shift_i (bin_shift) and counted per
    bin; returns the counts of bins bin_lo..bin_hi (int64)."""
    j = np.asarray(bins, dtype=np.int64) - bin_shift(fft_idx, t_first, t_hop, df, fdot)
    keep = (j >= bin_lo) & (j <= bin_hi)
    return np.bincount(j[keep] - bin_lo, minlength=bin_hi - bin_lo + 1).astype(np.int64)


def projection_cr(counts, j: int):
    """Sec. V: CR = (y - mu) / sigma of the projected count y at local bin j, mu and sigma the
    population mean and standard deviation of the counts of all other bins (the noise)."""
    c = np.asarray(counts, dtype=np.float64)
    rest = np.delete(c, j)
    mu = float(rest.mean())
    sigma = float(rest.std())
    return (float(c[j]) - mu) / sigma if sigma > 0.0 else 0.0


# ----------------------------------------------------------------------------------------------
# Sec. VI.D: longer FFTs for later times (T_FFT splicing)
# ----------------------------------------------------------------------------------------------
def max_spindown_at(t, n: float, f_hi: float, fdot_hi: float):
    """Largest |fdot(t)| over the power laws of braking index n (Eq. powlaws) with f0 <= f_hi and
    |fdot0| <= fdot_hi.  A member's |fdot(t)| = fdot0 (1 + u)^(-n/(n-1)) with u = (n-1) fdot0 t / f0
    grows with f0 and, over fdot0, peaks at u = n-1, i.e. fdot0 = f0 / t; so the bound is the
    fastest member's fdot_hi (1 + (n-1) fdot_hi t / f_hi)^(-n/(n-1)) while f_hi / t > fdot_hi, and
    f_hi n^(-n/(n-1)) / t after that."""
    t = np.asarray(t, dtype=np.float64)
    early = fdot_hi * (1.0 + (n - 1.0) * fdot_hi * t / f_hi) ** (-n / (n - 1.0))
    with np.errstate(divide="ignore"):
        late = f_hi * n ** (-n / (n - 1.0)) / t
    return np.where(t * fdot_hi < f_hi, early, late)


def time_of_spindown(fdot: float, n: float, f_hi: float, fdot_hi: float) -> float:
    """First time at which max_spindown_at falls to fdot (0 when it starts at or below it)."""
    if fdot_hi <= fdot:
        return 0.0
    t1 = ((fdot_hi / fdot) ** ((n - 1.0) / n) - 1.0) * f_hi / ((n - 1.0) * fdot_hi)
    if t1 * fdot_hi < f_hi:
        return t1
    return f_hi * n ** (-n / (n - 1.0)) / fdot


def tfft_portions(n: float, f_hi: float, fdot_hi: float, t_fft0: float, t_obs: float,
                  max_levels: int):
    """Sec. VI.D: the data from t0 to t_obs split into portions analysed with T_FFT = 2^L t_fft0,
    L = 0 .. max_levels-1.  Eq. dot_tfft: with T_FFT a signal stays within one bin while
    |fdot| <= 1/T_FFT^2; once the family's largest spin-down (max_spindown_at) has fallen by 4,
    T_FFT doubles.  Portion L spans [t_L, t_(L+1)) with t_L = time_of_spindown(1/T_L^2) (the last
    level runs to t_obs); levels whose span is empty or shorter than one FFT are left out, and the
    data before t_0 (spin-down above 1/t_fft0^2) is not analysed.  Returns a list of
    (level, t_begin, t_end, t_fft)."""
    out = []
    for L in range(max_levels):
        T = t_fft0 * 2.0 ** L
        a = min(time_of_spindown(1.0 / T ** 2, n, f_hi, fdot_hi), t_obs)
        if L + 1 < max_levels:
            b = min(time_of_spindown(1.0 / (2.0 * T) ** 2, n, f_hi, fdot_hi), t_obs)
        else:
            b = t_obs
        if b - a >= T:
            out.append((L, a, b, T))
    return out
