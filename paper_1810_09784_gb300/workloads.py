"""The synthetic workloads, shaped like the paper's searches (sizes, seeds, bands, k grids).

Numbers only: every quantity derived from them (x0 step, k step, map sizes, tables) is computed by
the library's planner.  t0 is the start of the data and FFT i is stamped at its centre.

  plain_small     fs 1024 Hz, 1800 s, T_FFT 2 s, 50% overlap (1799 FFTs), band 100-400 Hz, one
                  n = 5 injection at f0 = 350 Hz with spectral SNR 4; Hough at n = 5 with 500 k rows.
  plain_paper     fs 4096 Hz, 10080 s (2.8 h), T_FFT 4 s (5039 FFTs), 50-2000 Hz, 20 injections;
                  Hough at n = 5, 2000 k rows, in 100 Hz analysis bands whose peakmap band extends
                  50 Hz upwards (Sec. IV: the peakmap band is wider than the analysed band), top
                  candidate per 1 Hz.
  batched_n       the plain_small peakmap at 51 braking indices n = 2.0 .. 7.0, fewer k rows at
                  higher n (4000 -> 1000), one map per n.
  paper_grids     the plain_small peakmap on the paper's own grids: braking indices of
                  Eq. dn_powlaws over n = 2.5 .. 7 and, for each, the Eq. dkeqn k grid (|fdot|
                  1e-4 .. 1e-2 Hz/s) as uniform segments, one map per (n, segment).
  followup        Sec. V follow-up of each plain_paper injection (or of plain_small's): heterodyne
                  by the candidate's (f0, k, n), FFTs twice as long, original FrequencyHough in
                  f0 +- 5 Hz over 32 fdot rows, projection.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import synth


@dataclasses.dataclass
class SeriesSpec:
    fs: float
    t_obs: float
    t_fft: float
    seed: int
    injections: tuple = ()

    @property
    def n_samples(self) -> int:
        return int(round(self.fs * self.t_obs))

    @property
    def n_per_fft(self) -> int:
        return int(round(self.fs * self.t_fft))

    @property
    def n_fft(self) -> int:
        N = self.n_per_fft
        return (self.n_samples - N) // (N // 2) + 1

    @property
    def df(self) -> float:
        return 1.0 / self.t_fft

    @property
    def t_first(self) -> float:
        return self.t_fft / 2.0

    @property
    def t_hop(self) -> float:
        return self.t_fft / 2.0

    def series(self) -> np.ndarray:
        return synth.strain_series(self.n_samples, self.fs, self.seed, self.injections)


def grid_fields(spec: SeriesSpec, n: float, bin_lo: int, bin_hi: int, n_k: int, ana_lo: float,
                ana_hi: float, band_hz: float = 1.0, list_idx: int = 0) -> dict:
    """Request fields of one Hough map over the given peakmap band (k_min = 0, default steps)."""
    return dict(n=n, df=spec.df, bin_lo=bin_lo, bin_hi=bin_hi, n_fft=spec.n_fft,
                t_first=spec.t_first, t_hop=spec.t_hop, t_obs=spec.t_obs, n_k=n_k,
                k_min=0.0, dk=0.0, f_max=0.0, ana_lo=ana_lo, ana_hi=ana_hi, band_hz=band_hz,
                list=list_idx)


# ---- plain_small ------------------------------------------------------------------------------

def plain_small(seed: int = 1):
    fs, t_obs, t_fft, n = 1024.0, 1800.0, 2.0, 5.0
    N = int(fs * t_fft)
    # k on row 300 of the default grid: dk = dx0 / ((n-1) T_obs), dx0 = (n-1) df / f_max^n
    f_max = 799 * 0.5
    dk = (n - 1.0) * 0.5 / f_max ** n / ((n - 1.0) * t_obs)
    inj = synth.Injection(f0=350.0, k=300 * dk, n=n, amp=synth.amplitude_for_snr(4.0, 1.0, N))
    spec = SeriesSpec(fs, t_obs, t_fft, seed, (inj,))
    pm = dict(bin_lo=200, bin_hi=799)
    grids = [grid_fields(spec, n, 200, 799, 500, 100.0, 400.0)]
    return spec, pm, grids


# ---- plain_paper ------------------------------------------------------------------------------

def paper_injections(seed: int, n_inj: int = 20, snr: float = 4.0, fs: float = 4096.0,
                     t_fft: float = 4.0):
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    out = []
    N = int(fs * t_fft)
    for _ in range(n_inj):
        f0 = rng.uniform(500.0, 1800.0)
        n = rng.uniform(2.5, 7.0)
        fdot = min(10 ** rng.uniform(-4.0, -1.0), 1.0 / t_fft ** 2)   # Sec. VI.D: fdot <= 1/T_FFT^2
        k = fdot / f0 ** n
        out.append(synth.Injection(f0=f0, k=k, n=n, amp=synth.amplitude_for_snr(snr, 1.0, N),
                                   phase0=rng.uniform(0, 2 * math.pi)))
    return tuple(out)


def plain_paper(seed: int = 2, n_k: int = 2000, n: float = 5.0):
    fs, t_obs, t_fft = 4096.0, 10080.0, 4.0
    spec = SeriesSpec(fs, t_obs, t_fft, seed, paper_injections(seed))
    df = spec.df
    f_lo, f_hi, width, ext = 50.0, 2000.0, 100.0, 50.0
    pm = dict(bin_lo=int(round(f_lo / df)), bin_hi=int(round(f_hi / df)) - 1)
    grids = []
    a = f_lo
    while a < f_hi - 1e-9:
        b = min(a + width, f_hi)
        top = min(b + ext, f_hi)
        grids.append(grid_fields(spec, n, int(round(a / df)), int(round(top / df)) - 1, n_k, a, b))
        a = b
    return spec, pm, grids


# ---- batched_n --------------------------------------------------------------------------------

def batched_n(seed: int = 1):
    spec, pm, _ = plain_small(seed)
    grids = []
    for i in range(51):
        n = round(2.0 + 0.1 * i, 10)
        n_k = int(round(4000 - 3000 * (n - 2.0) / 5.0))
        grids.append(grid_fields(spec, n, pm["bin_lo"], pm["bin_hi"], n_k, 100.0, 400.0))
    return spec, pm, grids


# ---- paper_grids -----------------------------------------------------------------------------

def paper_grids(seed: int = 1, fdot=(1e-4, 1e-2), n_range=(2.5, 7.0), growth: float = 2.0,
                max_rows: int = 512):
    from . import gfh                 # the library's grid planners (Sec. VI)
    spec, pm, base = plain_small(seed)
    df, f_min, f_max = spec.df, 100.0, pm["bin_hi"] * spec.df
    grids = []
    for n in gfh.n_grid(n_range[0], n_range[1], df, f_min, f_max, fdot[1], spec.t_obs):
        for sg in gfh.k_segments(float(n), df, f_min, f_max, fdot[0], fdot[1], growth, max_rows):
            grids.append(dict(base[0], n=float(n), k_min=float(sg["k_min"]), dk=float(sg["dk"]),
                              n_k=int(sg["n_k"])))
    return spec, pm, grids


# ---- followup ----------------------------------------------------------------------------------

def followup_fields(inj, t_obs: float, t_fft: float, half_band: float = 5.0, n_k: int = 32,
                    t_first=None) -> tuple:
    """Sec. V follow-up of an injection: the series corrected by (f0, k, n) is searched with FFTs of
    length t_fft in f0 +- half_band by the original FrequencyHough (n = 0) over n_k fdot rows
    centred on 0 (the residual spin-down of a correction off by about one bin).  Returns the
    peakmap band (bin_lo, bin_hi) and the n = 0 grid request."""
    df = 1.0 / t_fft
    N_hop = t_fft / 2.0
    n_fft = int((t_obs - t_fft) // N_hop) + 1
    bin_lo = int(math.floor((inj.f0 - half_band) / df))
    bin_hi = int(math.ceil((inj.f0 + half_band) / df))
    dk = df / t_obs
    fields = dict(n=0.0, df=df, bin_lo=bin_lo, bin_hi=bin_hi, n_fft=n_fft,
                  t_first=t_fft / 2.0 if t_first is None else t_first, t_hop=N_hop, t_obs=t_obs,
                  n_k=n_k, k_min=-(n_k // 2) * dk, dk=dk, f_max=0.0,
                  ana_lo=inj.f0 - half_band + 1.0, ana_hi=inj.f0 + half_band - 1.0,
                  band_hz=2.0 * half_band, list=0)
    return (bin_lo, bin_hi), fields


# ---- uneven ------------------------------------------------------------------------------------

P0_THETA_2_5 = 0.0755      # noise peak probability of a strict local maximum above 2.5 (exp(1) power)


def uneven_specs(seed: int = 4, n_maps: int = 256, hours=(1.0, 24.0), width_hz=(20.0, 1950.0)):
    """The peakmaps of `uneven` (no peaks yet): per peakmap its duration, T_FFT, band, injections
    (f0, k, n) and the braking index it is searched at, each drawn from its own seeded stream."""
    specs = []
    for m in range(n_maps):
        rng = np.random.Generator(np.random.PCG64(seed * 100003 + m))
        t_obs = 3600.0 * math.exp(rng.uniform(math.log(hours[0]), math.log(hours[1])))
        t_fft = float(rng.choice([1.0, 2.0, 4.0, 8.0]))
        df = 1.0 / t_fft
        n_fft = int((t_obs - t_fft) // (t_fft / 2.0)) + 1
        w = math.exp(rng.uniform(math.log(width_hz[0]), math.log(width_hz[1])))
        f_lo = rng.uniform(50.0, 2000.0 - w)
        f_hi = f_lo + w
        bin_lo, bin_hi = int(math.ceil(f_lo / df)), int(math.floor(f_hi / df)) - 1
        injs = []
        for _ in range(int(rng.integers(0, 4))):
            n = rng.uniform(2.0, 7.0)
            f0 = rng.uniform(f_lo + 0.2 * w, f_hi)
            fdot = math.exp(rng.uniform(math.log(1e-4), math.log(1.0 / t_fft ** 2)))
            injs.append((f0, fdot / f0 ** n, n))
        n_hough = injs[0][2] if injs else rng.uniform(2.0, 7.0)
        specs.append(dict(t_obs=t_obs, t_fft=t_fft, df=df, n_fft=n_fft, bin_lo=bin_lo, bin_hi=bin_hi,
                          f_lo=bin_lo * df, f_hi=(bin_hi + 1) * df, injs=injs, n=n_hough, seed=seed * 100003 + m))
    return specs


def uneven_grids(specs, n_k: int = 1000):
    """Grid requests of the `uneven` peakmaps: 100 Hz analysis bands, each with its peakmap band
    50 Hz wider (capped at the peakmap's top); grids[m]['list'] = its peakmap."""
    grids = []
    for l, s in enumerate(specs):
        a = s["f_lo"]
        while a < s["f_hi"] - 1e-9:
            b = min(a + 100.0, s["f_hi"])
            top = min(b + 50.0, s["f_hi"])
            lo_bin = int(round(a / s["df"]))
            hi_bin = int(round(top / s["df"])) - 1
            if hi_bin >= lo_bin:
                grids.append(dict(n=s["n"], df=s["df"], bin_lo=lo_bin, bin_hi=hi_bin, n_fft=s["n_fft"],
                                  t_first=s["t_fft"] / 2, t_hop=s["t_fft"] / 2, t_obs=s["t_obs"],
                                  n_k=n_k, k_min=0.0, dk=0.0, f_max=0.0, ana_lo=a, ana_hi=b,
                                  band_hz=1.0, list=l))
            a = b
    return grids


def uneven(seed: int = 4, n_maps: int = 256, hours=(1.0, 24.0), width_hz=(20.0, 1950.0),
           n_k: int = 1000, p_track: float = 0.6):
    """Independent peakmaps of uneven size (statistical peakmap model, no time series): duration
    log-uniform in `hours`, T_FFT in {1, 2, 4, 8} s, a band of log-uniform width inside 50-2000 Hz,
    0-3 power-law injections (n in [2, 7], |fdot0| log-uniform up to 1/T_FFT^2).  Each peakmap is
    searched in 100 Hz analysis bands (peakmap band 50 Hz wider, capped at the band top) at the
    braking index of its first injection (else uniform in [2, 7]) with `n_k` k rows.

    Returns (lists, grids, truth): lists[l] = (fft_idx, bin); grids[m]['list'] = its peakmap.
    """
    import concurrent.futures
    import os

    specs = uneven_specs(seed, n_maps, hours, width_hz)

    def make_list(s):
        tracks = [synth.powerlaw_track(f0, k, n, s["df"], s["n_fft"], s["t_fft"] / 2, s["t_fft"] / 2)
                  for f0, k, n in s["injs"]]
        return synth.statistical_peaklist(s["n_fft"], s["bin_lo"], s["bin_hi"], P0_THETA_2_5,
                                          s["seed"], tracks, p_track)

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        lists = list(ex.map(make_list, specs))
    return lists, uneven_grids(specs, n_k), specs
