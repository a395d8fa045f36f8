"""Longer FFTs for later times (Sec. VI.D): one search per time portion of the data, all on the
common t0, and coincidences between the candidates of consecutive portions.

The portions come from the library's planner (`gfh.tfft_portions`: Eq. dot_tfft and the factor-4
rule).  A portion's samples start on a multiple of its FFT hop, its FFTs are stamped at their
centres from t0 (grid t_first = start + T_FFT/2), and its k step moves the last FFT's line one x0
column per k row.  Since every portion measures t from the same t0, one power law has the same
(x0, k) in all of them, and consecutive portions' candidates are matched with `gfh_coincide` on the
coarser of the two grids.  Orchestration only: every step runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import gfh


@dataclasses.dataclass
class Portion:
    level: int
    t_fft: float
    s_begin: int            # first sample of the portion's data
    s_end: int              # one past its last sample
    fields: list            # grid requests of the portion's maps (one per sub-band)


def portion_plan(portions, fs: float, n_samples: int, n: float, bands, n_k: int,
                 band_hz: float = 1.0, ext: float = 0.0):
    """Grid requests per portion: `bands` is a list of analysis bands (lo, hi) in Hz, each searched
    with its peakmap band widened by `ext` Hz upwards (Sec. IV extension), n_k k rows from k = 0."""
    out = []
    for p in portions:
        T = float(p["t_fft"])
        N = int(round(fs * T))
        hop = N // 2
        s0 = int(math.ceil(float(p["t_begin"]) * fs / hop)) * hop
        s1 = min(n_samples, int(math.floor(float(p["t_end"]) * fs)))
        if s1 - s0 < N:
            continue
        n_fft = (s1 - s0 - N) // hop + 1
        df = 1.0 / T
        t_first = s0 / fs + T / 2.0
        t_last = t_first + (n_fft - 1) * (T / 2.0)
        fields = []
        for (lo, hi) in bands:
            top = hi + ext
            bin_lo, bin_hi = int(round(lo / df)), int(round(top / df)) - 1
            fields.append(dict(n=n, df=df, bin_lo=bin_lo, bin_hi=bin_hi, n_fft=n_fft,
                               t_first=t_first, t_hop=T / 2.0, t_obs=t_last, n_k=n_k, k_min=0.0,
                               dk=0.0, f_max=0.0, ana_lo=lo, ana_hi=hi, band_hz=band_hz,
                               list=0))
        out.append(Portion(int(p["level"]), T, s0, s0 + (n_fft - 1) * hop + N, fields))
    return out


def coincide(ctx, cands_a, ga, cands_b, gb, radius: float = 3.0):
    """gfh_coincide of two portions' candidate records (device uint8 tensors of whole records) on
    the coarser grid: returns the (match, dist) device tensors for the records of `cands_a`, written
    on the context's stream (synchronise with it before reading them on another stream)."""
    import torch
    na = cands_a.numel() // gfh.CANDIDATE_BYTES
    nb = cands_b.numel() // gfh.CANDIDATE_BYTES
    match = torch.empty(na, dtype=torch.int32, device=cands_a.device)
    dist = torch.empty(na, dtype=torch.float64, device=cands_a.device)
    ctx.coincide(cands_a, na, cands_b, nb, max(ga.dx0, gb.dx0), max(ga.dk, gb.dk), radius, match,
                 dist)
    return match, dist


def update_count(grids, bins: np.ndarray) -> int:
    """Updates of one portion's maps: peaks inside each map's band x its k rows."""
    return sum(int(((bins >= g.bin_lo) & (bins <= g.bin_hi)).sum()) * g.n_k for g in grids)
