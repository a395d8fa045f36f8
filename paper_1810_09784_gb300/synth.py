"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: white Gaussian strain noise and power-law spin-down injections
(Sec. II, Eq. powlaws for f(t); the phase is the integral of Sec. V, Eq. phcor).  It holds no step of
the FrequencyHough method itself (no peakmap, no x = f^(1-n) transform, no Hough accumulation, no
candidate selection), so both the CUDA path and the CPU oracle can be fed from it.

Every array is a deterministic function of its seed (numpy PCG64).
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import math
import os

import numpy as np


@dataclasses.dataclass(frozen=True)
class Injection:
    """One power-law signal h(t) = amp * sin(phi(t) + phase0), f(t) from Sec. II Eq. powlaws."""

    f0: float       # frequency at t0 = start of the data [Hz]
    k: float        # spin-down constant of fdot = -k f^n (Sec. II Eq. diff_powlaws), k > 0
    n: float        # braking index
    amp: float      # strain amplitude in units of the noise sigma
    phase0: float = 0.0

    @property
    def fdot0(self) -> float:
        """Initial spin-down fdot0 = -k f0^n (Sec. II)."""
        return -self.k * self.f0 ** self.n


def amplitude_for_snr(snr: float, sigma: float, n_fft_samples: int) -> float:
    """Amplitude giving a mean spectral SNR `snr` at a bin centre with a boxcar window.

    A sinusoid of amplitude A gives |X|^2 = (A N / 2)^2 at its bin; white noise of variance
    sigma^2 gives E|X|^2 = N sigma^2.  Their ratio A^2 N / (4 sigma^2) = snr.
    """
    return 2.0 * sigma * math.sqrt(snr / n_fft_samples)


def powerlaw_phase(t: np.ndarray, f0: float, k: float, n: float) -> np.ndarray:
    """phi(t) = 2 pi * integral_0^t f(t') dt' for f(t) = f0 (1 + a t)^(-1/(n-1)), a = (n-1) k f0^(n-1).

    Closed form of the integral in Sec. V Eq. phcor: for n != 2 it is
    f0 (n-1) / (a (n-2)) [(1 + a t)^((n-2)/(n-1)) - 1]; for n = 2 it is (f0 / a) ln(1 + a t).
    """
    a = (n - 1.0) * k * f0 ** (n - 1.0)
    if a == 0.0:
        return 2.0 * np.pi * f0 * t
    if abs(n - 2.0) < 1e-12:
        return 2.0 * np.pi * (f0 / a) * np.log1p(a * t)
    e = (n - 2.0) / (n - 1.0)
    return 2.0 * np.pi * f0 * (n - 1.0) / (a * (n - 2.0)) * np.expm1(e * np.log1p(a * t))


def strain_series(n_samples: int, fs: float, seed: int, injections=(), sigma: float = 1.0,
                  chunk: int = 1 << 22) -> np.ndarray:
    """White Gaussian noise N(0, sigma^2) at `fs` plus injections, returned as float32.

    Noise comes from numpy PCG64(seed); injections are added in float64 before rounding.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = [rng.standard_normal(min(n_samples, s0 + chunk) - s0) * sigma
             for s0 in range(0, n_samples, chunk)]
    out = np.empty(n_samples, dtype=np.float32)

    def fill(ci):
        s0 = ci * chunk
        x = noise[ci]
        if injections:
            t = np.arange(s0, s0 + x.size, dtype=np.float64) / fs
            for inj in injections:
                x += inj.amp * np.sin(powerlaw_phase(t, inj.f0, inj.k, inj.n) + inj.phase0)
        out[s0:s0 + x.size] = x

    # chunks are independent (numpy ufuncs release the GIL): same result for any thread count
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(fill, range(len(noise))))
    return out


def strain_series_device(out, fs: float, seed: int, injections=(), sigma: float = 1.0):
    """The recipe of strain_series drawn on a CUDA device into the float32 tensor `out`: white
    Gaussian noise N(0, sigma^2) from torch's counter-based Philox generator seeded with `seed`,
    plus the injections' h(t) = amp sin(phi(t) + phase0) with phi the closed form of
    powerlaw_phase, summed in float64 before the one rounding to float32.  The noise draws differ
    from strain_series' (another generator); their distribution is the same."""
    import torch
    gen = torch.Generator(device=out.device)
    gen.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    if not injections:
        torch.randn(out.shape, generator=gen, out=out)
        if sigma != 1.0:
            out.mul_(sigma)
        return out
    x = torch.randn(out.shape, generator=gen, dtype=torch.float64, device=out.device)
    if sigma != 1.0:
        x.mul_(sigma)
    t = torch.arange(out.numel(), dtype=torch.float64, device=out.device).div_(fs)
    for inj in injections:
        a = (inj.n - 1.0) * inj.k * inj.f0 ** (inj.n - 1.0)
        if a == 0.0:
            ph = t * (2.0 * math.pi * inj.f0)
        elif abs(inj.n - 2.0) < 1e-12:
            ph = torch.log1p(t * a).mul_(2.0 * math.pi * inj.f0 / a)
        else:
            e = (inj.n - 2.0) / (inj.n - 1.0)
            ph = torch.expm1(torch.log1p(t * a).mul_(e)).mul_(
                2.0 * math.pi * inj.f0 * (inj.n - 1.0) / (a * (inj.n - 2.0)))
        x.add_(torch.sin(ph.add_(inj.phase0)).mul_(inj.amp))
    out.copy_(x)
    return out


def statistical_peaklist(n_fft: int, bin_lo: int, bin_hi: int, p_noise: float, seed: int,
                         tracks=(), p_track: float = 0.6):
    """Peak list (fft_idx, bin) sorted by (bin, fft) from a statistical model of a peakmap.

    Every (FFT, bin) cell is a noise peak independently with probability `p_noise` (drawn as a
    Bernoulli process along the FFTs of each bin through geometric gaps, so the cost follows the
    number of peaks, not of cells).  Each track is an array of bins, one per FFT (negative for none),
    whose cell is made a peak with probability `p_track`.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = bin_hi - bin_lo + 1
    expect = n_fft * p_noise
    g = int(expect + 6.0 * math.sqrt(expect + 1.0) + 16)
    fft_parts, bin_parts = [], []
    chunk = max(1, (1 << 24) // max(g, 1))
    for b0 in range(0, nb, chunk):
        b1 = min(nb, b0 + chunk)
        while True:
            pos = np.cumsum(rng.geometric(p_noise, size=(b1 - b0, g)), axis=1) - 1
            if np.all(pos[:, -1] >= n_fft):     # every bin's process ran past the last FFT
                break
            g *= 2
        rows, cols = np.nonzero(pos < n_fft)
        fft_parts.append(pos[rows, cols].astype(np.int64))
        bin_parts.append((rows + b0 + bin_lo).astype(np.int64))
    fi = np.concatenate(fft_parts) if fft_parts else np.zeros(0, np.int64)
    bj = np.concatenate(bin_parts) if bin_parts else np.zeros(0, np.int64)
    key = bj * n_fft + fi                        # sorted by (bin, fft), one peak per cell
    extra = []
    for tr in tracks:
        tr = np.asarray(tr, dtype=np.int64)
        i = np.nonzero((tr >= bin_lo) & (tr <= bin_hi) & (rng.random(tr.size) < p_track))[0]
        extra.append(tr[i] * n_fft + i)
    if extra:
        add = np.unique(np.concatenate(extra))
        pos = np.searchsorted(key, add)
        new = (pos >= key.size) | (key[np.minimum(pos, key.size - 1)] != add) if key.size else np.ones(add.size, bool)
        key = np.insert(key, pos[new], add[new])
    return (key % n_fft).astype(np.uint32), (key // n_fft).astype(np.uint32)


def powerlaw_track(f0: float, k: float, n: float, df: float, n_fft: int, t_first: float,
                   t_hop: float) -> np.ndarray:
    """Bin holding f(t_i) = f0 (1 + (n-1) k f0^(n-1) t_i)^(-1/(n-1)) at each FFT time t_i."""
    t = t_first + t_hop * np.arange(n_fft)
    f = f0 / (1.0 + (n - 1.0) * k * f0 ** (n - 1.0) * t) ** (1.0 / (n - 1.0))
    return np.floor(f / df + 0.5).astype(np.int64)


def random_peaklist(n_fft: int, bin_lo: int, bin_hi: int, density: float, seed: int):
    """Random (fft_idx, bin) pairs sorted by (bin, fft_idx), at most one per cell.

    A structural stand-in for a peakmap: each (FFT, bin) cell is occupied with probability
    `density`, and two occupied cells of one FFT are never adjacent in frequency (a peakmap's
    peaks are local maxima along frequency).  Used for Hough tests independent of the peakmap.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = bin_hi - bin_lo + 1
    occ = rng.random((n_fft, nb)) < density
    # drop the right neighbour of every occupied cell, scanning left to right
    for j in range(1, nb):
        occ[:, j] &= ~occ[:, j - 1]
    b_idx, f_idx = np.nonzero(occ.T)    # row-major over [bin][fft]: sorted by bin, then fft
    return f_idx.astype(np.uint32), (b_idx + bin_lo).astype(np.uint32)


# ---- counter-based statistical peakmaps ------------------------------------------------------------
#
# The same model as statistical_peaklist, with every draw a pure function of (seed, sample, stream,
# FFT i, bin j) so that a GPU kernel can draw any cell on its own: the splitmix64 finaliser of
# Steele, Lea and Flood ("Fast splittable pseudorandom number generators", OOPSLA 2014) applied to
#   key = mix(seed ^ sample * 0xD1B54A32D192ED03 ^ stream << 56),  u = mix(key ^ (i << 32 | j)) >> 40
# (all arithmetic mod 2^64).  Cell (i, j) of a sample is a peak when u(stream 0) < p_noise24, or when
# j is the track's bin in FFT i and u(stream 1) < p_track24 (probabilities times 2^24).

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)
_SAMPLE_MUL = np.uint64(0xD1B54A32D192ED03)


def mix64(z) -> np.ndarray:
    """The splitmix64 finaliser, elementwise on uint64 (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def sample_key(seed: int, sample, stream: int) -> np.ndarray:
    s = np.asarray(sample, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(seed) ^ (s * _SAMPLE_MUL) ^ (np.uint64(stream) << np.uint64(56)))


def cell_u24(seed: int, sample, stream: int, i, j) -> np.ndarray:
    """24-bit uniform of cell (i, j) (broadcasting over sample, i, j)."""
    key = sample_key(seed, sample, stream)
    lin = (np.asarray(i, dtype=np.uint64) << np.uint64(32)) | np.asarray(j, dtype=np.uint64)
    return (mix64(key ^ lin) >> np.uint64(40)).astype(np.uint32)


def hashed_peaklist(seed: int, sample: int, n_fft: int, bin_lo: int, bin_hi: int, p_noise24: int,
                    p_track24: int = 0, track=None):
    """Peak list (fft_idx, bin) of one sample, sorted by (bin, fft); track: bin per FFT or -1."""
    j = np.arange(bin_lo, bin_hi + 1, dtype=np.uint64)[:, None]
    i = np.arange(n_fft, dtype=np.uint64)[None, :]
    peak = cell_u24(seed, sample, 0, i, j) < np.uint32(p_noise24)
    if track is not None:
        tr = np.asarray(track, dtype=np.int64)
        ii = np.nonzero((tr >= bin_lo) & (tr <= bin_hi))[0]
        hit = cell_u24(seed, sample, 1, ii.astype(np.uint64), tr[ii].astype(np.uint64)) < np.uint32(p_track24)
        peak[tr[ii[hit]] - bin_lo, ii[hit]] = True
    jj, ff = np.nonzero(peak)
    return ff.astype(np.uint32), (jj + bin_lo).astype(np.uint32)


def hashed_uniform(seed: int, sample, stream: int, slot: int = 0) -> np.ndarray:
    """Uniform double in [0, 1) per sample from 53 bits of mix(key ^ slot) (sample parameters)."""
    key = sample_key(seed, sample, stream)
    return (mix64(key ^ np.uint64(slot)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
