"""Host logic of the Sec. VI.D portion search (no GPU): every portion's samples start on a multiple
of its FFT hop and hold exactly its FFTs, its FFTs are stamped at their centres from the common t0,
consecutive portions do not share samples, each analysis band becomes one grid request whose
extension reaches `ext` Hz above the band, the requests are valid grids, and the update count
equals a direct count over the peaks."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import splice


def portions(n, f_hi, fdot_hi, t_fft0, t_obs, levels):
    return [dict(level=L, t_begin=a, t_end=b, t_fft=T)
            for (L, a, b, T) in O.tfft_portions(n, f_hi, fdot_hi, t_fft0, t_obs, levels)]


CASES = [(1024.0, 1800.0, 5.0, 400.0, 0.2, 2.0, 2),        # the GPU test's two portions
         (4096.0, 10080.0, 5.0, 2000.0, 0.25, 2.0, 3),     # the splice bench workload
         (512.0, 36000.0, 2.5, 200.0, 1.0, 1.0, 5)]


@pytest.mark.parametrize("fs,t_obs,n,f_hi,fdot_hi,t_fft0,levels", CASES)
def test_portion_samples_and_timestamps(fs, t_obs, n, f_hi, fdot_hi, t_fft0, levels):
    n_samples = int(fs * t_obs)
    P = portions(n, f_hi, fdot_hi, t_fft0, t_obs, levels)
    bands = [(100.0, 150.0), (150.0, 200.0)]
    plan = splice.portion_plan(P, fs, n_samples, n, bands, 7, band_hz=1.0, ext=2.0)
    assert plan
    prev_end = 0
    for q in plan:
        src = next(p for p in P if p["level"] == q.level)
        N = int(round(fs * q.t_fft))
        hop = N // 2
        assert q.t_fft == src["t_fft"]
        assert q.s_begin % hop == 0 and q.s_begin >= src["t_begin"] * fs - 1e-9
        assert q.s_begin >= prev_end                         # no sample in two portions
        assert q.s_end <= min(n_samples, src["t_end"] * fs + 1e-9)
        prev_end = q.s_end
        assert len(q.fields) == len(bands)
        for f, (lo, hi) in zip(q.fields, bands):
            n_fft = f["n_fft"]
            assert q.s_end - q.s_begin == (n_fft - 1) * hop + N        # exactly its FFTs
            # one more FFT would run past the portion's end or the data
            assert q.s_begin + n_fft * hop + N > min(n_samples, math.floor(src["t_end"] * fs))
            assert f["t_first"] == pytest.approx(q.s_begin / fs + q.t_fft / 2, abs=1e-12)
            assert f["t_hop"] == q.t_fft / 2
            assert f["t_obs"] == pytest.approx(f["t_first"] + (n_fft - 1) * q.t_fft / 2, abs=1e-9)
            df = 1.0 / q.t_fft
            assert f["df"] == df and f["n"] == n and f["n_k"] == 7
            assert f["bin_lo"] == round(lo / df) and f["bin_hi"] == round((hi + 2.0) / df) - 1
            assert (f["ana_lo"], f["ana_hi"]) == (lo, hi)


def test_portion_shorter_than_one_fft_is_left_out():
    fs, t_obs = 256.0, 100.0
    P = [dict(level=0, t_begin=0.0, t_end=50.0, t_fft=2.0),
         dict(level=1, t_begin=50.0, t_end=53.0, t_fft=4.0),    # 3 s of data for a 4 s FFT
         dict(level=2, t_begin=53.0, t_end=100.0, t_fft=8.0)]
    plan = splice.portion_plan(P, fs, int(fs * t_obs), 5.0, [(20.0, 30.0)], 3)
    assert [q.level for q in plan] == [0, 2]
    # the 8 s portion starts on its own hop after 53 s: 56 s
    assert plan[1].s_begin == 56 * 256


def test_requests_are_valid_grids():
    fs, t_obs = 1024.0, 1800.0
    P = portions(5.0, 400.0, 0.2, 2.0, t_obs, 2)
    for q in splice.portion_plan(P, fs, int(fs * t_obs), 5.0, [(250.0, 400.0)], 11, band_hz=10.0):
        keep = {f.name for f in dataclasses.fields(O.Grid)}
        g = O.make_grid(O.Grid(**{k: v for k, v in q.fields[0].items() if k in keep}))
        assert g.n_k == 11 and g.n_x0 > 0 and O.n_bands(g) == 15


def test_update_count_is_a_direct_count():
    class G:
        def __init__(self, lo, hi, n_k):
            self.bin_lo, self.bin_hi, self.n_k = lo, hi, n_k
    rng = np.random.default_rng(3)
    bins = rng.integers(0, 400, size=5000)
    grids = [G(10, 99, 7), G(100, 250, 3), G(240, 399, 11)]      # overlapping extensions
    want = sum(g.n_k for b in bins for g in grids if g.bin_lo <= b <= g.bin_hi)
    assert splice.update_count(grids, bins) == want
    assert splice.update_count(grids, bins[:0]) == 0
