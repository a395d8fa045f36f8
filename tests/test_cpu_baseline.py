"""The all-cores CPU baseline runs the unmodified oracle split over processes: frames of the
peakmap (each frame is equalised and thresholded on its own) and k rows of the Hough map (each row
on its own).  Its results must be bit-identical to one oracle call on one core."""
import numpy as np

import bench
from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth


def test_split_oracle_equals_the_single_call():
    fs, t_obs, t_fft = 256.0, 300.0, 2.0
    inj = synth.Injection(f0=110.0, k=2e-11, n=5.0, amp=synth.amplitude_for_snr(6.0, 1.0, 512))
    x = synth.strain_series(int(fs * t_obs), fs, 3, (inj,))
    lo, hi = 150, 250
    fields = dict(n=5.0, df=1 / t_fft, bin_lo=lo, bin_hi=hi, n_fft=(x.size - 512) // 256 + 1,
                  t_first=1.0, t_hop=1.0, t_obs=t_obs, n_k=40, k_min=0.0, dk=0.0, f_max=0.0,
                  ana_lo=76.0, ana_hi=120.0, band_hz=1.0)
    with bench.OraclePool(cores=3) as pool:
        fi, bj = pool.peakmap(x, fs, t_fft, lo, hi)
        rf, rb = O.peakmap(x, fs, t_fft, lo, hi)
        assert fi.size > 1000
        assert np.array_equal(fi, rf) and np.array_equal(bj, rb)
        res = pool.rows(fi, bj, [(fields, [0, 3, 7]), (fields, [39])])
    og = O.make_grid(O.Grid(**fields))
    full = O.hough_map(og, rf, rb)
    got = [r for _, rows in res for r in rows]
    for r, row in zip([0, 3, 7, 39], got):
        assert np.array_equal(row, full[r])
    cores, model = bench.host_cpu()
    assert cores >= 1 and model
