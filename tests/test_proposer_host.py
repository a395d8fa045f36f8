"""Host side of the learned tile proposer (no GPU): the track probability against the noise tail
and its monotonicity, the drawn samples (deterministic in their ids, classes inside the 64 x 64
tiles or the null class, tracks inside the band, the injection's x0 column against the oracle's
grid), the detection radius and the recall summary."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import proposer as PR


def test_track_probability():
    # no signal: the exponential tail of a chi-square of 2 degrees of freedom over 2
    assert float(PR.track_probability(0.0)) == pytest.approx(math.exp(-2.5), rel=1e-12)
    p = PR.track_probability(np.linspace(0.0, 12.0, 49))
    assert np.all(np.diff(p) > 0) and p[-1] > 0.99
    # a bin holding a signal of power s: P(|s^(1/2) + z|^2 > 2.5) by direct integration over the
    # noise phase and amplitude (z complex normal of unit power)
    s = 3.0
    r = np.linspace(0.0, 8.0, 4001)[1:]
    ph = np.linspace(0.0, 2 * np.pi, 721)[:-1]
    R, PH = np.meshgrid(r, ph)
    inside = (np.sqrt(s) + R * np.cos(PH)) ** 2 + (R * np.sin(PH)) ** 2 > 2.5
    dens = 2 * R * np.exp(-R ** 2)                    # |z| Rayleigh, E|z|^2 = 1
    direct = float(np.sum(inside * dens) * (r[1] - r[0]) / ph.size)
    assert float(PR.track_probability(s)) == pytest.approx(direct, abs=2e-3)


def test_draw_is_deterministic_and_labelled(built_lib):
    spec = PR.ProposerSpec()
    ids = np.arange(40, 160)
    a, b = PR.draw(spec, ids), PR.draw(spec, ids)
    for f in dataclasses.fields(a):
        assert np.array_equal(getattr(a, f.name), getattr(b, f.name))
    # a sample does not depend on the batch it is drawn in
    c = PR.draw(spec, ids[7:9])
    assert np.array_equal(c.tracks, a.tracks[7:9]) and np.array_equal(c.labels, a.labels[7:9])
    assert 0 < a.signal.sum() < ids.size
    for i in range(ids.size):
        assert a.n[i] == PR.N_GRID[ids[i] % len(PR.N_GRID)]
        if not a.signal[i]:
            assert a.labels[i] == PR.NULL_CLASS and a.row[i] == -1 and a.col[i] == -1
            assert np.all(a.tracks[i] == -1) and a.p_track24[i] == 0
            continue
        assert 0 <= a.labels[i] < PR.NULL_CLASS
        assert a.labels[i] % PR.TILES == min(
            PR.TILES - 1, int((a.f0[i] - spec.ana_lo) / (spec.ana_hi - spec.ana_lo) * PR.TILES))
        tr = a.tracks[i]
        ok = tr >= 0
        assert np.all((tr[ok] >= spec.bin_lo) & (tr[ok] <= spec.bin_hi))
        assert np.all(np.diff(tr[ok]) <= 0)               # spinning down
        # the injection's k is on its row and its x0 column is the oracle grid's
        keep = {f.name for f in dataclasses.fields(O.Grid)}
        og = O.make_grid(O.Grid(**{k: v for k, v in spec.grid_fields(float(a.n[i])).items()
                                   if k in keep}))
        assert og.dk == pytest.approx(og.dx0 / ((a.n[i] - 1.0) * spec.t_obs), rel=1e-15)
        assert a.k[i] == pytest.approx(a.row[i] * og.dk, rel=1e-12, abs=1e-300)
        x0 = a.f0[i] ** (1.0 - a.n[i])
        assert a.col[i] == math.floor((x0 - og.x0_min) / og.dx0)
        assert a.p_track24[i] == round(float(PR.track_probability(a.snr[i])) * 2 ** 24)


def test_detected_radius():
    rec = np.zeros(4, dtype=[("count", np.int32), ("col", np.int64), ("row", np.int32)])
    rec["count"] = [5, 7, -1, 3]
    rec["col"] = [100, 200, 50, 400]
    rec["row"] = [10, 20, 5, 40]
    assert PR.detected(rec, 103, 10)                        # distance 3
    assert not PR.detected(rec, 103, 11)                    # sqrt(10) > 3
    assert not PR.detected(rec, 50, 5)                      # only an empty band's record there
    assert PR.detected(rec, 402, 42, radius=3.0)            # sqrt(8)


def test_summarize():
    rec = dict(signal=np.array([1, 1, 1, 0, 0], bool), det_full=np.array([1, 1, 0, 1, 0], bool),
               det_pruned=np.array([1, 0, 0, 1, 0], bool), agree=np.array([1, 0, 1, 1, 1], bool),
               full=np.array([0, 1, 0, 0, 1], bool), tiles=np.array([32, 0, 30, 28, 0]),
               truth_in_top=np.array([1, 1, 0, 0, 0], bool))
    s = PR.summarize(rec)
    assert (s["maps"], s["injected"], s["det_full"], s["det_kept"]) == (5, 3, 2, 1)
    assert s["recall"] == 0.5 and s["agreement"] == pytest.approx(2 / 3)
    assert s["fallback_frac"] == 0.4 and s["fallback_injected"] == pytest.approx(1 / 3)
    assert s["fallback_noise"] == 0.5 and s["mean_tiles_pruned"] == 30.0
    assert s["truth_in_top"] == pytest.approx(2 / 3)
