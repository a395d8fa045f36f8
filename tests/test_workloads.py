"""The synthetic workloads follow their stated recipes (no GPU): sizes, bands, grids and the drawn
parameter ranges of the plain, batched-n, follow-up and uneven workloads.  The k step of the one
injection placed on a chosen row is checked against the oracle's own grid."""
import dataclasses

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth, workloads as W


def oracle_grid(fields):
    keep = {f.name for f in dataclasses.fields(O.Grid)}
    return O.make_grid(O.Grid(**{k: v for k, v in fields.items() if k in keep}))


def test_plain_small():
    spec, pm, grids = W.plain_small()
    assert (spec.fs, spec.t_obs, spec.t_fft) == (1024.0, 1800.0, 2.0)
    assert spec.n_samples == 1843200 and spec.n_per_fft == 2048 and spec.n_fft == 1799
    assert (pm["bin_lo"], pm["bin_hi"]) == (200, 799)                     # 100-400 Hz
    (g,) = grids
    assert (g["n"], g["n_k"], g["ana_lo"], g["ana_hi"]) == (5.0, 500, 100.0, 400.0)
    (inj,) = spec.injections
    assert inj.f0 == 350.0 and inj.n == 5.0
    o = oracle_grid(g)
    assert inj.k / o.dk == pytest.approx(300.0, rel=1e-12)               # on k row 300
    # spectral SNR 4 with a boxcar window: A^2 N / (4 sigma^2) = 4
    assert inj.amp ** 2 * spec.n_per_fft / 4.0 == pytest.approx(4.0, rel=1e-12)


def test_plain_paper():
    spec, pm, grids = W.plain_paper()
    assert (spec.fs, spec.t_obs, spec.t_fft, spec.n_fft) == (4096.0, 10080.0, 4.0, 5039)
    assert (pm["bin_lo"], pm["bin_hi"]) == (200, 7999)                    # 50-2000 Hz, 7800 bins
    assert len(grids) == 20
    for q, g in enumerate(grids):
        lo = 50.0 + 100.0 * q
        hi = min(lo + 100.0, 2000.0)
        assert (g["ana_lo"], g["ana_hi"]) == (lo, hi)
        assert g["bin_lo"] == round(lo * 4) and g["bin_hi"] == round(min(hi + 50.0, 2000.0) * 4) - 1
        assert (g["n"], g["n_k"], g["n_fft"]) == (5.0, 2000, 5039)
    assert len(spec.injections) == 20
    for inj in spec.injections:
        fdot = inj.k * inj.f0 ** inj.n
        assert 500.0 <= inj.f0 <= 1800.0 and 2.5 <= inj.n <= 7.0
        assert 1e-4 * (1 - 1e-12) <= fdot <= 1.0 / 16.0 * (1 + 1e-12)      # capped at 1/T_FFT^2
        assert inj.amp == pytest.approx(synth.amplitude_for_snr(4.0, 1.0, 16384), rel=1e-15)


def test_batched_n():
    spec, pm, grids = W.batched_n()
    assert len(grids) == 51
    ns = [g["n"] for g in grids]
    assert ns[0] == 2.0 and ns[-1] == 7.0 and np.allclose(np.diff(ns), 0.1)
    ks = [g["n_k"] for g in grids]
    assert ks[0] == 4000 and ks[-1] == 1000 and all(a >= b for a, b in zip(ks, ks[1:]))
    assert all((g["bin_lo"], g["bin_hi"]) == (200, 799) for g in grids)


def test_followup_fields_are_an_original_fh_grid():
    inj = synth.Injection(f0=812.3, k=1e-19, n=4.0, amp=1.0)
    (lo, hi), f = W.followup_fields(inj, 10080.0, 8.0)
    df = 1.0 / 8.0
    assert f["n"] == 0.0 and f["df"] == df and f["dk"] == df / 10080.0
    assert f["k_min"] == -16 * f["dk"] and f["n_k"] == 32                 # fdot rows centred on 0
    assert lo * df <= 812.3 - 5.0 < (lo + 1) * df and (hi - 1) * df < 812.3 + 5.0 <= hi * df
    assert f["n_fft"] == 2519 and f["t_hop"] == 4.0
    g = oracle_grid(f)
    assert g.n_x0 > 0 and O.n_bands(g) == 1


def test_uneven_recipe():
    specs = W.uneven_specs()
    assert len(specs) == 256
    for s in specs:
        assert 3600.0 * (1 - 1e-12) <= s["t_obs"] <= 24 * 3600.0 * (1 + 1e-12)
        assert s["t_fft"] in (1.0, 2.0, 4.0, 8.0)
        assert s["n_fft"] == int((s["t_obs"] - s["t_fft"]) // (s["t_fft"] / 2)) + 1
        assert 50.0 <= s["f_lo"] < s["f_hi"] <= 2000.0
        w = s["f_hi"] - s["f_lo"]
        assert 20.0 - 2 * s["df"] <= w <= 1950.0
        assert len(s["injs"]) <= 3
        for f0, k, n in s["injs"]:
            fdot = k * f0 ** n
            assert 2.0 <= n <= 7.0 and s["f_lo"] - s["df"] <= f0 <= s["f_hi"] + s["df"]
            assert 1e-4 * (1 - 1e-12) <= fdot <= 1.0 / s["t_fft"] ** 2 * (1 + 1e-12)
        if s["injs"]:
            assert s["n"] == s["injs"][0][2]
        else:
            assert 2.0 <= s["n"] <= 7.0
    # the spread the recipe asks for: every T_FFT, short and long data, narrow and wide bands
    assert {s["t_fft"] for s in specs} == {1.0, 2.0, 4.0, 8.0}
    assert min(s["t_obs"] for s in specs) < 2 * 3600 and max(s["t_obs"] for s in specs) > 16 * 3600
    widths = [s["f_hi"] - s["f_lo"] for s in specs]
    assert min(widths) < 40.0 and max(widths) > 1000.0


def test_uneven_grids_tile_each_band():
    specs = W.uneven_specs()
    grids = W.uneven_grids(specs)
    assert len(grids) == 1290
    for l, s in enumerate(specs):
        mine = [g for g in grids if g["list"] == l]
        assert mine and mine[0]["ana_lo"] == s["f_lo"]
        for g, h in zip(mine, mine[1:]):
            assert h["ana_lo"] == g["ana_hi"]                          # consecutive 100 Hz bands
        assert mine[-1]["ana_hi"] == pytest.approx(s["f_hi"], abs=1e-9)
        for g in mine:
            assert g["ana_hi"] - g["ana_lo"] <= 100.0 + 1e-9
            assert g["bin_lo"] == round(g["ana_lo"] / s["df"])
            top = min(g["ana_hi"] + 50.0, s["f_hi"])
            assert g["bin_hi"] == round(top / s["df"]) - 1 and g["bin_hi"] <= s["bin_hi"]
            assert (g["n"], g["n_k"], g["n_fft"]) == (s["n"], 1000, s["n_fft"])
