"""The C ABI without a GPU: the library builds and loads, exports every declared entry point, and
its host-side planner (grids, fixed-point tables, column tables) equals the oracle bit for bit."""
import dataclasses
import pathlib
import re

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import workloads

HEADER = pathlib.Path(__file__).resolve().parent.parent / "include" / "gfh.h"


def declared_functions():
    text = HEADER.read_text()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+(gfh_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(built_lib):
    names = declared_functions()
    assert len(names) >= 15
    L = built_lib.lib()
    for name in names:
        assert hasattr(L, name), name
    assert sorted(built_lib.EXPORTED) == names


def test_autotune_cache_host_calls(built_lib):
    """The autotuner's cache is host state: its size and clearing need no GPU."""
    built_lib.autotune_cache_clear()
    assert built_lib.autotune_cache_size() == 0


def test_strerror(built_lib):
    assert built_lib.strerror(0) == "ok"
    assert "invalid" in built_lib.strerror(built_lib.GFH_ERR_ARG)


def _pairs():
    out = []
    spec, pm, grids = workloads.plain_small()
    out += grids
    _, _, grids = workloads.plain_paper()
    out += [grids[0], grids[7], grids[-2], grids[-1]]
    _, _, grids = workloads.batched_n()
    out += [grids[0], grids[13], grids[-1]]
    out.append(dict(grids[5], k_min=3e-19, dk=5e-18, f_max=401.0, band_hz=0.5))
    # original FrequencyHough (n = 0): spin-down only, and both signs of fdot
    base = workloads.plain_small()[2][0]
    out.append(dict(base, n=0.0, n_k=64))
    out.append(dict(base, n=0.0, n_k=64, k_min=-32 * 0.5 / 1800.0, ana_lo=150.0, ana_hi=350.0))
    return out


def oracle_grid(fields):
    keep = {f.name for f in dataclasses.fields(O.Grid)}
    return O.make_grid(O.Grid(**{k: v for k, v in fields.items() if k in keep}))


@pytest.mark.parametrize("fields", _pairs(), ids=lambda f: f"n{f['n']}_b{f['bin_lo']}-{f['bin_hi']}_k{f['n_k']}")
def test_grid_and_tables_match_oracle(built_lib, fields):
    g = built_lib.grid_make(built_lib.Grid(**fields))
    o = oracle_grid(fields)
    for name in ("dx0", "dk", "x0_min", "n_x0", "f_max"):
        assert getattr(g, name) == getattr(o, name), name      # bit-exact doubles
    assert g.ld_x0 % 32 == 0 and g.ld_x0 >= g.n_x0
    assert g.n_bands == O.n_bands(o)
    U, B, S = built_lib.grid_tables(g)
    assert np.array_equal(U, np.array(O.edge_positions(o), dtype=np.int64))
    oB, oS = O.fft_shifts(o)
    assert np.array_equal(B, np.array(oB, dtype=np.int64))
    assert np.array_equal(S, np.array(oS, dtype=np.int64))


@pytest.mark.parametrize("fields", _pairs()[:5], ids=str)
def test_column_tables_match_oracle(built_lib, fields):
    g = built_lib.grid_make(built_lib.Grid(**fields))
    o = oracle_grid(fields)
    band, f0, f0n = built_lib.grid_columns(g)
    of0, of0n, oband = O.column_bands(o)
    assert np.array_equal(band, oband.astype(np.int32))
    assert np.array_equal(f0, of0)
    assert np.array_equal(f0n, of0n)


def test_invalid_requests_are_rejected(built_lib):
    _, _, grids = workloads.plain_small()
    base = grids[0]
    for bad in (dict(n=1.0), dict(bin_hi=base["bin_lo"] - 1), dict(n_k=0), dict(df=0.0),
                dict(ana_hi=base["ana_lo"]), dict(band_hz=0.0), dict(k_min=-1.0), dict(n=0.5),
                dict(n=-1.0)):
        with pytest.raises(built_lib.GfhError) as e:
            built_lib.grid_make(built_lib.Grid(**dict(base, **bad)))
        assert e.value.code == built_lib.GFH_ERR_ARG
    # k < 0 (spin-up) is the original FrequencyHough's alone
    g = built_lib.grid_make(built_lib.Grid(**dict(base, n=0.0, k_min=-1e-3)))
    assert g.dx0 == base["df"]


def test_n_grid_matches_oracle(built_lib):
    args = (2.5, 7.0, 0.5, 100.0, 400.0, 0.02, 1800.0)
    got = built_lib.n_grid(*args)
    ref = np.array(O.n_grid(*args))
    assert got.size == ref.size
    assert np.allclose(got, ref, rtol=0, atol=1e-7)     # libm vs numpy exp/log1p: last-ulp level
    assert got[0] == 2.5 and got[-1] == 7.0


@pytest.mark.parametrize("growth", [1.0, 1.5, 2.0, 4.0])
def test_k_segments_match_oracle(built_lib, growth):
    args = (5.0, 0.5, 100.0, 400.0, 1e-6, 1e-3)
    got = built_lib.k_segments(*args, growth=growth)
    ref = O.k_segments(*args, growth=growth)
    assert got.size == len(ref)
    for g, (k0, dk, rows) in zip(got, ref):
        assert (float(g["k_min"]), float(g["dk"]), int(g["n_k"])) == (k0, dk, rows)


def test_k_segments_feed_grids(built_lib):
    """Each segment is a valid k grid of a map: grid_make accepts it and keeps its step."""
    segs = built_lib.k_segments(4.0, 0.5, 100.0, 400.0, 1e-5, 1e-4, growth=2.0, max_rows=400)
    _, _, grids = workloads.plain_small()
    for s in segs[:5]:
        g = built_lib.grid_make(built_lib.Grid(**dict(grids[0], n=4.0, k_min=float(s["k_min"]),
                                                      dk=float(s["dk"]), n_k=int(s["n_k"]))))
        assert g.dk == float(s["dk"]) and g.n_k == int(s["n_k"])
