"""GPU parity of the Hough map and candidates against the oracle, through the C ABI."""

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth, workloads

from gpu_util import (alloc_outputs, assert_candidates_equal, oracle_grid, read_cands,
                      read_stats, to_dev)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run_hough(gfh, ctx, fields, fi, bj, tile=None):
    g = gfh.grid_make(gfh.Grid(**fields))
    hmap, cands, stats = alloc_outputs(torch, g)
    dfi, dbj = to_dev(torch, fi.astype(np.uint32)), to_dev(torch, bj.astype(np.uint32))
    if tile is None:
        ctx.hough(dfi, dbj, len(fi), g, hmap, cands, stats)
    else:
        off = to_dev(torch, np.array([0, len(fi)], np.int64))
        plan = gfh.Plan(ctx, [g], [hmap], [cands], stats, tile=tile)
        plan.execute(dfi, dbj, off, 1)
        torch.cuda.synchronize()
        plan.close()
    torch.cuda.synchronize()
    assert ctx.check() == gfh.GFH_OK
    return g, hmap.cpu().numpy(), read_cands(gfh, cands), read_stats(gfh, stats)


def check_against_oracle(g, hm, cands, stats, fields, fi, bj):
    o = oracle_grid(fields)
    ref = O.hough_map(o, fi, bj)
    assert np.array_equal(hm[:, : g.n_x0], ref)
    assert np.all(hm[:, g.n_x0:] == 0)
    oc, (s1, s2, cells) = O.select_candidates(o, ref)
    assert (int(stats["sum"][0]), int(stats["sum_sq"][0]), int(stats["cells"][0])) == (s1, s2, cells)
    assert_candidates_equal(cands, oc, g.n_bands)


def medium_case(seed, n=5.0, n_k=37, n_fft=60, nb=300, bin_lo=200, density=0.08, **kw):
    fields = dict(n=n, df=0.5, bin_lo=bin_lo, bin_hi=bin_lo + nb - 1, n_fft=n_fft, t_first=1.0,
                  t_hop=1.0, t_obs=float(n_fft + 1), n_k=n_k, k_min=0.0, dk=0.0, f_max=0.0,
                  ana_lo=bin_lo * 0.5 + 1.0, ana_hi=(bin_lo + nb) * 0.5 - 3.0, band_hz=1.0, list=0)
    fields.update(kw)
    fi, bj = synth.random_peaklist(n_fft, bin_lo - 2, bin_lo + nb + 1, density, seed)
    return fields, fi, bj


# (rows, cols, threads[, drawing form]); form 1 draws one form per warp
TILES = [(8, 128, 256), (16, 1024, 512), (16, 3072, 512), (32, 640, 256), (8, 4096, 512),
         (32, 1536, 256), (16, 384, 512), (8, 3072, 512), (8, 2048, 512), (16, 3072, 1024),
         (32, 1024, 1024), (16, 640, 1024), (8, 128, 256, 1), (16, 3072, 1024, 1),
         (8, 3072, 512, 1), (4, 1024, 256, 1)]


@pytest.mark.parametrize("tile", TILES, ids=str)
def test_medium_maps_every_tile_shape(built_lib, gpu_ctx, tile):
    for seed, kw in ((1, {}), (2, dict(n=7.0, n_k=5)), (3, dict(n=2.0, n_k=70)),
                     (4, dict(n=3.5, k_min=1e-9, dk=4e-10))):
        fields, fi, bj = medium_case(seed, **kw)
        g, hm, c, s = run_hough(built_lib, gpu_ctx, fields, fi, bj, tile=tile)
        check_against_oracle(g, hm, c, s, fields, fi, bj)


def test_plain_small_full_map(built_lib, gpu_ctx):
    """1800 s at 1024 Hz, 100-400 Hz, n = 5, 500 k rows: every cell and candidate."""
    spec, pm, grids = workloads.plain_small()
    x = spec.series()
    fi, bj = O.peakmap(x, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"])
    g, hm, c, s = run_hough(built_lib, gpu_ctx, grids[0], fi, bj)
    check_against_oracle(g, hm, c, s, grids[0], fi, bj)
    # the injection (row 300, f0 = 350 Hz) is the loudest candidate
    best = c[np.argmax(c["count"])]
    assert int(best["row"]) == pytest.approx(300, abs=2) and abs(best["f0"] - 350.0) < 1.0


def test_autotuned_plan_gives_the_same_map(built_lib, gpu_ctx):
    """The autotuner only changes the tile shape: the map and candidates stay bit-exact."""
    fields, fi, bj = medium_case(5, n_k=45, nb=400)
    g = built_lib.grid_make(built_lib.Grid(**fields))
    hmap, cands, stats = alloc_outputs(torch, g)
    dfi, dbj = to_dev(torch, fi), to_dev(torch, bj)
    off = to_dev(torch, np.array([0, len(fi)], np.int64))
    plan = built_lib.Plan(gpu_ctx, [g], [hmap], [cands], stats)
    best, ms = plan.autotune(dfi, dbj, off, 1, reps=1)
    assert best[0] in (4, 8, 16, 32) and ms > 0
    hmap.fill_(-7)
    plan.execute(dfi, dbj, off, 1)
    torch.cuda.synchronize()
    plan.close()
    check_against_oracle(g, hmap.cpu().numpy(), read_cands(built_lib, cands),
                         read_stats(built_lib, stats), fields, fi, bj)


def test_autotune_cache(built_lib, gpu_ctx):
    """A plan whose signature was tuned before takes the cached shape: the cache keeps one entry
    per signature, a second plan of the same grid and lists reuses it, another peak density is a
    new entry, and the maps stay bit-exact."""
    gfh = built_lib
    gfh.autotune_cache_clear()
    assert gfh.autotune_cache_size() == 0
    fields, fi, bj = medium_case(6, n_k=45, nb=400)
    g = gfh.grid_make(gfh.Grid(**fields))
    dfi, dbj = to_dev(torch, fi), to_dev(torch, bj)
    off = to_dev(torch, np.array([0, len(fi)], np.int64))
    shapes = []
    for _ in range(2):
        hmap, cands, stats = alloc_outputs(torch, g)
        plan = gfh.Plan(gpu_ctx, [g], [hmap], [cands], stats, tile=(4, 1024, 256))
        best, ms = plan.autotune(dfi, dbj, off, 1, reps=1)
        shapes.append(best)
        assert gfh.autotune_cache_size() == 1 and ms > 0
        hmap.fill_(-7)
        plan.execute(dfi, dbj, off, 1)
        torch.cuda.synchronize()
        plan.close()
        check_against_oracle(g, hmap.cpu().numpy(), read_cands(gfh, cands), read_stats(gfh, stats),
                             fields, fi, bj)
    assert shapes[0] == shapes[1]
    # a sparser list of the same grid: another density class, another entry
    keep = np.arange(len(fi)) % 4 == 0
    fi4, bj4 = fi[keep], bj[keep]
    hmap, cands, stats = alloc_outputs(torch, g)
    plan = gfh.Plan(gpu_ctx, [g], [hmap], [cands], stats)
    plan.autotune(to_dev(torch, fi4), to_dev(torch, bj4),
                  to_dev(torch, np.array([0, len(fi4)], np.int64)), 1, reps=1)
    plan.close()
    assert gfh.autotune_cache_size() == 2
    gfh.autotune_cache_clear()
    assert gfh.autotune_cache_size() == 0


def test_edge_cases(built_lib, gpu_ctx):
    fields, fi, bj = medium_case(9)
    # empty list: all-zero map, candidates at the first cell of each band
    g, hm, c, s = run_hough(built_lib, gpu_ctx, fields, fi[:0], bj[:0])
    check_against_oracle(g, hm, c, s, fields, fi[:0], bj[:0])
    # one peak; a single k row; peaks on the first and last bins of the band
    g, hm, c, s = run_hough(built_lib, gpu_ctx, fields, fi[:1], bj[:1])
    check_against_oracle(g, hm, c, s, fields, fi[:1], bj[:1])
    f1 = dict(fields, n_k=1)
    g, hm, c, s = run_hough(built_lib, gpu_ctx, f1, fi, bj)
    check_against_oracle(g, hm, c, s, f1, fi, bj)
    edge_fi = np.array([0, 5, 59, 3], np.uint32)
    edge_bj = np.array([fields["bin_lo"], fields["bin_lo"], fields["bin_hi"], fields["bin_hi"]], np.uint32)
    g, hm, c, s = run_hough(built_lib, gpu_ctx, fields, edge_fi, edge_bj)
    check_against_oracle(g, hm, c, s, fields, edge_fi, edge_bj)


def test_bad_input_sets_flag_without_fault(built_lib, gpu_ctx):
    fields, fi, bj = medium_case(10)
    g = built_lib.grid_make(built_lib.Grid(**fields))
    hmap, cands, stats = alloc_outputs(torch, g)
    bad_bj = bj[::-1].copy()                                  # unsorted
    gpu_ctx.hough(to_dev(torch, fi), to_dev(torch, bad_bj), len(fi), g, hmap, cands, stats)
    assert gpu_ctx.check() == built_lib.GFH_ERR_INPUT
    bad_fi = fi.copy()
    bad_fi[len(fi) // 2] = fields["n_fft"] + 5                # FFT index out of range
    gpu_ctx.hough(to_dev(torch, bad_fi), to_dev(torch, bj), len(fi), g, hmap, cands, stats)
    assert gpu_ctx.check() == built_lib.GFH_ERR_INPUT
    assert gpu_ctx.check() == built_lib.GFH_OK                # flag was cleared
    g2, hm, c, s = run_hough(built_lib, gpu_ctx, fields, fi, bj)   # context still usable
    check_against_oracle(g2, hm, c, s, fields, fi, bj)


def test_select_alone_on_oracle_map(built_lib, gpu_ctx):
    fields, fi, bj = medium_case(11, n_k=23)
    o = oracle_grid(fields)
    ref = O.hough_map(o, fi, bj)
    g = built_lib.grid_make(built_lib.Grid(**fields))
    hm = np.zeros((g.n_k, g.ld_x0), np.int32)
    hm[:, : g.n_x0] = ref
    _, cands, stats = alloc_outputs(torch, g)
    gpu_ctx.select(to_dev(torch, hm), g, cands, stats)
    torch.cuda.synchronize()
    oc, (s1, s2, cells) = O.select_candidates(o, ref)
    st = read_stats(built_lib, stats)
    assert (int(st["sum"][0]), int(st["sum_sq"][0]), int(st["cells"][0])) == (s1, s2, cells)
    assert_candidates_equal(read_cands(built_lib, cands), oc, g.n_bands)


@pytest.fixture(scope="module")
def paper_case():
    spec, pm, grids = workloads.plain_paper()
    x = spec.series()
    fi, bj = O.peakmap(x, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"])
    return spec, pm, grids, x, fi, bj


def test_plain_paper_all_subbands(built_lib, gpu_ctx, paper_case):
    """2.8 h at 4096 Hz, 50-2000 Hz in 20 sub-bands at n = 5 with 2000 k rows, one launch:
    two sub-band maps compared cell by cell, three full rows and 200 sampled cells of every other
    map, and every candidate's count checked by direct counting."""
    spec, pm, grids, x, fi, bj = paper_case
    gs = [built_lib.grid_make(built_lib.Grid(**f)) for f in grids]
    maps = [torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda") for g in gs]
    cands = [torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in gs]
    stats = torch.zeros(24 * len(gs), dtype=torch.uint8, device="cuda")
    plan = built_lib.Plan(gpu_ctx, gs, maps, cands, stats)
    plan.execute(to_dev(torch, fi), to_dev(torch, bj), to_dev(torch, np.array([0, len(fi)], np.int64)), 1)
    torch.cuda.synchronize()
    assert gpu_ctx.check() == built_lib.GFH_OK
    rng = np.random.default_rng(0)
    st = read_stats(built_lib, stats)
    for m, (f, g) in enumerate(zip(grids, gs)):
        o = oracle_grid(f)
        hm = maps[m].cpu().numpy()
        assert np.all(hm[:, g.n_x0:] == 0)
        c = read_cands(built_lib, cands[m])
        if m in (0, len(gs) - 1):
            ref = O.hough_map(o, fi, bj)
            assert np.array_equal(hm[:, : g.n_x0], ref)
            oc, (s1, s2, cells) = O.select_candidates(o, ref)
            assert (int(st["sum"][m]), int(st["sum_sq"][m]), int(st["cells"][m])) == (s1, s2, cells)
            assert_candidates_equal(c, oc, g.n_bands)
            continue
        for r in (0, g.n_k // 2, g.n_k - 1):
            assert np.array_equal(hm[r, : g.n_x0], O.hough_row(o, fi, bj, r))
        rows = rng.integers(0, g.n_k, 200)
        cols = rng.integers(0, g.n_x0, 200)
        assert np.array_equal(hm[rows, cols], O.hough_cells(o, fi, bj, rows, cols))
        ok = c["count"] >= 0
        assert np.array_equal(O.hough_cells(o, fi, bj, c["row"][ok], c["col"][ok]), c["count"][ok])
        # every candidate is its band's maximum: no sampled cell of the band exceeds it
        _, _, band = O.column_bands(o)
        for r_, c_ in zip(rows, cols):
            b = band[c_]
            if b >= 0:
                assert hm[r_, c_] <= c["count"][b]
    plan.close()


def test_shared_atomic_probe_counts_every_update(built_lib, gpu_ctx):
    """The roofline probe's three access patterns each land every one of their atomic adds (the
    array of every block sums to threads x iterations) and report positive cycle counts."""
    gfh = built_lib
    blocks, threads, iters = 8, 256, 64
    cycles = torch.zeros(blocks, dtype=torch.int64, device="cuda")
    sink = torch.zeros(blocks, dtype=torch.int32, device="cuda")
    assert gpu_ctx.sms() >= 1
    for mode in (0, 1, 2):
        sink.zero_()
        gpu_ctx.probe_smem_atomics(mode, blocks, threads, iters, cycles, sink)
        torch.cuda.synchronize()
        assert bool((sink == threads * iters).all()), mode
        assert bool((cycles > 0).all())
