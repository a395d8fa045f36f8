"""Batched search: one plan (one Hough launch) over many braking indices with uneven map sizes,
against the oracle map by map."""
import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth, workloads

from gpu_util import assert_candidates_equal, oracle_grid, read_cands, read_stats, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_peaks():
    spec, pm, _ = workloads.plain_small()
    fi, bj = O.peakmap(spec.series(), spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"])
    return fi, bj


def test_batched_braking_indices_one_launch(built_lib, gpu_ctx, small_peaks):
    """Six of the 51 braking indices (n = 2.0 .. 7.0, 4000 -> 1000 k rows) in one plan: small maps
    cell by cell, the largest (n = 7, 0.55M columns) by rows and cells, every candidate's count by
    direct counting."""
    gfh = built_lib
    fi, bj = small_peaks
    _, _, all_fields = workloads.batched_n()
    pick = [0, 7, 13, 30, 42, 50]                    # n = 2.0, 2.7, 3.3, 5.0, 6.2, 7.0
    fields = [all_fields[i] for i in pick]
    gs = [gfh.grid_make(gfh.Grid(**f)) for f in fields]
    maps = [torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda") for g in gs]
    cands = [torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in gs]
    stats = torch.zeros(24 * len(gs), dtype=torch.uint8, device="cuda")
    plan = gfh.Plan(gpu_ctx, gs, maps, cands, stats)
    plan.execute(to_dev(torch, fi), to_dev(torch, bj), to_dev(torch, np.array([0, len(fi)], np.int64)), 1)
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    st = read_stats(gfh, stats)
    rng = np.random.default_rng(1)
    for m, (f, g) in enumerate(zip(fields, gs)):
        o = oracle_grid(f)
        c = read_cands(gfh, cands[m])
        if g.n_k * g.n_x0 < 6e7:
            hm = maps[m].cpu().numpy()
            ref = O.hough_map(o, fi, bj)
            assert np.array_equal(hm[:, : g.n_x0], ref), f["n"]
            assert np.all(hm[:, g.n_x0:] == 0)
            oc, (s1, s2, cells) = O.select_candidates(o, ref)
            assert (int(st["sum"][m]), int(st["sum_sq"][m]), int(st["cells"][m])) == (s1, s2, cells)
            assert_candidates_equal(c, oc, g.n_bands)
        else:
            for r in (0, 1, g.n_k // 3, g.n_k - 1):
                assert np.array_equal(maps[m][r, : g.n_x0].cpu().numpy(), O.hough_row(o, fi, bj, r))
            rows = rng.integers(0, g.n_k, 300)
            cols = rng.integers(0, g.n_x0, 300)
            got = maps[m][torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
            assert np.array_equal(got, O.hough_cells(o, fi, bj, rows, cols))
            ok = c["count"] >= 0
            assert np.array_equal(O.hough_cells(o, fi, bj, c["row"][ok], c["col"][ok]), c["count"][ok])
    plan.close()


def test_uneven_peakmaps_scaled_down(built_lib, gpu_ctx):
    """The uneven workload's generator at small sizes (minutes of data, narrow bands): every
    sub-band map of every peakmap, from one launch, equals the oracle's."""
    gfh = built_lib
    lists, fields, _ = workloads.uneven(seed=11, n_maps=6, hours=(0.05, 0.3), width_hz=(20.0, 160.0),
                                        n_k=24)
    off = np.cumsum([0] + [len(f) for f, _ in lists]).astype(np.int64)
    all_fi = np.concatenate([f for f, _ in lists]).astype(np.uint32)
    all_bj = np.concatenate([b for _, b in lists]).astype(np.uint32)
    gs = [gfh.grid_make(gfh.Grid(**f)) for f in fields]
    assert len(gs) > len(lists)                       # several sub-bands for some peakmaps
    maps = [torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda") for g in gs]
    cands = [torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in gs]
    plan = gfh.Plan(gpu_ctx, gs, maps, cands, None)
    plan.execute(to_dev(torch, all_fi), to_dev(torch, all_bj), to_dev(torch, off), len(lists))
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    for m, (f, g) in enumerate(zip(fields, gs)):
        fi, bj = lists[f["list"]]
        o = oracle_grid(f)
        ref = O.hough_map(o, fi, bj)
        assert np.array_equal(maps[m].cpu().numpy()[:, : g.n_x0], ref), m
        oc, _ = O.select_candidates(o, ref)
        assert_candidates_equal(read_cands(gfh, cands[m]), oc, g.n_bands)
    plan.close()


def test_plans_of_different_sizes_interleave(built_lib, gpu_ctx):
    """Plans with different shared-memory needs for the same kernel shape can be created in any
    order and executed in any order (the kernel attribute is not per plan)."""
    gfh = built_lib
    rng = np.random.default_rng(9)
    fi, bj = synth.random_peaklist(80, 198, 702, 0.07, 9)
    plans, outs = [], []
    for ana_hi in (349.0, 120.0):            # many bands per tile, then few
        f = dict(n=5.0, df=0.5, bin_lo=200, bin_hi=699, n_fft=80, t_first=1.0, t_hop=1.0,
                 t_obs=81.0, n_k=16, ana_lo=100.5, ana_hi=ana_hi, band_hz=0.5)
        g = gfh.grid_make(gfh.Grid(**f))
        hm = torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda")
        c = torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda")
        plans.append(gfh.Plan(gpu_ctx, [g], [hm], [c], None, tile=(8, 2048, 256)))
        outs.append((f, g, hm, c))
    off = to_dev(torch, np.array([0, len(fi)], np.int64))
    for p in plans:                           # the first (larger) plan runs after the second exists
        p.execute(to_dev(torch, fi), to_dev(torch, bj), off, 1)
    torch.cuda.synchronize()
    for f, g, hm, c in outs:
        o = oracle_grid(f)
        ref = O.hough_map(o, fi, bj)
        assert np.array_equal(hm.cpu().numpy()[:, : g.n_x0], ref)
        oc, _ = O.select_candidates(o, ref)
        assert_candidates_equal(read_cands(gfh, c), oc, g.n_bands)
    for p in plans:
        p.close()


def test_many_uneven_peak_lists_one_launch(built_lib, gpu_ctx):
    """Several independent peak lists (different FFT counts, bands, braking indices) searched by one
    plan; each map equals the oracle's."""
    gfh = built_lib
    rng = np.random.default_rng(3)
    fields, lists = [], []
    for l in range(7):
        n_fft = int(rng.integers(20, 120))
        bin_lo = int(rng.integers(150, 400))
        nb = int(rng.integers(40, 300))
        n = float(rng.uniform(2.0, 7.0))
        fi, bj = synth.random_peaklist(n_fft, bin_lo - 1, bin_lo + nb, 0.07, 100 + l)
        lists.append((fi, bj))
        fields.append(dict(n=n, df=0.5, bin_lo=bin_lo, bin_hi=bin_lo + nb - 1, n_fft=n_fft,
                           t_first=1.0, t_hop=1.0, t_obs=float(n_fft + 1),
                           n_k=int(rng.integers(1, 90)), ana_lo=bin_lo * 0.5 + 0.5,
                           ana_hi=(bin_lo + nb) * 0.5 - 0.5, band_hz=1.0, list=l))
    off = np.cumsum([0] + [len(fi) for fi, _ in lists]).astype(np.int64)
    all_fi = np.concatenate([fi for fi, _ in lists]).astype(np.uint32)
    all_bj = np.concatenate([bj for _, bj in lists]).astype(np.uint32)
    gs = [gfh.grid_make(gfh.Grid(**f)) for f in fields]
    maps = [torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda") for g in gs]
    cands = [torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in gs]
    stats = torch.zeros(24 * len(gs), dtype=torch.uint8, device="cuda")
    plan = gfh.Plan(gpu_ctx, gs, maps, cands, stats, tile=(8, 1024, 256))
    plan.execute(to_dev(torch, all_fi), to_dev(torch, all_bj), to_dev(torch, off), len(lists))
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    st = read_stats(gfh, stats)
    for m, (f, g) in enumerate(zip(fields, gs)):
        fi, bj = lists[m]
        o = oracle_grid(f)
        ref = O.hough_map(o, fi, bj)
        hm = maps[m].cpu().numpy()
        assert np.array_equal(hm[:, : g.n_x0], ref)
        oc, (s1, s2, cells) = O.select_candidates(o, ref)
        assert (int(st["sum"][m]), int(st["sum_sq"][m]), int(st["cells"][m])) == (s1, s2, cells)
        assert_candidates_equal(read_cands(gfh, cands[m]), oc, g.n_bands)
    plan.close()
