"""The batched search on paper-derived grids: braking indices from Eq. dn_powlaws and, for each, the
Eq. dkeqn k grid as uniform segments, all as maps of one plan over one peak list.  Rows against the
oracle bit for bit; the injection found at its braking index, f0 and spin-down."""
import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth, workloads

from gpu_util import oracle_grid, read_cands, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_paper_grids_in_one_plan(built_lib, gpu_ctx):
    gfh = built_lib
    spec, pm, base = workloads.plain_small()
    df, fmin, fmax = spec.df, 100.0, pm["bin_hi"] * spec.df
    fdot_lo, fdot_hi = 1e-3, 4e-3
    ns = gfh.n_grid(4.8, 5.2, df, fmin, fmax, fdot_hi, spec.t_obs)
    assert 2 <= ns.size <= 50
    f0_true, fdot_true, n_true = 330.0, 2.2e-3, float(ns[ns.size // 2])
    k_true = fdot_true / f0_true ** n_true
    track = synth.powerlaw_track(f0_true, k_true, n_true, df, spec.n_fft, spec.t_first, spec.t_hop)
    track[(track < pm["bin_lo"]) | (track > pm["bin_hi"])] = -1
    fi, bj = synth.hashed_peaklist(5, 0, spec.n_fft, pm["bin_lo"], pm["bin_hi"],
                                   int(0.0755 * 2 ** 24), int(0.9 * 2 ** 24), track)
    fields = []
    for n in ns:
        for s in gfh.k_segments(float(n), df, fmin, fmax, fdot_lo, fdot_hi, growth=2.0, max_rows=512):
            fields.append(dict(base[0], n=float(n), k_min=float(s["k_min"]), dk=float(s["dk"]),
                               n_k=int(s["n_k"]), list=0))
    gs = [gfh.grid_make(gfh.Grid(**f)) for f in fields]
    maps = [torch.empty((g.n_k, g.ld_x0), dtype=torch.int32, device="cuda") for g in gs]
    cands = [torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in gs]
    plan = gfh.Plan(gpu_ctx, gs, maps, cands)
    plan.execute(to_dev(torch, fi), to_dev(torch, bj), to_dev(torch, np.array([0, fi.size], np.int64)), 1)
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    rng = np.random.default_rng(0)
    for m in rng.choice(len(gs), size=min(6, len(gs)), replace=False):
        o = oracle_grid(fields[m])
        for r in (0, gs[m].n_k - 1, gs[m].n_k // 2):
            assert np.array_equal(maps[m][r, : gs[m].n_x0].cpu().numpy(), O.hough_row(o, fi, bj, r))
    recs = [read_cands(gfh, t) for t in cands]
    best = max((int(c["count"]), m, i) for m, r in enumerate(recs) for i, c in enumerate(r) if c["count"] >= 0)
    _, m, i = best
    c = recs[m][i]
    assert abs(float(c["f0"]) - f0_true) < 1.0
    assert abs(-float(c["fdot0"]) / fdot_true - 1) < 0.1
    # the n step keeps neighbouring braking indices within one bin of each other (Eq. dn_powlaws):
    # the injection's own n finds it about as strongly as the best map
    own = max(int(c["count"]) for mm, r in enumerate(recs) if abs(fields[mm]["n"] - n_true) < 1e-12
              for c in r)
    assert own >= 0.9 * best[0]
    plan.close()


def test_coarse_and_fine_k_steps_in_one_plan(built_lib, gpu_ctx):
    """Maps whose lines move less than two x0 columns per k row (differenced along k) and maps
    with coarse k steps (differenced along x0 on every row) in one plan: both bit-exact against
    the oracle, maps and candidates; the coarse-tile search refuses such a plan."""
    from gpu_util import assert_candidates_equal
    gfh = built_lib
    spec, pm, base = workloads.plain_small()
    fi, bj = synth.random_peaklist(spec.n_fft, pm["bin_lo"], pm["bin_hi"], 0.0755, 9)
    g_fine = gfh.grid_make(gfh.Grid(**dict(base[0], n_k=40)))
    fields = [dict(base[0], n_k=40),                                   # default step
              dict(base[0], n_k=23, dk=g_fine.dk * 7.5),               # 7.5 columns per row
              dict(base[0], n=3.0, n_k=17, k_min=g_fine.dk, dk=1.3e-11)]   # ~3 columns per row
    gs = [gfh.grid_make(gfh.Grid(**f)) for f in fields]
    maps = [torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda") for g in gs]
    cands = [torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in gs]
    plan = gfh.Plan(gpu_ctx, gs, maps, cands, tile=(8, 2048, 512))
    plan.execute(to_dev(torch, fi), to_dev(torch, bj), to_dev(torch, np.array([0, fi.size], np.int64)), 1)
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    for f, g, m, c in zip(fields, gs, maps, cands):
        o = oracle_grid(f)
        ref = O.hough_map(o, fi, bj)
        assert np.array_equal(m.cpu().numpy()[:, : g.n_x0], ref), f["n_k"]
        oc, _ = O.select_candidates(o, ref)
        assert_candidates_equal(read_cands(gfh, c), oc, g.n_bands)
    with pytest.raises(gfh.GfhError):
        plan.set_coarse(64, 64, 8)
    plan.close()
