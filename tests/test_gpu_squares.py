"""Squares candidates (two per square) and coincidences between two detectors' candidates, against
the oracle: integers bit-exact, fp64 fields equal (the same IEEE operations)."""
import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth, workloads

from gpu_util import oracle_grid, read_cands, read_stats, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _map(gfh, gpu_ctx, fields, fi, bj):
    g = gfh.grid_make(gfh.Grid(**fields))
    hm = torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda")
    gpu_ctx.hough(to_dev(torch, fi), to_dev(torch, bj), len(fi), g, hm)
    return g, hm


def _check(gfh, recs, ref, n_sq):
    assert len(recs) == 2 * n_sq
    for q in range(n_sq):
        for which in (0, 1):
            got = recs[2 * q + which]
            assert int(got["band"]) == q and int(got["reserved"]) == which
            want = ref.get((q, which))
            if want is None:
                assert int(got["count"]) == -1
                continue
            assert (int(got["count"]), int(got["row"]), int(got["col"])) == (want["count"], want["row"], want["col"])
            for name in ("cr", "x0", "k", "f0", "fdot0"):
                assert float(got[name]) == want[name], (q, which, name)


@pytest.mark.parametrize("n_sx,n_sk,min_dk", [(5, 5, 3), (7, 3, 0), (1, 1, 3), (13, 11, 5), (64, 64, 3)])
def test_squares_match_oracle(built_lib, gpu_ctx, n_sx, n_sk, min_dk):
    gfh = built_lib
    spec, pm, grids = workloads.plain_small()
    fields = dict(grids[0], n_k=97)
    fi, bj = synth.random_peaklist(spec.n_fft, pm["bin_lo"], pm["bin_hi"], 0.0755, 5)
    g, hm = _map(gfh, gpu_ctx, fields, fi, bj)
    out = torch.zeros(2 * n_sx * n_sk * 64, dtype=torch.uint8, device="cuda")
    stats = torch.zeros(24, dtype=torch.uint8, device="cuda")
    gpu_ctx.select_squares(hm, g, n_sx, n_sk, out, min_dk=min_dk, stats=stats)
    torch.cuda.synchronize()
    ref, (s1, s2, n) = O.select_squares(oracle_grid(fields), hm.cpu().numpy()[:, :g.n_x0], n_sx, n_sk, min_dk)
    _check(gfh, read_cands(gfh, out), ref, n_sx * n_sk)
    st = read_stats(gfh, stats)
    assert (int(st["sum"][0]), int(st["sum_sq"][0]), int(st["cells"][0])) == (s1, s2, n)


def test_two_detectors_coincide_on_the_injection(built_lib, gpu_ctx):
    """Two detectors see the same power-law track in independent noise: each map's squares give a
    candidate at the injection, and the two coincide within 3 bins (Sec. IV); the GPU matches the
    oracle's nearest-neighbour indices and distances exactly."""
    gfh = built_lib
    spec, pm, grids = workloads.plain_small()
    fields = grids[0]
    g0 = gfh.grid_make(gfh.Grid(**fields))
    n, f0 = fields["n"], 330.0
    k = 217 * g0.dk
    track = synth.powerlaw_track(f0, k, n, spec.df, spec.n_fft, spec.t_first, spec.t_hop)
    track[(track < pm["bin_lo"]) | (track > pm["bin_hi"])] = -1
    sets, recs = [], []
    for det in (11, 12):
        fi, bj = synth.hashed_peaklist(det, 0, spec.n_fft, pm["bin_lo"], pm["bin_hi"],
                                       int(0.0755 * 2 ** 24), int(0.7 * 2 ** 24), track)
        g, hm = _map(gfh, gpu_ctx, fields, fi, bj)
        out = torch.zeros(2 * 25 * 64, dtype=torch.uint8, device="cuda")
        gpu_ctx.select_squares(hm, g, 5, 5, out)
        sets.append(out)
        recs.append(read_cands(gfh, out))
    match = torch.empty(50, dtype=torch.int32, device="cuda")
    dist = torch.empty(50, dtype=torch.float64, device="cuda")
    gpu_ctx.coincide(sets[0], 50, sets[1], 50, g0.dx0, g0.dk, 3.0, match, dist)
    torch.cuda.synchronize()
    a = [dict(x0=float(r["x0"]), k=float(r["k"])) for r in recs[0]]
    b = [dict(x0=float(r["x0"]), k=float(r["k"])) for r in recs[1]]
    valid_a = recs[0]["count"] >= 0
    valid_b = recs[1]["count"] >= 0
    bi = [j for j in range(50) if valid_b[j]]
    om, od = O.coincidences([a[i] for i in range(50) if valid_a[i]], [b[j] for j in bi], g0.dx0, g0.dk, 3.0)
    gm, gd = match.cpu().numpy(), dist.cpu().numpy()
    for t, i in enumerate([i for i in range(50) if valid_a[i]]):
        assert gd[i] == od[t]
        assert gm[i] == (bi[om[t]] if om[t] >= 0 else -1)
    # the injection: the strongest candidate of detector A sits at the true (x0, k) and coincides
    top = int(np.argmax(recs[0]["count"]))
    x0_true = f0 ** (1.0 - n)
    col_true = int(np.floor((x0_true - g0.x0_min) / g0.dx0))
    assert abs(int(recs[0]["row"][top]) - 217) <= 3 and abs(int(recs[0]["col"][top]) - col_true) <= 3
    assert gm[top] >= 0 and gd[top] <= 3.0
