"""Sec. VI.D on the GPU: a power law spinning down fast enough that its first portion needs 2 s FFTs
and its second allows 4 s FFTs is searched portion by portion (peakmap of the portion's samples,
Hough map on the common t0); every portion's map and candidates equal the oracle's on the same
peaks, the injection is the top candidate of its band in both portions, and the two candidates
coincide (Sec. IV distance <= 3 on the coarser grid) exactly as the oracle's coincidences say."""
import math

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import splice, synth

from gpu_util import alloc_outputs, assert_candidates_equal, oracle_grid, read_cands, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FS, T_OBS, N_BR = 1024.0, 1800.0, 5.0
F0, FDOT0 = 390.0, 0.2


def test_portions_find_and_connect_the_injection(built_lib, gpu_ctx):
    gfh = built_lib
    k = FDOT0 / F0 ** N_BR
    inj = synth.Injection(f0=F0, k=k, n=N_BR, amp=synth.amplitude_for_snr(6.0, 1.0, 2048))
    n_samples = int(FS * T_OBS)
    x = synth.strain_series(n_samples, FS, 21, (inj,))
    portions = gfh.tfft_portions(N_BR, 400.0, FDOT0, 2.0, T_OBS, 2)
    assert [float(p["t_fft"]) for p in portions] == [2.0, 4.0]
    plan = splice.portion_plan(portions, FS, n_samples, N_BR, [(250.0, 400.0)], 1, band_hz=10.0)
    x_dev = to_dev(torch, x)
    found = []
    for P in plan:
        f = dict(P.fields[0])
        g1 = oracle_grid(f)
        f["n_k"] = int(math.ceil(1.3 * k / g1.dk)) + 1          # k rows up to 1.3 k of the injection
        N = int(FS * P.t_fft)
        lo, hi = f["bin_lo"], f["bin_hi"]
        cap = 400000
        fo = torch.empty(cap, dtype=torch.int32, device="cuda")
        bo = torch.empty(cap, dtype=torch.int32, device="cuda")
        n_pk = gpu_ctx.peakmap(x_dev[P.s_begin:P.s_end], FS, P.t_fft, lo, hi, 2.5, fo, bo)
        assert (P.s_end - P.s_begin - N) // (N // 2) + 1 == f["n_fft"]
        fi, bj = fo[:n_pk].cpu().numpy().astype(np.uint32), bo[:n_pk].cpu().numpy().astype(np.uint32)
        ofi, _ = O.peakmap(x[P.s_begin:P.s_end], FS, P.t_fft, lo, hi)
        assert abs(len(fi) - len(ofi)) <= max(5, len(ofi) // 2000)
        g = gfh.grid_make(gfh.Grid(**f))
        hmap, cands, stats = alloc_outputs(torch, g)
        gpu_ctx.hough(fo[:n_pk], bo[:n_pk], n_pk, g, hmap, cands, stats)
        torch.cuda.synchronize()
        assert gpu_ctx.check() == gfh.GFH_OK
        o = oracle_grid(f)
        ref = O.hough_map(o, fi, bj)
        assert np.array_equal(hmap.cpu().numpy()[:, :g.n_x0], ref)
        oc, _ = O.select_candidates(o, ref)
        assert_candidates_equal(read_cands(gfh, cands), oc, g.n_bands)
        # the injection: top candidate of the band holding f0, within 3 bins of its (x0, k)
        band = int((F0 - 250.0) // 10.0)
        c = next(r for r in oc if r["band"] == band)
        dx = (c["x0"] - float(O.x_of_f(F0, N_BR))) / o.dx0
        dkr = (c["k"] - k) / o.dk
        assert math.hypot(dx, dkr) <= 3.0, (P.t_fft, dx, dkr)
        assert c["cr"] > 5.0
        found.append((g, cands, oc))
    (ga, ca, oa), (gb, cb, ob) = found
    match, dist = splice.coincide(gpu_ctx, ca, ga, cb, gb)
    torch.cuda.synchronize()
    m, d = match.cpu().numpy(), dist.cpu().numpy()
    # oracle coincidences on the same records
    ra, rb = read_cands(gfh, ca), read_cands(gfh, cb)
    va = [i for i in range(len(ra)) if ra["count"][i] >= 0]
    vb = [j for j in range(len(rb)) if rb["count"][j] >= 0]
    om, od = O.coincidences([dict(x0=float(ra["x0"][i]), k=float(ra["k"][i])) for i in va],
                            [dict(x0=float(rb["x0"][j]), k=float(rb["k"][j])) for j in vb],
                            max(ga.dx0, gb.dx0), max(ga.dk, gb.dk), 3.0)
    for t, i in enumerate(va):
        assert d[i] == od[t]
        assert m[i] == (vb[om[t]] if om[t] >= 0 else -1)
    band = int((F0 - 250.0) // 10.0)
    assert m[band] == band and d[band] <= 3.0
