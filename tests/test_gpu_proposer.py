"""The exact Hough restricted to coarse tiles (the proposer's search) against the oracle's full map:
every computed cell exact, no other cell written, candidates the best computed cell per band."""
import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import proposer as PR
from paper_1810_09784_gb300 import synth

from gpu_util import oracle_grid, read_cands, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPEC = PR.ProposerSpec()


def coarse_mask(fields, g, ids, ck=64, cx=64):
    """Cells of coarse tiles `ids` as defined by gfh_plan_set_coarse (rows with floor(r ck / K) = kt;
    analysis columns of x0 tile xt, range widened to multiples of 4)."""
    o = oracle_grid(fields)
    f0c, _, band = O.column_bands(o)
    xt_col = np.clip(np.floor((f0c - fields["ana_lo"]) / (fields["ana_hi"] - fields["ana_lo"]) * cx),
                     0, cx - 1).astype(np.int64)
    mask = np.zeros((g.n_k, g.ld_x0), bool)
    kt_row = (np.arange(g.n_k) * ck) // g.n_k
    for cid in ids:
        if cid < 0 or cid >= ck * cx:
            continue
        kt, xt = divmod(int(cid), cx)
        cols = np.nonzero((band >= 0) & (xt_col == xt))[0]
        if cols.size == 0:
            continue
        c_lo, c_hi = cols.min() & ~3, min(g.ld_x0, (cols.max() + 4) & ~3)
        mask[np.ix_(kt_row == kt, np.arange(c_lo, c_hi))] = True
    return mask, band


def best_per_band(ref, mask, band, n_bands):
    """Highest count per band over masked analysis cells, ties to the lowest (row, column)."""
    out = {}
    W = ref.shape[1]
    for b in range(n_bands):
        cols = np.nonzero(band[:W] == b)[0]
        if cols.size == 0:
            continue
        sub = np.where(mask[:, cols], ref[:, cols], -1)
        if sub.max() < 0:
            out[b] = (-1, -1, -1)
            continue
        r, c = np.unravel_index(np.argmax(sub), sub.shape)   # row-major: lowest row, then column
        out[b] = (int(sub[r, c]), int(r), int(cols[c]))
    return out


def _peaks(sample, n):
    smp = PR.draw(SPEC, [sample])
    if not smp.signal[0]:
        return smp, synth.hashed_peaklist(SPEC.seed, sample, SPEC.n_fft, SPEC.bin_lo, SPEC.bin_hi,
                                          SPEC.p_noise24)
    return smp, synth.hashed_peaklist(SPEC.seed, sample, SPEC.n_fft, SPEC.bin_lo, SPEC.bin_hi,
                                      SPEC.p_noise24, int(smp.p_track24[0]), smp.tracks[0])


def test_all_tiles_equal_full_search(built_lib, gpu_ctx):
    gfh = built_lib
    fields = SPEC.grid_fields(5.0)
    g = gfh.grid_make(gfh.Grid(**fields))
    _, (fi, bj) = _peaks(3, 5.0)
    full = torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda")
    part = torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda")
    cf = torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda")
    cp = torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda")
    pf = gfh.Plan(gpu_ctx, [g], [full], [cf])
    pp = gfh.Plan(gpu_ctx, [g], [part], [cp], tile=(8, 1024, 256))
    pp.set_coarse(64, 64, 4096)
    f_d, b_d = to_dev(torch, fi), to_dev(torch, bj)
    off = to_dev(torch, np.array([0, fi.size], np.int64))
    pf.execute(f_d, b_d, off, 1)
    sel = torch.arange(4096, dtype=torch.int32, device="cuda").view(1, 4096)
    pp.execute_tiles(f_d, b_d, off, 1, sel, 4096)
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    o = oracle_grid(fields)
    _, _, band = O.column_bands(o)
    ana = np.nonzero(band >= 0)[0]
    a, b = full.cpu().numpy(), part.cpu().numpy()
    assert np.array_equal(a[:, ana], b[:, ana])
    ca, cb = read_cands(gfh, cf), read_cands(gfh, cp)
    for name in ("count", "row", "col", "f0", "k"):
        assert np.array_equal(ca[name], cb[name]), name


def test_selected_tiles_exact_and_nothing_else(built_lib, gpu_ctx):
    """Three braking indices in one plan, each with its own 32 tiles (some -1), against the
    oracle's full maps."""
    gfh = built_lib
    ns = [2.5, 4.0, 5.5]
    fields = [SPEC.grid_fields(n, i) for i, n in enumerate(ns)]
    gs = [gfh.grid_make(gfh.Grid(**f)) for f in fields]
    maps = [torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda") for g in gs]
    cands = [torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in gs]
    plan = gfh.Plan(gpu_ctx, gs, maps, cands, tile=(8, 2048, 512))
    plan.set_coarse(64, 64, 32)
    lists = [_peaks(s, n)[1] for s, n in zip((11, 12, 13), ns)]
    fi = np.concatenate([l[0] for l in lists])
    bj = np.concatenate([l[1] for l in lists])
    offs = np.cumsum([0] + [l[0].size for l in lists]).astype(np.int64)
    rng = np.random.default_rng(4)
    sel = np.stack([rng.choice(4096, 32, replace=False) for _ in ns]).astype(np.int32)
    sel[0, 5] = -1
    sel[1, :4] = [0, 63, 4032, 4095]                  # the four corners
    sel[2, 7] = 9999                                  # out of range: selects nothing
    plan.execute_tiles(to_dev(torch, fi), to_dev(torch, bj), to_dev(torch, offs), 3,
                       to_dev(torch, sel), 32)
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    for m, (f, g) in enumerate(zip(fields, gs)):
        o = oracle_grid(f)
        ref = O.hough_map(o, lists[m][0], lists[m][1])
        mask, band = coarse_mask(f, g, sel[m])
        got = maps[m].cpu().numpy()
        W = g.n_x0
        assert np.array_equal(got[:, :W][mask[:, :W]], ref[mask[:, :W]]), f["n"]
        assert np.all(got[:, :W][~mask[:, :W]] == -7)
        exp = best_per_band(ref, mask[:, :W], band, g.n_bands)
        c = read_cands(gfh, cands[m])
        for rec in c:
            want = exp.get(int(rec["band"]), (-1, -1, -1))
            assert (int(rec["count"]), int(rec["row"]), int(rec["col"])) == want, (f["n"], int(rec["band"]))


@pytest.mark.parametrize("fft_order", [True, False], ids=["fft-sorted", "fft-shuffled"])
def test_selected_tiles_high_rows_and_frequencies(built_lib, gpu_ctx, fft_order):
    """Coarse tiles at the high-f0 end and in the upper k rows, where a tile is a few columns wide
    and its bins' FFT shifts spread far wider: with each bin's peaks in FFT order the search walks
    only their FFT sub-ranges; with the FFTs shuffled inside each bin it walks every peak read.
    Every computed cell equals the oracle's full map, nothing else is written."""
    gfh = built_lib
    ns = [2.0, 4.0, 5.5]
    fields = [SPEC.grid_fields(n, i) for i, n in enumerate(ns)]
    gs = [gfh.grid_make(gfh.Grid(**f)) for f in fields]
    maps = [torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda") for g in gs]
    cands = [torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in gs]
    plan = gfh.Plan(gpu_ctx, gs, maps, cands, tile=(8, 3072, 512))
    plan.set_coarse(64, 64, 24)
    lists = [_peaks(s, n)[1] for s, n in zip((21, 22, 23), ns)]
    rng = np.random.default_rng(6)
    if not fft_order:
        shuffled = []
        for f, b in lists:
            key = rng.permutation(f.size)
            o = np.lexsort((key, b))            # bins ascending, FFTs in random order inside a bin
            shuffled.append((f[o], b[o]))
        lists = shuffled
    fi = np.concatenate([l[0] for l in lists])
    bj = np.concatenate([l[1] for l in lists])
    offs = np.cumsum([0] + [l[0].size for l in lists]).astype(np.int64)
    # 24 tiles per map: x0 tiles 40-63, k tiles 32-63 (and two at the top corner)
    sel = np.stack([rng.choice([kt * 64 + xt for kt in range(32, 64) for xt in range(40, 64)], 24,
                               replace=False) for _ in ns]).astype(np.int32)
    sel[:, 0] = 63 * 64 + 63
    sel[:, 1] = 62 * 64 + 63
    plan.execute_tiles(to_dev(torch, fi), to_dev(torch, bj), to_dev(torch, offs), 3,
                       to_dev(torch, sel), 24)
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    for m, (f, g) in enumerate(zip(fields, gs)):
        ref = O.hough_map(oracle_grid(f), lists[m][0], lists[m][1])
        mask, _ = coarse_mask(f, g, sel[m])
        got = maps[m].cpu().numpy()
        W = g.n_x0
        assert np.array_equal(got[:, :W][mask[:, :W]], ref[mask[:, :W]]), f["n"]
        assert np.all(got[:, :W][~mask[:, :W]] == -7)
    plan.close()


def test_autotune_keeps_coarse_tiles(built_lib, gpu_ctx):
    gfh = built_lib
    fields = SPEC.grid_fields(3.0)
    g = gfh.grid_make(gfh.Grid(**fields))
    _, (fi, bj) = _peaks(21, 3.0)
    hm = torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda")
    c = torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda")
    plan = gfh.Plan(gpu_ctx, [g], [hm], [c])
    plan.set_coarse(64, 64, 8)
    f_d, b_d = to_dev(torch, fi), to_dev(torch, bj)
    off = to_dev(torch, np.array([0, fi.size], np.int64))
    plan.autotune(f_d, b_d, off, 1, reps=1)
    hm.fill_(-7)
    sel = to_dev(torch, np.array([[5, 700, 1400, 2100, 2800, 3500, 4000, 64 * 10 + 40]], np.int32))
    plan.execute_tiles(f_d, b_d, off, 1, sel, 8)
    torch.cuda.synchronize()
    ref = O.hough_map(oracle_grid(fields), fi, bj)
    mask, _ = coarse_mask(fields, g, sel.cpu().numpy()[0])
    got = hm.cpu().numpy()[:, :g.n_x0]
    assert np.array_equal(got[mask[:, :g.n_x0]], ref[mask[:, :g.n_x0]])
    assert np.all(got[~mask[:, :g.n_x0]] == -7)


def _work(summ):
    """Coarse tiles searched per map, a full search counting all 4096."""
    f = summ["fallback_frac"]
    return f * 4096 + (1 - f) * summ["mean_tiles_pruned"]


def test_trained_network_gains_over_the_search_without_it(built_lib, gpu_ctx):
    """A short training run (51,200 maps whose peakmaps the library builds from seeded strain
    series, trained by its own forward/backward/AdamW kernels) against the same network untrained
    and against the non-learned line-sum ranker, all judged by the full exact Hough on the same 408
    held-out series maps at the same threshold: untrained, the proposals never reach the threshold
    and every map falls back to the full search; trained, most maps are searched on at most 32
    coarse tiles and the detections of the full search are kept; the line ranker's work and
    recall on the same maps are printed beside it."""
    gfh = built_lib
    bank = PR.HoughBank(gpu_ctx, SPEC, max_sel=32)
    untrained = gfh.Cnn(gpu_ctx, 256, seed=1)
    s0 = PR.summarize(PR.evaluate(gpu_ctx, untrained, SPEC, 100011, 51 * 8, bank, 0.1))
    untrained.close()
    net = gfh.Cnn(gpu_ctx, 256, seed=1)
    losses = PR.train(gpu_ctx, net, SPEC, 0, 51200, batch=256, lr=2e-3)
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:5])
    s1 = PR.summarize(PR.evaluate(gpu_ctx, net, SPEC, 100011, 51 * 8, bank, 0.1))
    heur = PR.calibrate_heuristic(gpu_ctx, SPEC, 60000, 2048)
    s2 = PR.summarize(PR.evaluate(gpu_ctx, heur, SPEC, 100011, 51 * 8, bank, 0.1))
    print("untrained", s0)
    print("trained", s1, "work", _work(s1))
    print("line heuristic", (heur.beta, heur.det_a, heur.det_b), s2, "work", _work(s2))
    assert s0["fallback_frac"] >= 0.95 and s0["recall"] == 1.0
    assert s1["fallback_frac"] <= 0.6 and s1["mean_tiles_pruned"] <= 32
    assert s1["recall"] >= 0.95
    assert s2["det_full"] == s1["det_full"]            # the same maps, the same full search
    net.close()
    bank.plan.close()


def test_line_scores_against_the_oracle(built_lib, gpu_ctx):
    """gfh_line_scores on images of series peakmaps: the line sums equal the oracle's exactly (the
    fp32 sums of bf16 pixels are exact), the logits within fp32 rounding of the standardisation."""
    from oracle import cnn_oracle as C
    gfh = built_lib
    smp = PR.draw(SPEC, np.arange(500, 504))
    buf = PR.DeviceBatch(SPEC, 4)
    buf.load(gpu_ctx, SPEC, smp)
    scores = torch.empty((4, 4096), dtype=torch.float32, device="cuda")
    logits = torch.empty((4, gfh.N_CLASSES), dtype=torch.float32, device="cuda")
    nb = SPEC.bin_hi - SPEC.bin_lo + 1
    gfh.line_scores(gpu_ctx, buf.images, SPEC.n_k, nb, 2.0, 0.5, 3.0, logits, scores)
    torch.cuda.synchronize()
    img = C.bf16_value(buf.images.view(torch.int16).cpu().numpy().view(np.uint16))
    sc, lg = scores.cpu().numpy(), logits.cpu().numpy()
    for b in range(4):
        ref = C.line_scores(img[b, :, :, 0], SPEC.n_k, nb)
        assert np.array_equal(sc[b].astype(np.float64), ref), b
        lref = C.heuristic_logits(ref, 2.0, 0.5, 3.0)
        assert np.all(np.abs(lg[b] - lref) <= 1e-4 * (1.0 + np.abs(lref))), b


def test_series_peakmaps_hold_the_injected_track(built_lib, gpu_ctx):
    """The series recipe on the device: a noise-only sample gives the peak density of an equalised
    exponential spectrum (p0 within 3 %), and a strong injection (SNR 8) leaves a peak within one
    bin of its Eq. powlaws track in most FFTs, where noise alone would put one in about 20 %."""
    import dataclasses
    spec = dataclasses.replace(SPEC, snr_lo=8.0, snr_hi=8.0)
    src = PR.PeakSource(gpu_ctx, spec, 8)
    smp = PR.draw(spec, np.arange(0, 8))
    src.load(smp)
    fi = src.fft_c.cpu().numpy().astype(np.int64)
    bj = src.bin_c.cpu().numpy().astype(np.int64)
    nb = spec.bin_hi - spec.bin_lo + 1
    checked = 0
    for b in range(8):
        lo, hi = src.offs_host[b], src.offs_host[b + 1]
        f, j = fi[lo:hi], bj[lo:hi]
        assert np.all(np.diff(j * spec.n_fft + f) > 0)            # sorted by (bin, FFT), unique
        if not smp.signal[b]:
            dens = (hi - lo) / (spec.n_fft * nb)
            assert abs(dens / spec.p_noise - 1) < 0.03, dens
            continue
        tr = smp.tracks[b]
        cells = set((j * spec.n_fft + f).tolist())
        ok = [i for i in range(spec.n_fft) if tr[i] >= spec.bin_lo + 1 and tr[i] <= spec.bin_hi - 1]
        hit = sum(any((tr[i] + d) * spec.n_fft + i in cells for d in (-1, 0, 1)) for i in ok)
        assert hit >= 0.7 * len(ok), (b, hit, len(ok))
        checked += 1
    assert checked >= 2


def test_pruned_search_with_full_flags(built_lib, gpu_ctx):
    """Maps flagged for the full search inside execute_tiles equal gfh_plan_execute exactly (map
    and candidates); the other maps keep their selected tiles only."""
    gfh = built_lib
    ns = [3.0, 5.0]
    fields = [SPEC.grid_fields(n, i) for i, n in enumerate(ns)]
    gs = [gfh.grid_make(gfh.Grid(**f)) for f in fields]
    maps = [torch.full((g.n_k, g.ld_x0), -7, dtype=torch.int32, device="cuda") for g in gs]
    cands = [torch.zeros(g.n_bands * 64, dtype=torch.uint8, device="cuda") for g in gs]
    plan = gfh.Plan(gpu_ctx, gs, maps, cands)
    plan.set_coarse(64, 64, 16)
    lists = [_peaks(s, n)[1] for s, n in zip((31, 32), ns)]
    fi = to_dev(torch, np.concatenate([l[0] for l in lists]))
    bj = to_dev(torch, np.concatenate([l[1] for l in lists]))
    offs = to_dev(torch, np.cumsum([0] + [l[0].size for l in lists]).astype(np.int64))
    sel = np.full((2, 16), -1, np.int32)
    sel[0, :3] = [100, 2000, 4000]
    sel[1, :5] = [1, 2, 3, 64 * 30 + 20, 64 * 63 + 63]
    full = to_dev(torch, np.array([0, 1], np.int32))
    plan.execute_tiles(fi, bj, offs, 2, to_dev(torch, sel), 16, full)
    torch.cuda.synchronize()
    assert gpu_ctx.check() == gfh.GFH_OK
    ref0 = O.hough_map(oracle_grid(fields[0]), *lists[0])
    mask, band = coarse_mask(fields[0], gs[0], sel[0])
    got0 = maps[0].cpu().numpy()[:, :gs[0].n_x0]
    assert np.array_equal(got0[mask[:, :gs[0].n_x0]], ref0[mask[:, :gs[0].n_x0]])
    assert np.all(got0[~mask[:, :gs[0].n_x0]] == -7)
    o1 = oracle_grid(fields[1])
    ref1 = O.hough_map(o1, *lists[1])
    assert np.array_equal(maps[1].cpu().numpy()[:, :gs[1].n_x0], ref1)
    oc, _ = O.select_candidates(o1, ref1)
    c1 = read_cands(gfh, cands[1])
    by_band = {c["band"]: c for c in oc}
    for rec in c1:
        want = by_band.get(int(rec["band"]))
        if want is None:
            assert rec["count"] == -1
        else:
            assert (int(rec["count"]), int(rec["row"]), int(rec["col"])) == (want["count"], want["row"], want["col"])
    plan.close()
