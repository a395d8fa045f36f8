"""GPU parity of the follow-up stage (Sec. V) against the oracle, through the C ABI: the original
FrequencyHough maps (n = 0, both signs of fdot) bit-exact, the heterodyne within its derived phase
bound, the complex-series peakmap up to marginal decisions, the projection bit-exact, and the whole
chain on an injection followed up with parameters one grid step off."""
import math

import numpy as np
import pytest

from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth, workloads

from gpu_util import alloc_outputs, assert_candidates_equal, oracle_grid, read_cands, read_stats, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Heterodyne bound, relative to |h|: the phase is exact in fp64 at the anchors (~1e-9 cycle), the
# second..fourth-order terms (< 1/8 cycle) carry three float32 roundings (< 3 x 2^-24 / 8 = 2.3e-8
# cycle) and a 2^-34 step, the fraction is rounded to 2^-32 cycle, and the angle 2 pi x fraction
# (|angle| <= pi) is formed in float32 with two roundings (< 2 x 2^-24 x pi = 3.8e-7 rad): in all
# < 2 pi x 2.4e-8 + 3.8e-7 = 5.3e-7 rad.  The hardware sine and cosine are within 2^-21.41 =
# 3.7e-7 absolutely on [-pi, pi] (sqrt 2 x 3.7e-7 = 5.3e-7 on the complex factor) and the products
# h cos, h sin add one rounding each (2 x 6e-8): |dz| / |h| < 5.3e-7 + 5.3e-7 + 1.2e-7 = 1.2e-6.
# Taken with a factor two.
HET_TOL = 2.4e-6


def run_plan(gfh, ctx, fields, fi, bj, tile):
    g = gfh.grid_make(gfh.Grid(**fields))
    hmap, cands, stats = alloc_outputs(torch, g)
    off = to_dev(torch, np.array([0, len(fi)], np.int64))
    plan = gfh.Plan(ctx, [g], [hmap], [cands], stats, tile=tile)
    plan.execute(to_dev(torch, fi.astype(np.uint32)), to_dev(torch, bj.astype(np.uint32)), off, 1)
    torch.cuda.synchronize()
    plan.close()
    assert ctx.check() == gfh.GFH_OK
    return g, hmap.cpu().numpy(), read_cands(gfh, cands), read_stats(gfh, stats)


@pytest.mark.parametrize("k_rows_below", [0, 20, 48])
@pytest.mark.parametrize("tile", [(8, 128, 256), (16, 3072, 512)], ids=str)
def test_original_fh_maps_match_oracle(built_lib, gpu_ctx, k_rows_below, tile):
    """n = 0 maps over the plain_small peak statistics (600 bins, 1799 FFTs), 64 fdot rows of which
    k_rows_below are spin-up, across several tiles with a ragged last tile: every cell and every
    candidate equal to the oracle."""
    gfh = built_lib
    _, _, grids = workloads.plain_small()
    dk = 0.5 / 1800.0
    fields = dict(grids[0], n=0.0, n_k=64, k_min=-k_rows_below * dk, dk=dk, band_hz=3.0)
    fi, bj = synth.random_peaklist(1799, 198, 801, 0.0755, 17 + k_rows_below)
    g, hm, cands, stats = run_plan(gfh, gpu_ctx, fields, fi, bj, tile)
    o = oracle_grid(fields)
    assert (g.n_x0, g.dx0, g.x0_min) == (o.n_x0, o.dx0, o.x0_min)
    ref = O.hough_map(o, fi, bj)
    assert np.array_equal(hm[:, :g.n_x0], ref)
    oc, (s1, s2, cells) = O.select_candidates(o, ref)
    assert (int(stats["sum"][0]), int(stats["sum_sq"][0]), int(stats["cells"][0])) == (s1, s2, cells)
    assert_candidates_equal(cands, oc, g.n_bands)


def assert_heterodyne_close(got, h, want):
    err = np.abs(got.astype(np.complex128) - want)
    bad = err > HET_TOL * np.abs(h) + 1e-30
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:3], err[bad][:3])


@pytest.mark.parametrize("n,f0,fdot0,t_start,n_samples", [
    (5.0, 300.0, 0.04, 0.0, 1024 * 37 + 13), (2.0, 812.5, 0.9, 3.0, 4096 * 9 + 1),
    (7.0, 95.3, 0.002, 1234.5, 1024 * 64), (2.5, 1500.0, 0.0625, 17.0, 5000),
    (3.0, 440.0, 0.0, 0.0, 3001)])
def test_heterodyne_matches_oracle(built_lib, gpu_ctx, n, f0, fdot0, t_start, n_samples):
    gfh = built_lib
    rng = np.random.default_rng(int(f0))
    fs = 4096.0
    h = rng.standard_normal(n_samples).astype(np.float32)
    k = O.k_from_spindown(f0, fdot0, n)
    dh = to_dev(torch, h)
    out = torch.empty(2 * n_samples, dtype=torch.float32, device="cuda")
    gpu_ctx.heterodyne(dh, fs, t_start, f0, k, n, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.complex64)
    want = O.heterodyne(h, fs, t_start, f0, k, n)
    assert_heterodyne_close(got, h, want)
    # a pointer off the 16-byte lattice takes the sample-by-sample path: same values
    out2 = torch.empty(2 * n_samples, dtype=torch.float32, device="cuda")
    gpu_ctx.heterodyne(dh[1:], fs, t_start + 1.0 / fs, f0, k, n, out2[2:])
    torch.cuda.synchronize()
    got2 = out2[2:].cpu().numpy().view(np.complex64)
    assert_heterodyne_close(got2, h[1:], O.heterodyne(h[1:], fs, t_start + 1.0 / fs, f0, k, n))


def test_heterodyne_full_size_sampled(built_lib, gpu_ctx):
    """The 10080 s, 4096 Hz series (41.3M samples) corrected by its first injection, checked against
    the oracle sample by sample at 20000 seeded positions (and both ends)."""
    gfh = built_lib
    spec, _, _ = workloads.plain_paper()
    inj = spec.injections[0]
    h = spec.series()
    dh = to_dev(torch, h)
    out = torch.empty(2 * h.size, dtype=torch.float32, device="cuda")
    gpu_ctx.heterodyne(dh, spec.fs, 0.0, inj.f0, inj.k, inj.n, out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    idx = np.unique(np.concatenate([rng.integers(0, h.size, 20000), [0, 1, h.size - 1]]))
    got = out.view(torch.complex64)[torch.from_numpy(idx).cuda()].cpu().numpy()
    t = idx.astype(np.float64) / spec.fs
    want = h[idx].astype(np.float64) * np.exp(-2j * np.pi * O.spindown_cycles(t, inj.f0, inj.k, inj.n))
    assert_heterodyne_close(got, h[idx], want)


def test_heterodyne_rejects_too_fast_a_spindown(built_lib, gpu_ctx):
    gfh = built_lib
    h = torch.zeros(4096, dtype=torch.float32, device="cuda")
    out = torch.empty(8192, dtype=torch.float32, device="cuda")
    k = O.k_from_spindown(100.0, 50.0, 5.0)            # 50 Hz/s: > 1/8 cycle of curvature per anchor
    with pytest.raises(gfh.GfhError) as e:
        gpu_ctx.heterodyne(h, 4096.0, 0.0, 100.0, k, 5.0, out)
    assert e.value.code == gfh.GFH_ERR_ARG


def marginal(R, fi, bj, bin_lo, tol=2e-4):
    c = bj.astype(np.int64) - bin_lo + 1
    r = R[fi, c]
    return ((np.abs(r - 2.5) < tol * 2.5) | (np.abs(r - R[fi, c - 1]) < tol * r)
            | (np.abs(r - R[fi, c + 1]) < tol * r))


def gpu_peakmap_complex(gfh, ctx, z64, fs, t_fft, lo, hi, cap):
    fo = torch.empty(cap, dtype=torch.int32, device="cuda")
    bo = torch.empty(cap, dtype=torch.int32, device="cuda")
    dz = to_dev(torch, z64.view(np.float32))
    n = ctx.peakmap_complex(dz, fs, t_fft, lo, hi, 2.5, fo, bo)
    return fo[:n].cpu().numpy().astype(np.int64), bo[:n].cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("band", [(1380, 1420), (700, 1500)])
def test_complex_peakmap_matches_oracle(built_lib, gpu_ctx, band):
    """plain_small's series corrected by its injection, FFTs of 4 s (twice the search's): peaks equal
    to the oracle's (fp64 FFT of the same complex64 samples) up to decisions within rounding of a
    tie or the threshold."""
    gfh = built_lib
    spec, _, _ = workloads.plain_small()
    inj = spec.injections[0]
    z64 = O.heterodyne(spec.series(), spec.fs, 0.0, inj.f0, inj.k, inj.n).astype(np.complex64)
    lo, hi = band
    t_fft = 4.0
    P = O.complex_power_spectra(z64, spec.fs, t_fft)
    R = O.equalise(P, lo, hi)
    ofi, obj = O.peaks_from_power(P, lo, hi)
    fi, bj = gpu_peakmap_complex(gfh, gpu_ctx, z64, spec.fs, t_fft, lo, hi, 2 * len(ofi) + 16)
    n_fft = P.shape[0]
    key = bj * n_fft + fi
    okey = obj.astype(np.int64) * n_fft + ofi
    assert np.all(np.diff(key) > 0)
    diff = np.concatenate([np.setdiff1d(key, okey), np.setdiff1d(okey, key)])
    assert len(diff) <= max(5, len(okey) // 2000)
    if len(diff):
        assert np.all(marginal(R, diff % n_fft, diff // n_fft, lo))


def test_projection_bit_exact(built_lib, gpu_ctx):
    gfh = built_lib
    rng = np.random.default_rng(12)
    n_fft, lo, hi, df = 899, 1380, 1420, 0.25
    fi = rng.integers(0, n_fft, 50000).astype(np.uint32)
    bj = rng.integers(lo - 30, hi + 30, 50000).astype(np.uint32)
    for fdot in (-0.0173, 0.0, 3.3e-4, -1e-3 / 3.0):
        counts = torch.full((hi - lo + 1,), -5, dtype=torch.int32, device="cuda")
        gpu_ctx.project_peaks(to_dev(torch, fi), to_dev(torch, bj), len(fi), 2.0, 2.0, df, fdot,
                              lo, hi, counts)
        torch.cuda.synchronize()
        want = O.project_peaks(fi, bj, 2.0, 2.0, df, fdot, lo, hi)
        assert np.array_equal(counts.cpu().numpy().astype(np.int64), want), fdot
    counts = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    gpu_ctx.project_peaks(None, None, 0, 2.0, 2.0, df, 0.0, lo, lo, counts)
    torch.cuda.synchronize()
    assert int(counts.item()) == 0


def test_follow_up_chain_recovers_the_injection(built_lib, gpu_ctx):
    """plain_small's injection (n = 5, f0 = 350 Hz, fdot0 = -0.043 Hz/s, spectral SNR 4) followed up
    from a candidate one k row and one x0 column off: every stage on the GPU equals the oracle on the
    same inputs, the residual line is the original FrequencyHough's strongest cell and its
    projection stands far above the noise bins."""
    gfh = built_lib
    spec, _, grids = workloads.plain_small()
    inj = spec.injections[0]
    g0 = oracle_grid(grids[0])
    # the candidate: one x0 column and one k row away from the injection
    x0 = float(O.x_of_f(inj.f0, inj.n)) + g0.dx0
    f0_c = float(O.f_of_x(x0, inj.n))
    k_c = inj.k + g0.dk
    h = spec.series()
    dh = to_dev(torch, h)
    z = torch.empty(2 * h.size, dtype=torch.float32, device="cuda")
    gpu_ctx.heterodyne(dh, spec.fs, 0.0, f0_c, k_c, inj.n, z)
    torch.cuda.synchronize()
    z64 = z.cpu().numpy().view(np.complex64)
    assert_heterodyne_close(z64[::997], h[::997], O.heterodyne(h, spec.fs, 0.0, f0_c, k_c, inj.n)[::997])
    t_fft = 2.0 * spec.t_fft
    (lo, hi), fields = workloads.followup_fields(
        type(inj)(f0=f0_c, k=k_c, n=inj.n, amp=inj.amp), spec.t_obs, t_fft)
    cap = 200000
    fo = torch.empty(cap, dtype=torch.int32, device="cuda")
    bo = torch.empty(cap, dtype=torch.int32, device="cuda")
    n_pk = gpu_ctx.peakmap_complex(z, spec.fs, t_fft, lo, hi, 2.5, fo, bo)
    fi, bj = fo[:n_pk].cpu().numpy().astype(np.uint32), bo[:n_pk].cpu().numpy().astype(np.uint32)
    ofi, obj = O.peakmap_complex(z64, spec.fs, t_fft, lo, hi)
    assert abs(len(fi) - len(ofi)) <= 5
    # original FrequencyHough on the GPU's peaks, against the oracle on the same peaks
    g = gfh.grid_make(gfh.Grid(**fields))
    hmap, cands, stats = alloc_outputs(torch, g)
    gpu_ctx.hough(fo[:n_pk], bo[:n_pk], n_pk, g, hmap, cands, stats)
    torch.cuda.synchronize()
    o = oracle_grid(fields)
    ref = O.hough_map(o, fi, bj)
    hm = hmap.cpu().numpy()[:, :g.n_x0]
    assert np.array_equal(hm, ref)
    oc, _ = O.select_candidates(o, ref)
    gc = read_cands(gfh, cands)
    assert_candidates_equal(gc, oc, g.n_bands)
    # the residual line is in nearly every FFT (the oracle chain gives 875 of 899, CR 7.1: the map
    # is 32 x 75 cells and the line's own strip widens sigma)
    best = max(oc, key=lambda c: c["count"])
    assert best["count"] >= 0.8 * fields["n_fft"] and best["cr"] > 5.0
    assert abs(best["f0"] - inj.f0) < 0.6         # within a few new bins of the true f0
    # projection with the residual spin-down: the line collects in one bin
    counts = torch.empty(hi - lo + 1, dtype=torch.int32, device="cuda")
    gpu_ctx.project_peaks(fo[:n_pk], bo[:n_pk], n_pk, fields["t_first"], fields["t_hop"],
                          fields["df"], best["fdot0"], lo, hi, counts)
    torch.cuda.synchronize()
    c = counts.cpu().numpy().astype(np.int64)
    want = O.project_peaks(fi, bj, fields["t_first"], fields["t_hop"], fields["df"], best["fdot0"], lo, hi)
    assert np.array_equal(c, want)
    # a fdot one row off the truth (ties go to the lowest row) may split the line over two bins:
    # the oracle chain gives 442 of 875 in the top bin, projection CR 6.4
    j = int(np.argmax(c))
    assert c[j] >= 0.4 * fields["n_fft"] and O.projection_cr(c, j) > 4.0
    assert abs((lo + j) * fields["df"] - best["f0"]) <= 2 * fields["df"]


# ---- the one-pass form: heterodyne + band spectra + peaks ------------------------------------------

# Peak decisions of the one-pass form may differ from an fp64 FFT only within its rounding: the
# heterodyne's 1.2e-6 relative per sample, float32 radix-2 stages (log2 N levels of 2^-24) and the
# 32-step twiddle recurrences (< 64 x 2^-24 = 3.8e-6 relative per term) bound |dX| by about
# 1e-5 sum|h| per frame, i.e. a relative error of the power below ~1e-3 at the threshold.
BAND_TOL = 1e-3


def band_case(spec, inj, t_fft, half=5.0):
    df = 1.0 / t_fft
    return int(math.floor((inj.f0 - half) / df)), int(math.ceil((inj.f0 + half) / df))


@pytest.mark.parametrize("dx,dkr", [(0, 0), (1, -1)])
def test_band_peaks_match_oracle(built_lib, gpu_ctx, dx, dkr):
    """plain_small's series corrected by its injection (or a candidate one x0 column and one k row
    off), 8 s frames: the one-pass peaks equal the oracle's (fp64 heterodyne and FFT) and the
    two-call GPU path's up to decisions within rounding of a tie or theta."""
    gfh = built_lib
    spec, _, grids = workloads.plain_small()
    inj = spec.injections[0]
    g0 = oracle_grid(grids[0])
    f0 = float(O.f_of_x(float(O.x_of_f(inj.f0, inj.n)) + dx * g0.dx0, inj.n))
    k = inj.k + dkr * g0.dk
    h = spec.series()
    t_fft = 8.0
    lo, hi = band_case(spec, inj, t_fft)
    dh = to_dev(torch, h)
    cap = 200000
    fo = torch.empty(cap, dtype=torch.int32, device="cuda")
    bo = torch.empty(cap, dtype=torch.int32, device="cuda")
    n1 = gpu_ctx.heterodyne_band_peaks(dh, spec.fs, 0.0, f0, k, inj.n, t_fft, lo, hi, 2.5, fo, bo)
    key1 = bo[:n1].cpu().numpy().astype(np.int64)
    f1 = fo[:n1].cpu().numpy().astype(np.int64)
    z = O.heterodyne(h, spec.fs, 0.0, f0, k, inj.n)
    P = O.complex_power_spectra(z, spec.fs, t_fft)
    R = O.equalise(P, lo, hi)
    ofi, obj = O.peaks_from_power(P, lo, hi)
    n_fft = P.shape[0]
    a = key1 * n_fft + f1
    b = obj.astype(np.int64) * n_fft + ofi
    assert np.all(np.diff(a) > 0) and len(b) > 1000
    diff = np.concatenate([np.setdiff1d(a, b), np.setdiff1d(b, a)])
    assert len(diff) <= max(5, len(b) // 1000)
    if len(diff):
        assert np.all(marginal(R, diff % n_fft, diff // n_fft, lo, tol=BAND_TOL))
    # the two-call GPU path on the same candidate
    zt = torch.empty(2 * h.size, dtype=torch.float32, device="cuda")
    gpu_ctx.heterodyne(dh, spec.fs, 0.0, f0, k, inj.n, zt)
    n2 = gpu_ctx.peakmap_complex(zt, spec.fs, t_fft, lo, hi, 2.5, fo, bo)
    c = bo[:n2].cpu().numpy().astype(np.int64) * n_fft + fo[:n2].cpu().numpy().astype(np.int64)
    diff2 = np.concatenate([np.setdiff1d(a, c), np.setdiff1d(c, a)])
    assert len(diff2) <= max(5, len(c) // 1000)
    if len(diff2):
        assert np.all(marginal(R, diff2 % n_fft, diff2 // n_fft, lo, tol=BAND_TOL))


def test_band_peaks_full_size_sampled_frames(built_lib, gpu_ctx):
    """The 41.3M-sample series and its fifth injection, 8 s frames (N = 32768): the peaks of four
    frames (first, two inner, last) equal the oracle's computed on those frames alone."""
    gfh = built_lib
    spec, _, _ = workloads.plain_paper()
    inj = spec.injections[4]
    h = spec.series()
    t_fft = 8.0
    lo, hi = band_case(spec, inj, t_fft)
    fo = torch.empty(400000, dtype=torch.int32, device="cuda")
    bo = torch.empty(400000, dtype=torch.int32, device="cuda")
    n1 = gpu_ctx.heterodyne_band_peaks(to_dev(torch, h), spec.fs, 0.0, inj.f0, inj.k, inj.n, t_fft,
                                       lo, hi, 2.5, fo, bo)
    fi = fo[:n1].cpu().numpy().astype(np.int64)
    bj = bo[:n1].cpu().numpy().astype(np.int64)
    N = int(spec.fs * t_fft)
    hop = N // 2
    n_fft = (h.size - N) // hop + 1
    for f in (0, 700, 1901, n_fft - 1):
        s0 = f * hop
        z = O.heterodyne(h[s0:s0 + N], spec.fs, s0 / spec.fs, inj.f0, inj.k, inj.n)
        P = O.complex_power_spectra(z, spec.fs, t_fft)
        R = O.equalise(P, lo, hi)
        _, obj = O.peaks_from_power(P, lo, hi)
        got = bj[fi == f]
        diff = np.concatenate([np.setdiff1d(got, obj), np.setdiff1d(obj.astype(np.int64), got)])
        assert len(diff) <= 2, (f, diff)
        if len(diff):
            assert np.all(marginal(R, np.zeros(len(diff), np.int64), diff, lo, tol=BAND_TOL)), f


def test_band_peaks_reject_unsupported_shapes(built_lib, gpu_ctx):
    gfh = built_lib
    h = torch.zeros(1 << 16, dtype=torch.float32, device="cuda")
    o = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(gfh.GfhError) as e:        # N = 4096 < 32 x 256
        gpu_ctx.heterodyne_band_peaks(h, 1024.0, 0.0, 300.0, 0.0, 5.0, 4.0, 1150, 1250, 2.5, o, o)
    assert e.value.code == gfh.GFH_ERR_SIZE
    with pytest.raises(gfh.GfhError) as e:        # N not a power of two
        gpu_ctx.heterodyne_band_peaks(h, 1000.0, 0.0, 300.0, 0.0, 5.0, 8.0, 2300, 2400, 2.5, o, o)
    assert e.value.code == gfh.GFH_ERR_ARG
