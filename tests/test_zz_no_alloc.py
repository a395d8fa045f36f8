"""The allocation-free peak selection entry point (gfh_peaks_from_power_static).

It exists for callers that cannot allocate device memory - an application whose GPU memory is all
owned by another allocator, where a cudaMalloc inside the library could fail and where the implicit
device synchronisation of cudaMalloc/cudaFree would stall its other streams.  Its scratch is a
fixed device array inside the library, shared by every call, so these tests check that two calls
in a row (the second reusing what the first left behind) each give exactly the same peaks as the
regular entry point, and that a request too large for the array is refused.  The file is named to
be collected last.
"""
import numpy as np
import pytest

from gpu_util import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def regular(gfh, ctx, P, lo, hi, cap):
    fo = torch.empty(cap, dtype=torch.int32, device="cuda")
    bo = torch.empty(cap, dtype=torch.int32, device="cuda")
    n = ctx.peaks_from_power(P, lo, hi, 2.5, fo, bo)
    return fo[:n].cpu().numpy(), bo[:n].cpu().numpy()


def static(gfh, P, lo, hi, cap):
    fo = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    bo = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    n_dev = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    gfh.peaks_from_power_static(torch.cuda.current_stream(), P, lo, hi, 2.5, fo, bo, n_dev)
    torch.cuda.synchronize()
    n = int(n_dev.item())
    return fo[:n].cpu().numpy(), bo[:n].cpu().numpy()


def test_two_calls_in_a_row_match_the_regular_entry_point(built_lib, gpu_ctx):
    rng = np.random.default_rng(21)
    # a large request first, then a smaller one that reuses the same scratch
    cases = [(5040, 200, 1999, 4.0), (700, 300, 1100, 1.0)]
    for n_fft, lo, hi, scale in cases:
        P = to_dev(torch, (rng.exponential(size=(n_fft, hi + 40)) * scale).astype(np.float32))
        cap = n_fft * (hi - lo + 1) // 4
        ref = regular(built_lib, gpu_ctx, P, lo, hi, cap)
        got = static(built_lib, P, lo, hi, cap)
        assert len(got[0]) > 1000
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_request_beyond_the_static_scratch_is_refused(built_lib):
    P = torch.zeros((40000, 2100), dtype=torch.float32, device="cuda")
    fo = torch.empty(16, dtype=torch.int32, device="cuda")
    n_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(built_lib.GfhError) as e:
        built_lib.peaks_from_power_static(torch.cuda.current_stream(), P, 200, 2000, 2.5, fo, fo, n_dev)
    assert e.value.code == built_lib.GFH_ERR_SIZE


def scratch_bytes(n_fft, bins):
    """Scratch of one call: the 256-aligned peak bit matrix (one 32-bit word per 32 FFTs per bin)
    and bins + 1 int64 counts."""
    words = (n_fft + 31) // 32
    return (bins * words * 4 + 255) // 256 * 256 + (bins + 1) * 8


def test_the_documented_size_and_the_exact_limit(built_lib, gpu_ctx):
    """7800 bins x 5040 FFTs (the paper-shaped peakmap) fits and matches the regular entry point;
    with 7800 bins the largest fitting size is 266 words of 32 FFTs (8512 FFTs), which also
    matches, and one FFT more (a 267th word) is refused before anything is launched."""
    lo, bins = 130, 7800
    hi = lo + bins - 1
    assert scratch_bytes(8512, bins) <= built_lib.STATIC_SCRATCH_BYTES < scratch_bytes(8513, bins)
    rng = np.random.default_rng(5)
    for n_fft in (5040, 8512):
        P = to_dev(torch, rng.exponential(size=(n_fft, hi + 2)).astype(np.float32))
        cap = n_fft * bins // 10
        ref = regular(built_lib, gpu_ctx, P, lo, hi, cap)
        got = static(built_lib, P, lo, hi, cap)
        assert len(got[0]) > 100000
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        del P
    P = torch.zeros((8513, hi + 2), dtype=torch.float32, device="cuda")
    fo = torch.empty(16, dtype=torch.int32, device="cuda")
    n_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(built_lib.GfhError) as e:
        built_lib.peaks_from_power_static(torch.cuda.current_stream(), P, lo, hi, 2.5, fo, fo, n_dev)
    assert e.value.code == built_lib.GFH_ERR_SIZE


def test_more_peaks_than_capacity(built_lib, gpu_ctx):
    """With a capacity below the number of peaks, the count written is the total and the outputs
    hold the first `cap` peaks of the regular entry point's (bin, FFT) order; nothing past them is
    touched."""
    rng = np.random.default_rng(9)
    n_fft, lo, hi = 600, 200, 700
    P = to_dev(torch, rng.exponential(size=(n_fft, hi + 2)).astype(np.float32))
    ref = regular(built_lib, gpu_ctx, P, lo, hi, n_fft * (hi - lo + 1))
    cap = 1000
    assert len(ref[0]) > 5 * cap
    fo = torch.full((cap + 8,), -1, dtype=torch.int32, device="cuda")
    bo = torch.full((cap + 8,), -1, dtype=torch.int32, device="cuda")
    n_dev = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    built_lib.peaks_from_power_static(torch.cuda.current_stream(), P, lo, hi, 2.5, fo[:cap],
                                      bo[:cap], n_dev)
    torch.cuda.synchronize()
    assert int(n_dev.item()) == len(ref[0])
    f, b = fo.cpu().numpy(), bo.cpu().numpy()
    assert np.array_equal(f[:cap], ref[0][:cap]) and np.array_equal(b[:cap], ref[1][:cap])
    assert np.all(f[cap:] == -1) and np.all(b[cap:] == -1)
