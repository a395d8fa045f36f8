"""Pins of the oracle's remaining helpers (no GPU): the bfloat16 rounding of the network oracle
against PyTorch's float32 -> bfloat16 conversion (round to nearest even) on ties, signs and
subnormals; the parameter layout's pack / unpack; the Sec. V bin shift on lines whose drift per
FFT is a known fraction of a bin; the complex-series peakmap of a real series against the real
series' peakmap."""
import numpy as np
import pytest

from oracle import cnn_oracle as C
from oracle import gfh_oracle as O
from paper_1810_09784_gb300 import synth

torch = pytest.importorskip("torch")


def test_bf16_rounding_is_round_to_nearest_even():
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.standard_normal(20000).astype(np.float32),
        (rng.standard_normal(2000) * 1e-39).astype(np.float32),         # subnormal float32
        (rng.standard_normal(2000) * 1e30).astype(np.float32),
        np.array([0.0, -0.0, 1.0, -1.0, 65504.0, 3.0e38], np.float32)])
    # exact ties: the low 16 bits 0x8000, with an even and an odd bfloat16 below
    base = rng.integers(0x00800000, 0x7F000000, size=4000, dtype=np.uint32) & np.uint32(0xFFFF0000)
    ties = (base | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = C.bf16_bits(x.astype(np.float64))
    assert np.array_equal(got, want)
    # and the value round trip
    assert np.array_equal(C.bf16(x.astype(np.float64)),
                          torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy())
    assert np.array_equal(C.to_f32(x.astype(np.float64)), x.astype(np.float64))


def test_parameter_layout_pack_unpack():
    off, total = C.layout()
    spans = sorted((o, o + int(np.prod(sh))) for o, sh in off.values())
    assert spans[0][0] == 0 and spans[-1][1] == total
    assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))          # contiguous, no overlap
    rng = np.random.default_rng(5)
    v = rng.standard_normal(total)
    parts = C.unpack(v)
    assert set(parts) == set(off)
    assert np.array_equal(C.pack(parts), v)


def test_bin_shift_on_known_drifts():
    df, t_hop = 0.25, 2.0
    i = np.arange(40)
    # one bin per FFT hop: shift = i (t_first = 0)
    assert np.array_equal(O.bin_shift(i, 0.0, t_hop, df, df / t_hop), i)
    # half a bin per hop: floor(i / 2 + 1/2)
    assert np.array_equal(O.bin_shift(i, 0.0, t_hop, df, 0.5 * df / t_hop), (i + 1) // 2)
    # spin-down: minus one bin per hop gives -i, minus half a bin per hop -(i // 2) (the exact
    # halves round up)
    assert np.array_equal(O.bin_shift(i, 0.0, t_hop, df, -df / t_hop), -i)
    assert np.array_equal(O.bin_shift(i, 0.0, t_hop, df, -0.5 * df / t_hop), -(i // 2))
    # away from exact halves the shift is odd in fdot
    up = O.bin_shift(i, 0.0, t_hop, df, 0.3 * df / t_hop)
    down = O.bin_shift(i, 0.0, t_hop, df, -0.3 * df / t_hop)
    away = np.abs((0.3 * i) % 1.0 - 0.5) > 1e-9
    assert np.array_equal(down[away], -up[away]) and up[-1] == 12
    # t_first shifts the time origin: FFT i at t_first = t_hop is FFT i + 1 at t_first = 0
    t_first = t_hop
    assert np.array_equal(O.bin_shift(i, t_first, t_hop, df, 0.3 * df / t_hop),
                          O.bin_shift(i + 1, 0.0, t_hop, df, 0.3 * df / t_hop))
    assert O.bin_shift(i, t_first, t_hop, df, 0.0).max() == 0


def test_complex_peakmap_of_a_real_series():
    fs, t_fft = 512.0, 2.0
    inj = synth.Injection(f0=120.0, k=0.0, n=5.0, amp=synth.amplitude_for_snr(6.0, 1.0, 1024))
    x = synth.strain_series(int(fs * 200), fs, 9, (inj,))
    lo, hi = 200, 300
    fr, br = O.peakmap(x, fs, t_fft, lo, hi)
    fc, bc = O.peakmap_complex(x.astype(np.complex128), fs, t_fft, lo, hi)
    real = set(zip(fr.tolist(), br.tolist()))
    cplx = set(zip(fc.tolist(), bc.tolist()))
    # the spectra agree to float32 rounding, so only decisions at a tie or at theta can differ
    assert len(real ^ cplx) <= max(1, len(real) // 2000)
    assert len(real) > 100
    # the injection's bin holds a peak in most FFTs in both
    for f, b in ((fr, br), (fc, bc)):
        assert np.sum(b == 240) > 0.8 * (f.max() + 1)
