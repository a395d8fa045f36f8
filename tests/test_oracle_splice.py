"""Pins of the Sec. VI.D portion planner (longer FFTs for later times): the family's spin-down bound
against a brute-force maximum over power laws of Eq. powlaws, the crossing times, Eq. dot_tfft and
the factor-4 rule at the portion edges; the C planner against the oracle (no GPU)."""
import numpy as np
import pytest

from oracle import gfh_oracle as O


def brute_max_spindown(t, n, f_hi, fdot_hi, nf=60, nd=3001):
    """max |fdot(t)| = k f(t)^n over a grid of members (f0, fdot0), f(t) from Eq. powlaws."""
    best = 0.0
    for f0 in np.linspace(f_hi / 4, f_hi, nf):
        fdot0 = np.linspace(0.0, fdot_hi, nd)[1:]
        k = fdot0 / f0 ** n
        f = O.powerlaw_f(t, f0, k, n)
        best = max(best, float(np.max(k * f ** n)))
    return best


@pytest.mark.parametrize("n,f_hi,fdot_hi", [(5.0, 400.0, 0.2), (2.5, 500.0, 1.0), (7.0, 1500.0, 0.06)])
def test_spindown_bound_is_the_family_maximum(n, f_hi, fdot_hi):
    for t in (0.0, 30.0, 0.7 * f_hi / fdot_hi, 2.0 * f_hi / fdot_hi, 9000.0):
        want = brute_max_spindown(t, n, f_hi, fdot_hi)
        got = float(O.max_spindown_at(t, n, f_hi, fdot_hi))
        assert got >= want * (1 - 1e-12)            # a bound
        assert got == pytest.approx(want, rel=2e-3)  # and attained (up to the grid)


@pytest.mark.parametrize("n,f_hi,fdot_hi", [(5.0, 400.0, 0.2), (2.5, 500.0, 1.0), (7.0, 1500.0, 0.06)])
def test_crossing_times(n, f_hi, fdot_hi):
    for fdot in (fdot_hi / 2, fdot_hi / 30, fdot_hi / 1000):
        t = O.time_of_spindown(fdot, n, f_hi, fdot_hi)
        assert float(O.max_spindown_at(t, n, f_hi, fdot_hi)) == pytest.approx(fdot, rel=1e-12)
        assert float(O.max_spindown_at(t * 0.999, n, f_hi, fdot_hi)) > fdot
    assert O.time_of_spindown(2 * fdot_hi, n, f_hi, fdot_hi) == 0.0


@pytest.mark.parametrize("n,f_hi,fdot_hi,t_fft0,t_obs,levels", [
    (5.0, 400.0, 0.2, 1.0, 1800.0, 4), (2.5, 500.0, 1.0, 1.0, 36000.0, 5),
    (7.0, 1500.0, 0.06, 2.0, 86400.0, 4), (5.0, 400.0, 0.2, 2.0, 100.0, 3)])
def test_portions_follow_eq_dot_tfft_and_the_factor_four(n, f_hi, fdot_hi, t_fft0, t_obs, levels):
    P = O.tfft_portions(n, f_hi, fdot_hi, t_fft0, t_obs, levels)
    assert P
    for (L, a, b, T) in P:
        assert T == t_fft0 * 2 ** L and 0.0 <= a < b <= t_obs and b - a >= T
        # Eq. dot_tfft: within the portion every member stays within one bin per FFT
        assert float(O.max_spindown_at(a, n, f_hi, fdot_hi)) <= 1.0 / T ** 2 * (1 + 1e-12)
    for (L0, a0, b0, T0), (L1, a1, b1, T1) in zip(P, P[1:]):
        assert b0 == a1 and T1 == 2 * T0                       # contiguous, doubling
        if a0 > 0.0:                                           # factor 4 between interior edges
            r = float(O.max_spindown_at(a0, n, f_hi, fdot_hi) / O.max_spindown_at(a1, n, f_hi, fdot_hi))
            assert r == pytest.approx(4.0, rel=1e-9)


def test_c_planner_equals_oracle(built_lib):
    gfh = built_lib
    for args in [(5.0, 400.0, 0.2, 1.0, 1800.0, 4), (2.5, 500.0, 1.0, 1.0, 36000.0, 5),
                 (7.0, 1500.0, 0.06, 2.0, 86400.0, 4), (3.3, 900.0, 5.0, 0.5, 5e5, 8)]:
        got = gfh.tfft_portions(*args)
        want = O.tfft_portions(*args)
        assert len(got) == len(want)
        for g, (L, a, b, T) in zip(got, want):
            assert int(g["level"]) == L and float(g["t_fft"]) == T
            assert float(g["t_begin"]) == pytest.approx(a, rel=1e-13, abs=1e-9)
            assert float(g["t_end"]) == pytest.approx(b, rel=1e-13, abs=1e-9)
    with pytest.raises(gfh.GfhError):
        gfh.tfft_portions(1.0, 400.0, 0.2, 1.0, 1800.0, 4)
    with pytest.raises(gfh.GfhError) as e:
        gfh.tfft_portions(2.5, 500.0, 1.0, 1.0, 36000.0, 5, cap=1)
    assert e.value.code == gfh.GFH_ERR_SIZE
