"""The SRUR radar cubes of §VI (eq. (r_i), eq. (s_u), Table III, Table IV), pinned by the
system's own physics rather than by restating the generator: the range-bin spacing against
the Table III bandwidth, the unambiguous range and velocity the section states, the array's
half-wavelength angle mapping, the axis and sign conventions through a dense 3-D FFT of
noise-free bursts, and the Swerling-I amplitude statistics."""
import math

import numpy as np
import pytest

import rsft_inputs as ri

SYS = ri.SrurSystem()


def _freq(**kw):
    base = dict(range_m=100.0, velocity=0.0, doa_deg=0.0, snr_db=0.0)
    base.update(kw)
    return ri.srur_frequencies(SYS, [ri.SrurTarget(**base)])[0]


def test_range_bin_is_the_bandwidth_resolution():
    # one range bin of the R-sample de-chirped sweep is c / (2 B) with B the swept bandwidth;
    # Table III lists B_w = 150 MHz, and R / f_s x rho sweeps 149.85 MHz of it
    bins_per_m = (_freq(range_m=801.0)[0] - _freq(range_m=800.0)[0]) * SYS.range_bins
    assert bins_per_m == pytest.approx(2.0 * SYS.bandwidth / SYS.c, rel=2e-3)


def test_stated_unambiguous_range_and_velocity():
    # §VI-C: measurements are unambiguous below 1.5 km and 300 m/s
    assert 0.0 < _freq(range_m=SYS.r_max * 0.999)[0] < 1.0
    assert _freq(range_m=SYS.r_max * 0.999)[0] > _freq(range_m=1000.0)[0]
    assert 0.0 < _freq(velocity=299.0)[2] < 1.0
    assert _freq(velocity=299.0)[2] > _freq(velocity=240.0)[2]


def test_half_wavelength_array_angle_mapping():
    assert _freq(doa_deg=0.0)[1] == 0.0                       # broadside: no phase step
    assert _freq(doa_deg=90.0)[1] == pytest.approx(0.5)       # endfire: the array's Nyquist
    assert _freq(doa_deg=-30.0)[1] == pytest.approx(1.0 - _freq(doa_deg=30.0)[1])
    # targets 3 and 4 of Table IV, 4 degrees apart: about two angle bins of the 64-element array
    f3, f4 = ri.srur_frequencies(SYS, ri.TABLE_IV["equal"][2:4])
    assert 1.5 < (f3[1] - f4[1]) * SYS.elements < 3.0


@pytest.mark.parametrize("k", range(4))
def test_dense_fft_peak_at_each_table_iv_target(k):
    tgt = ri.TABLE_IV["equal"][k]
    cubes, freqs, amps = ri.srur_bursts(SYS, [tgt], 1, seed=3, amplitudes=np.array([[1.5 - 0.5j]]), noise_var=0.0)
    spec = np.abs(np.fft.fftn(cubes[0].astype(np.complex128)))
    peak = np.unravel_index(int(np.argmax(spec)), SYS.shape)
    n = np.asarray(SYS.shape)
    expect = np.floor(freqs[0] * n).astype(int)   # the peak is one of the two bins around f N
    assert all(p in (e % nd, (e + 1) % nd) for p, e, nd in zip(peak, expect, n)), (peak, freqs[0] * n)
    nearest = np.rint(freqs[0] * n).astype(int) % n
    far = [abs(f * nd - round(f * nd)) < 0.4 for f, nd in zip(freqs[0], n)]
    assert all(p == q for p, q, ok in zip(peak, nearest, far) if ok), (peak, nearest)


def test_amplitude_static_within_a_burst():
    tgt = ri.TABLE_IV["mixed"][0]
    cubes, freqs, amps = ri.srur_bursts(SYS, [tgt], 2, seed=5, noise_var=0.0)
    for s in range(2):
        x = cubes[s]
        i = [np.array([0, 7, 2047]), np.array([0, 33, 63]), np.array([0, 5, 31])]
        phase = np.exp(2j * np.pi * sum(freqs[0][d] * i[d] for d in range(3)))
        np.testing.assert_allclose(x[i[0], i[1], i[2]], amps[s, 0] * phase, rtol=2e-6, atol=2e-6 * abs(amps[s, 0]))
    assert abs(amps[0, 0] - amps[1, 0]) > 0


def test_swerling_one_amplitude_statistics():
    tg = ri.TABLE_IV["mixed"]
    a = ri.srur_amplitudes(tg, 4000, seed=9)
    s2 = 10.0 ** (np.array([t.snr_db for t in tg]) / 10.0)
    p = np.abs(a) ** 2 / s2
    # |a|^2 / s2 is exponential with mean 1: mean, variance, and the median at ln 2
    np.testing.assert_allclose(p.mean(axis=0), 1.0, atol=0.06)
    np.testing.assert_allclose(p.var(axis=0), 1.0, atol=0.15)
    np.testing.assert_allclose(np.median(p, axis=0), math.log(2.0), atol=0.05)
    # uniform phase: the mean of a / |a| vanishes; bursts are independent (lag-1 correlation)
    u = a / np.abs(a)
    assert np.all(np.abs(u.mean(axis=0)) < 0.05)
    c = np.abs(np.mean(u[1:] * np.conj(u[:-1]), axis=0))
    assert np.all(c < 0.05)


def test_noise_is_unit_circular_gaussian():
    cubes, _, _ = ri.srur_bursts(SYS, ri.TABLE_IV["equal"], 1, seed=4, amplitudes=np.zeros((1, 4)))
    x = cubes[0].astype(np.complex128).ravel()
    assert np.mean(np.abs(x) ** 2) == pytest.approx(1.0, rel=5e-3)
    assert abs(np.mean(x.real ** 2) - np.mean(x.imag ** 2)) < 5e-3
    assert abs(np.mean(x)) < 2e-3


def test_oracle_locates_the_table_iv_targets_in_segment_mode():
    """The radar scene end to end through the FP64 oracle (one burst per loop, 8 bursts,
    B = 64 x 16 x 8, 60 dB Chebyshev, P_fa = 1e-6): every Table IV target, including the pair
    4 degrees apart, has a located cell within one bin, as §VI reports for the RSFT."""
    import oracle as O
    cubes, freqs, _ = ri.srur_bursts(SYS, ri.TABLE_IV["mixed"], 8, seed=4001)
    op = O.make_plan(SYS.shape, (64, 16, 8), 8, seed=4001, atten_db=60.0, p_fa=1e-6, k_max=4, noise_var=1.0)
    out = O.rsft(op, [c.astype(np.complex128) for c in cubes], estimate=False)
    n = np.asarray(SYS.shape)
    idx = np.stack(np.unravel_index(out["located"], SYS.shape), axis=1)
    for f in freqs:
        d = np.abs(idx - np.rint(f * n).astype(int) % n)
        assert np.any(np.all(np.minimum(d, n - d) <= 1, axis=1)), f * n
