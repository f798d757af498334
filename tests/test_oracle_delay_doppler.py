"""Pins of the delay-Doppler focusing restatement (Section IV.C): point targets land in
their beam and, after the range-migration correction, at the nadir gate; the centroid
correction moves the nadir echo to the zero-Doppler beam; focusing preserves energy."""
import dataclasses
import math

import numpy as np
import pytest

import scenegen as sg
from oracle import delay_doppler as dd

H = 800e3


def _radar(G=32):
    return sg.RadarParams(n_gates=G)


def test_point_target_focuses_to_its_beam_and_the_corrected_gate():
    """A target at along-track offset x_f of beam f0 has phase advance nu_f0 per pulse and a
    range excess of s gates; choose the speed so that s = 3 exactly: its energy lands in beam
    f0 at gate g1 - 3, with amplitude N_b (unnormalised along-track DFT)."""
    rd = _radar()
    Nb, f0, g1, s = 16, 11, 20, 3
    lam = rd.c_mps / rd.carrier_hz
    nu = (f0 - Nb // 2) / Nb
    x = math.sqrt(2.0 * H * rd.gate_width_m * s)
    vh = nu * lam * H * rd.prf_hz / (2.0 * x)
    pf = sg.PlatformParams(p0=(0.0, 0.0, H), v=(vh, 0.0, 0.0), r_ref0=H, r_ref_rate=0.0)
    assert dd.migration_gates(rd, pf, Nb, H)[f0] == pytest.approx(s, rel=1e-12)
    k = np.arange(Nb)
    iq = np.zeros((Nb, rd.n_gates), complex)
    iq[:, g1] = 0.7 * np.exp(2j * np.pi * nu * k + 0.4j)
    Y, W = dd.focus(rd, pf, iq, 0, Nb)
    expect = np.zeros((Nb, rd.n_gates), complex)
    expect[f0, g1 - s] = 0.7 * Nb * np.exp(0.4j)
    np.testing.assert_allclose(Y[0], expect, atol=1e-11)
    assert W[0, g1 - s] == pytest.approx((0.7 * Nb) ** 2 / Nb, rel=1e-12)
    assert W[0].sum() == pytest.approx(W[0, g1 - s], rel=1e-12)


def test_integer_shift_is_a_roll_and_fractional_shift_interpolates():
    rd = _radar(64)
    Nb = 8
    rng = np.random.Generator(np.random.PCG64(2))
    iq = rng.standard_normal((Nb, rd.n_gates)) + 1j * rng.standard_normal((Nb, rd.n_gates))
    pf = sg.PlatformParams(p0=(0.0, 0.0, H), v=(0.0, 0.0, 0.0), r_ref0=H, r_ref_rate=0.0)
    Y0, _ = dd.focus(rd, pf, iq, 0, Nb)                 # no motion: no migration
    B = np.fft.fftshift(np.fft.fft(iq, axis=0), axes=0)
    np.testing.assert_allclose(Y0[0], B, atol=1e-10)
    # a beam shifted by an integer s equals np.roll(B_f, -s)
    lam = rd.c_mps / rd.carrier_hz
    f0, s = 6, 5
    nu = (f0 - Nb // 2) / Nb
    vh = nu * lam * H * rd.prf_hz / (2.0 * math.sqrt(2.0 * H * rd.gate_width_m * s))
    pf = dataclasses.replace(pf, v=(vh, 0.0, 0.0))
    Y, _ = dd.focus(rd, pf, iq, 0, Nb)
    np.testing.assert_allclose(Y[0, f0], np.roll(B[f0], -s), atol=1e-10)


def test_centroid_correction_moves_the_nadir_echo_to_zero_doppler():
    rd = _radar()
    Nb = 32
    pf = sg.PlatformParams(p0=(0.0, 0.0, H), v=(0.0, 0.0, 3.0), r_ref0=H, r_ref_rate=0.0)
    nu_c = dd.centroid(rd, pf)
    lam = rd.c_mps / rd.carrier_hz
    assert nu_c == pytest.approx(-2 * 3.0 / (lam * rd.prf_hz), rel=1e-15)
    k = np.arange(Nb)
    iq = np.zeros((Nb, rd.n_gates), complex)
    iq[:, 9] = np.exp(2j * np.pi * nu_c * k)            # the nadir echo: range grows at V_z
    Y, _ = dd.focus(rd, pf, iq, 0, Nb)
    assert np.abs(Y[0, Nb // 2, 9]) == pytest.approx(Nb, rel=1e-12)
    assert np.abs(Y[0]).sum() == pytest.approx(Nb, rel=1e-9)


def test_focusing_preserves_energy_and_migration_is_symmetric():
    rd = _radar(48)
    Nb = 64
    pf = sg.nadir_track(256)
    rng = np.random.Generator(np.random.PCG64(5))
    iq = rng.standard_normal((256, rd.n_gates)) + 1j * rng.standard_normal((256, rd.n_gates))
    Y, W = dd.focus(rd, pf, iq, 100, Nb)
    for b in range(4):
        e_in = (np.abs(iq[b * Nb:(b + 1) * Nb]) ** 2).sum()
        assert (np.abs(Y[b]) ** 2).sum() == pytest.approx(Nb * e_in, rel=1e-12)
        assert W[b].sum() == pytest.approx(e_in, rel=1e-12)
    s = dd.migration_gates(rd, pf, Nb, H)
    assert s[Nb // 2] == 0.0
    np.testing.assert_allclose(s[1:Nb // 2], s[Nb - 1:Nb // 2:-1], rtol=1e-14)
    # the outer beam (nu = -1/2) at 7 km/s from 800 km: x = lambda R PRF / (4 V)
    lam = rd.c_mps / rd.carrier_hz
    x = 0.5 * lam * H * rd.prf_hz / (2 * 7000.0)
    assert s[0] == pytest.approx(x * x / (2 * H * rd.gate_width_m), rel=1e-12)
