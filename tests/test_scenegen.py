"""The seeded input recipe (scenegen) against what it claims to generate.

The workloads stand in for the paper's Sentinel-3 SRAL scene (Section IV): a 1 m facet
grid, a linear deep-water swell of 100 m wavelength travelling along +x (the S1 swell of
Section IV.D), heights of 0.5 m standard deviation, lognormal NRCS, a nadir track at
800 km and 7 km/s.  These checks pin the generator to those statements and to the
kinematics of linear deep-water waves, so that a slip in the inputs (a wrong sign of the
orbital velocities, a misplaced spectral peak, a transposed grid) cannot pass unnoticed
into both sides of the parity tests.
"""
import math

import numpy as np
import pytest

import scenegen as sg


def test_grid_layout_and_determinism():
    L = 64
    a = sg.sea_surface(L, 5)
    ix, iy = np.meshgrid(np.arange(L), np.arange(L))            # n = iy * L + ix
    assert np.array_equal(a["x"], ((ix - (L - 1) / 2.0)).astype(np.float32).ravel())
    assert np.array_equal(a["y"], ((iy - (L - 1) / 2.0)).astype(np.float32).ravel())
    assert a["area"] == 1.0 and tuple(a["origin"]) == (0.0, 0.0, 0.0)
    for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs"):
        assert a[k].dtype == np.float32 and a[k].shape == (L * L,)
    b = sg.sea_surface(L, 5)
    c = sg.sea_surface(L, 6)
    for k in ("z", "vx", "vy", "vz", "nrcs"):
        assert np.array_equal(a[k], b[k])
        assert not np.array_equal(a[k], c[k])


def test_height_and_nrcs_distributions():
    L = 256
    s = sg.sea_surface(L, 3)
    z = s["z"].astype(np.float64)
    assert np.std(z) == pytest.approx(0.5, rel=1e-6)          # scaled to the sample std
    assert abs(np.mean(z)) < 1e-6                             # no k = 0 component
    ln = np.log(s["nrcs"].astype(np.float64))
    n = ln.size
    assert abs(np.mean(ln) + 2.0) < 5 * 0.5 / math.sqrt(n)    # lognormal(mu = -2, ...)
    assert abs(np.std(ln) - 0.5) < 5 * 0.5 / math.sqrt(2 * n)  # (..., sigma = 0.5)


def test_swell_peak_and_direction():
    """The height spectrum sits on the +x side, centred on k_p = 2 pi / 100 m^-1."""
    L = 1024
    s = sg.sea_surface(L, 7)
    Z = np.fft.fft2(s["z"].astype(np.float64).reshape(L, L))
    P = np.abs(Z) ** 2
    k = 2 * math.pi * np.fft.fftfreq(L)
    kx, ky = np.broadcast_to(k[None, :], (L, L)), np.broadcast_to(k[:, None], (L, L))
    # a real field has a Hermitian spectrum: count each wave once, on the kx > 0 side
    half = kx > 0
    assert P[kx == 0].sum() < 1e-10 * P.sum()
    w = P[half] / P[half].sum()
    kp = 2 * math.pi / 100.0
    assert np.sum(w * kx[half]) == pytest.approx(kp, rel=0.03)
    assert abs(np.sum(w * ky[half])) < 0.03 * kp
    # the spread of the Gaussian spectrum: sigma_k = max(0.006, 3 * 2 pi / L)
    sk = max(0.006, 3 * 2 * math.pi / L)
    assert math.sqrt(np.sum(w * ky[half] ** 2)) == pytest.approx(sk, rel=0.1)


def test_orbital_velocities_of_linear_deep_water_waves():
    """Each wave component of wave vector k (kx > 0) and height H(k) has, in linear
    deep-water theory, a vertical surface velocity -j omega H(k) and a horizontal one
    omega k/|k| H(k), omega = sqrt(g |k|): checked component by component."""
    L = 256
    s = sg.sea_surface(L, 11)
    F = {k: np.fft.fft2(s[k].astype(np.float64).reshape(L, L)) for k in ("z", "vx", "vy", "vz")}
    k = 2 * math.pi * np.fft.fftfreq(L)
    kx, ky = np.broadcast_to(k[None, :], (L, L)), np.broadcast_to(k[:, None], (L, L))
    kmag = np.hypot(kx, ky)
    half = kx > 0
    om = np.sqrt(9.81 * kmag[half])
    H = F["z"][half]

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    assert rel(F["vz"][half], -1j * om * H) < 1e-5
    assert rel(F["vx"][half], om * kx[half] / kmag[half] * H) < 1e-5
    assert rel(F["vy"][half], om * ky[half] / kmag[half] * H) < 1e-4
    # hence, for waves travelling towards +x, v_x is in phase with the height and v_z leads
    # it by a quarter period: v_z = -c dz/dx for a single wave
    z = s["z"].reshape(L, L).astype(np.float64)
    assert np.corrcoef(s["vx"], s["z"])[0, 1] > 0.9
    dzdx = np.gradient(z, axis=1).ravel()
    assert np.corrcoef(s["vz"], dzdx)[0, 1] < -0.9


def test_spectrum_reproduces_the_surface():
    """sea_spectrum (the description the surface update synthesises from) and sea_surface
    make the same t = 0 heights from the same draws."""
    L = 128
    s = sg.sea_surface(L, 21)
    sp = sg.sea_spectrum(L, 21)
    z = sp["scale"] * np.real(np.fft.ifft2(sp["coef"]))
    assert np.allclose(z.ravel(), s["z"], rtol=0, atol=1e-6)
    assert np.array_equal(sp["nrcs"], s["nrcs"])
    assert np.array_equal(sp["x"], s["x"]) and np.array_equal(sp["y"], s["y"])


def test_tracks_and_configurations():
    pf = sg.nadir_track(4096)
    t_mid = 4096 / (2 * 18_000.0)
    # P(t) = p0 + v t crosses the scene centre (x = 0) at mid-run, 800 km up
    assert pf.p0[0] + pf.v[0] * t_mid == pytest.approx(0.0, abs=1e-9)
    assert pf.p0[2] == 800e3 and pf.r_ref0 == 800e3 and pf.v == (7000.0, 0.0, 0.0)
    rd = sg.RadarParams()
    assert rd.c_mps / rd.carrier_hz == pytest.approx(0.022084159, rel=1e-8)   # Ku band
    c1 = sg.config(1)
    assert (c1["L"], c1["n_pulses"], c1["fast"].n_fast, c1["fast"].n_doppler) == (2048, 4096, 64, 64)
    sides = sg.cfg3_sides()
    assert sides.size == 128 and sides.min() >= 1024 and sides.max() <= 4096
    assert np.array_equal(sides, sg.cfg3_sides())
