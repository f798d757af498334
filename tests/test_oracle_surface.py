"""Pins of the spectral surface update (the surface regenerated at every update of
Algorithm 1 from linear deep-water waves): a single wave against its closed form, the time
derivative against v_z, the seeded generator at t = 0, and the dispersion relation."""
import math

import numpy as np
import pytest

import scenegen as sg
from oracle import surface as sf


def _single_wave(L, ix, iy, amp, spacing=1.0):
    coef = np.zeros((L, L), complex)
    coef[iy, ix] = amp
    xs = (np.arange(L) - (L - 1) / 2.0) * spacing
    return {"coef": coef, "scale": 1.0, "spacing": spacing, "L": L,
            "x": np.broadcast_to(xs[None, :], (L, L)).astype(np.float32).ravel(),
            "y": np.broadcast_to(xs[:, None], (L, L)).astype(np.float32).ravel(),
            "nrcs": np.ones(L * L, np.float32), "origin": (0.0, 0.0, 0.0), "area": 1.0}


@pytest.mark.parametrize("ix,iy", [(3, 0), (5, 2), (1, 14)])
def test_single_wave_travels_with_the_deep_water_speed(ix, iy):
    """One coefficient a e^{j phi} at grid wave number k: eta = |a| cos(k.r - omega t + phi)
    / L^2 on the grid points r = (i, j) spacing (index origin at the first node),
    omega = sqrt(g |k|); v_z = d eta/dt; (v_x, v_y) = omega k_hat eta."""
    L, spacing = 16, 2.0
    a = 0.8 * np.exp(0.3j)
    spec = _single_wave(L, ix, iy, a, spacing)
    k1 = 2 * math.pi * np.fft.fftfreq(L, d=spacing)
    kx, ky = k1[ix], k1[iy]
    k = math.hypot(kx, ky)
    w = math.sqrt(sf.G_EARTH * k)
    i, j = np.meshgrid(np.arange(L), np.arange(L))
    for t in (0.0, 0.7, 13.25):
        ph = kx * i * spacing + ky * j * spacing - w * t + 0.3
        f = sf.surface_at(spec, t)
        np.testing.assert_allclose(f["z"], (0.8 * np.cos(ph) / L ** 2).ravel(), atol=1e-15)
        np.testing.assert_allclose(f["vz"], (0.8 * w * np.sin(ph) / L ** 2).ravel(), atol=1e-15)
        np.testing.assert_allclose(f["vx"], (0.8 * w * kx / k * np.cos(ph) / L ** 2).ravel(), atol=1e-15)
        np.testing.assert_allclose(f["vy"], (0.8 * w * ky / k * np.cos(ph) / L ** 2).ravel(), atol=1e-15)


def test_time_derivative_of_height_is_vz():
    spec = sg.sea_spectrum(64, 3)
    t, h = 4.0, 1e-3
    dz = (sf.surface_at(spec, t + h)["z"] - sf.surface_at(spec, t - h)["z"]) / (2 * h)
    vz = sf.surface_at(spec, t)["vz"]
    assert np.abs(dz - vz).max() < 1e-5 * np.abs(vz).max()


def test_t0_fields_are_the_seeded_surface():
    for L, seed in ((48, 2), (64, 9)):
        spec = sg.sea_spectrum(L, seed)
        ref = sg.sea_surface(L, seed)
        sc = sf.scene_at(spec, 0.0)
        for key in ("x", "y", "z", "vx", "vy", "vz", "nrcs"):
            np.testing.assert_array_equal(sc[key], ref[key])
        assert sc["t0"] == 0.0


def test_heights_keep_their_variance_and_the_period_of_each_wave():
    """Linear waves: the height variance does not change with time (Parseval over the
    one-sided spectrum), and a surface of one wave repeats after its period."""
    spec = sg.sea_spectrum(64, 5)
    v0 = np.var(sf.surface_at(spec, 0.0)["z"])
    assert np.var(sf.surface_at(spec, 37.0)["z"]) == pytest.approx(v0, rel=1e-10)
    one = _single_wave(32, 4, 0, 1.0)
    T = 2 * math.pi / math.sqrt(sf.G_EARTH * 2 * math.pi * 4 / 32)
    np.testing.assert_allclose(sf.surface_at(one, T)["z"], sf.surface_at(one, 0.0)["z"], atol=1e-15)
