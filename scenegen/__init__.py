"""Seeded synthetic inputs for the radar raw-data summation.

This module only *generates inputs*: sea-surface scatterer sets, radar and
platform parameter sets, random Doppler spectra and target waveforms.  It holds
none of the summation method's arithmetic (no range, phase, gate, Doppler,
FFT-of-spectra or weighting code), so both the CUDA path and the CPU oracle can
draw their inputs from it without sharing method code.

Workload shapes follow the paper's altimetry scenario (Section IV: Ku band
13.575 GHz, ~18 kHz PRF, 1 m scatterer grid, nadir track) and the five
configurations this library is measured on:

* ``cfg0``  regular mode, 256 x 256 surface, 64 pulses;
* ``cfg1``  fast mode, 2048 x 2048 surface, 4096 pulses, n_fast = 64,
  64 Doppler bins, square-root raised-cosine blend;
* ``cfg2``  4096 x 4096 surface, 8192 pulses (precision study);
* ``cfg3``  128 realizations of uneven size (1024..4096 sides) on a 100 km
  track, fast mode;
* ``cfg4``  adjoint: 1024 x 1024 surface, 256 pulses, fast mode.

Surface recipe (stands in for the paper's Choppy-Wave-Model surfaces, which
are out of scope): a linear deep-water random-phase wave field from a
one-sided Gaussian spectrum centred on k_p = 2 pi / 100 m^-1 along +x
(the swell shape of Section IV.D, S1), widths
sigma_kx = sigma_ky = max(0.006, 3 * 2 pi / L) m^-1, heights scaled to a sample
standard deviation of 0.5 m, orbital velocities from the same coefficients
(omega = sqrt(g |k|)), and NRCS drawn i.i.d. lognormal(mu=-2, sigma=0.5) in
linear units.  Grid index n = iy * L + ix (row-major, x fastest), positions
centred on the origin with 1 m spacing.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional

import numpy as np

C_LIGHT = 299_792_458.0
G_EARTH = 9.81

__all__ = [
    "C_LIGHT",
    "AntennaTable",
    "RadarParams",
    "antenna_table",
    "PlatformParams",
    "FastParams",
    "WINDOWS",
    "nadir_track",
    "sea_surface",
    "sea_spectrum",
    "point_scene",
    "random_spectra",
    "random_iq",
    "target_waveform",
    "cfg3_sides",
    "CONFIGS",
    "config",
]

# Blend windows between consecutive spectra (numbering shared by both sides).
WINDOWS = {"sqrt_linear": 0, "sqrt_raised_cosine": 1, "linear": 2}


@dataclasses.dataclass(frozen=True, eq=False)
class AntennaTable:
    """Two-way complex antenna pattern on a u-v grid: ``gain[j, i]`` at direction cosines
    u = u0 + i du, v = v0 + j dv (complex, shape [nv, nu])."""

    gain: np.ndarray
    u0: float
    du: float
    v0: float
    dv: float


@dataclasses.dataclass(frozen=True)
class RadarParams:
    """Instrument constants (SI units).  ``antenna``: a tabulated two-way pattern, or None
    for the analytic Gaussian pattern of beamwidth ``beamwidth_rad``."""

    carrier_hz: float = 13.575e9
    prf_hz: float = 18_000.0
    c_mps: float = C_LIGHT
    gate_width_m: float = 0.47
    beamwidth_rad: float = math.radians(1.3)
    n_gates: int = 128
    antenna: Optional[AntennaTable] = None


def antenna_table(seed: int, n: int = 129, half_width: float = 0.05,
                  width: float = 0.0193, ripple: float = 0.3) -> AntennaTable:
    """Seeded synthetic two-way pattern on an n x n grid over |u|, |v| <= half_width: an
    elliptical main lobe exp(-(u/a)^2 - (v/b)^2) with a and b drawn within 15 % of
    ``width``, a small seeded boresight offset and a smooth phase ripple of up to
    ``ripple`` rad (the shape a measured pattern table has near the main lobe)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a, b = width * (1.0 + 0.15 * (2.0 * rng.random(2) - 1.0))
    u_off, v_off = 0.05 * width * (2.0 * rng.random(2) - 1.0)
    ku, kv, ph = rng.random(3) * np.array([2.0, 2.0, 2.0 * math.pi])
    g = np.linspace(-half_width, half_width, n)
    U, V = g[None, :], g[:, None]
    amp = np.exp(-((U - u_off) / a) ** 2 - ((V - v_off) / b) ** 2)
    phase = ripple * np.sin(ku * U / width + kv * V / width + ph)
    d = float(g[1] - g[0])
    return AntennaTable(gain=amp * np.exp(1j * phase), u0=float(g[0]), du=d, v0=float(g[0]), dv=d)


@dataclasses.dataclass(frozen=True)
class PlatformParams:
    """Platform track P(t) = p0 + v t and reference range r_ref(t) = r_ref0 + r_ref_rate t."""

    p0: tuple = (0.0, 0.0, 800e3)
    v: tuple = (7_000.0, 0.0, 0.0)
    r_ref0: float = 800e3
    r_ref_rate: float = 0.0


@dataclasses.dataclass(frozen=True)
class FastParams:
    """Fast-mode schedule: spectra every n_fast pulses, n_doppler bins, blend window."""

    n_fast: int = 64
    n_doppler: int = 64
    window: str = "sqrt_raised_cosine"


def nadir_track(n_pulses: int, prf_hz: float = 18_000.0, altitude_m: float = 800e3,
                speed_mps: float = 7_000.0, t_mid: Optional[float] = None) -> PlatformParams:
    """Nadir-looking platform whose ground track crosses the scene centre at t_mid.

    Default t_mid = n_pulses / (2 PRF), i.e. mid-run.  The range window is
    centred on the mean surface: r_ref = altitude (flat earth).
    """
    if t_mid is None:
        t_mid = n_pulses / (2.0 * prf_hz)
    return PlatformParams(p0=(-speed_mps * t_mid, 0.0, altitude_m), v=(speed_mps, 0.0, 0.0),
                          r_ref0=altitude_m, r_ref_rate=0.0)


def _fft_backend(backend: str, device):
    if backend == "numpy":
        return None
    import torch  # noqa: F401  (optional backend)
    return torch


def sea_surface(L: int, seed: int, spacing: float = 1.0, height_std: float = 0.5,
                k_peak: float = 2.0 * math.pi / 100.0, sigma_k: Optional[float] = None,
                nrcs_mu: float = -2.0, nrcs_sigma: float = 0.5, backend: str = "numpy",
                device=None) -> Dict[str, object]:
    """Seeded L x L sea surface of scatterers (float32 structure-of-arrays).

    Returns a dict with keys x, y, z, vx, vy, vz, nrcs (each length L*L,
    float32; numpy arrays, or torch tensors on ``device`` when
    ``backend == "torch"``), plus ``origin`` (3 floats) and ``area`` (m^2).

    The random draws always come from numpy's PCG64(seed) in a fixed order
    (two standard-normal planes for the complex coefficients, then the NRCS
    plane), so both backends see the same numbers; the torch backend only
    moves the inverse FFTs onto the device for large batches.
    """
    if L < 2:
        raise ValueError("L must be >= 2")
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal((L, L))
    im = rng.standard_normal((L, L))
    ln_nrcs = rng.normal(nrcs_mu, nrcs_sigma, size=(L, L))
    if sigma_k is None:
        sigma_k = max(0.006, 3.0 * 2.0 * math.pi / (L * spacing))
    torch = _fft_backend(backend, device)
    xp = np if torch is None else torch
    dev = None if torch is None else (device if device is not None else "cpu")

    def arr(a):
        return a if torch is None else torch.from_numpy(a).to(dev)

    # the same float64 arithmetic on either backend (numpy on the host, torch on `device`)
    k1 = arr(2.0 * math.pi * np.fft.fftfreq(L, d=spacing))
    kx = k1[None, :]
    ky = k1[:, None]
    spec = xp.exp(-((kx - k_peak) ** 2 + ky ** 2) / (2.0 * sigma_k ** 2))
    spec = xp.where(kx > 0.0, spec, xp.zeros_like(spec))  # one-sided: waves travel towards +x
    amp = xp.sqrt(spec) * (arr(re) + 1j * arr(im)) / math.sqrt(2.0)
    del re, im
    kmag = xp.sqrt(kx ** 2 + ky ** 2)
    omega = xp.sqrt(G_EARTH * kmag)
    safe = xp.where(kmag > 0, kmag, xp.ones_like(kmag))
    ux = xp.where(kmag > 0, kx / safe, xp.zeros_like(kmag))
    uy = xp.where(kmag > 0, ky / safe, xp.zeros_like(kmag))
    ifft2 = np.fft.ifft2 if torch is None else torch.fft.ifft2
    eta = ifft2(amp).real
    wz = ifft2(-1j * omega * amp).real
    wx = ifft2(omega * ux * amp).real
    wy = ifft2(omega * uy * amp).real
    del amp
    xs = (np.arange(L, dtype=np.float64) - (L - 1) / 2.0) * spacing
    nrcs = np.exp(ln_nrcs).astype(np.float32).ravel()
    if torch is None:
        scale = height_std / float(np.std(eta))
        X = np.broadcast_to(xs[None, :], (L, L))
        Y = np.broadcast_to(xs[:, None], (L, L))
        out = {
            "x": X.astype(np.float32).ravel(),
            "y": Y.astype(np.float32).ravel(),
            "z": (eta * scale).astype(np.float32).ravel(),
            "vx": (wx * scale).astype(np.float32).ravel(),
            "vy": (wy * scale).astype(np.float32).ravel(),
            "vz": (wz * scale).astype(np.float32).ravel(),
            "nrcs": nrcs,
        }
    else:
        scale = height_std / float(eta.std(unbiased=False))
        xt = torch.from_numpy(xs).to(dev)
        out = {
            "x": xt[None, :].expand(L, L).reshape(-1).to(torch.float32),
            "y": xt[:, None].expand(L, L).reshape(-1).to(torch.float32),
            "z": (eta * scale).to(torch.float32).reshape(-1),
            "vx": (wx * scale).to(torch.float32).reshape(-1),
            "vy": (wy * scale).to(torch.float32).reshape(-1),
            "vz": (wz * scale).to(torch.float32).reshape(-1),
            "nrcs": torch.from_numpy(nrcs).to(dev),
        }
    out["origin"] = (0.0, 0.0, 0.0)
    out["area"] = float(spacing * spacing)
    return out


def sea_spectrum(L: int, seed: int, spacing: float = 1.0, height_std: float = 0.5,
                 k_peak: float = 2.0 * math.pi / 100.0, sigma_k: Optional[float] = None,
                 nrcs_mu: float = -2.0, nrcs_sigma: float = 0.5) -> Dict[str, object]:
    """The spectral description behind ``sea_surface(L, seed, ...)`` (same draws): the
    one-sided complex wave coefficients ``coef`` [L, L] (complex128, index [iy, ix], wave
    numbers 2 pi fftfreq(L, spacing) along x and y), the amplitude ``scale`` that gives the
    t = 0 heights a standard deviation of ``height_std``, the facet grid x, y and the NRCS
    (float32, length L*L), ``origin``, ``area``, ``spacing``.  The surface at time t is
    synthesised from these by the spectral update (linear deep-water waves)."""
    if L < 2:
        raise ValueError("L must be >= 2")
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal((L, L))
    im = rng.standard_normal((L, L))
    ln_nrcs = rng.normal(nrcs_mu, nrcs_sigma, size=(L, L))
    if sigma_k is None:
        sigma_k = max(0.006, 3.0 * 2.0 * math.pi / (L * spacing))
    k1 = 2.0 * math.pi * np.fft.fftfreq(L, d=spacing)
    kx, ky = k1[None, :], k1[:, None]
    spec = np.exp(-((kx - k_peak) ** 2 + ky ** 2) / (2.0 * sigma_k ** 2))
    spec = np.where(kx > 0.0, spec, 0.0)
    coef = np.sqrt(spec) * (re + 1j * im) / math.sqrt(2.0)
    scale = height_std / float(np.std(np.real(np.fft.ifft2(coef))))
    xs = (np.arange(L, dtype=np.float64) - (L - 1) / 2.0) * spacing
    return {"coef": coef, "scale": scale, "spacing": float(spacing), "L": int(L),
            "x": np.broadcast_to(xs[None, :], (L, L)).astype(np.float32).ravel(),
            "y": np.broadcast_to(xs[:, None], (L, L)).astype(np.float32).ravel(),
            "nrcs": np.exp(ln_nrcs).astype(np.float32).ravel(),
            "origin": (0.0, 0.0, 0.0), "area": float(spacing * spacing)}


def point_scene(points, area: float = 1.0, origin=(0.0, 0.0, 0.0)) -> Dict[str, object]:
    """Scene of explicit scatterers: ``points`` is a sequence of
    (x, y, z, vx, vy, vz, nrcs) tuples (float32 after conversion)."""
    arr = np.asarray(points, dtype=np.float64).reshape(-1, 7)
    keys = ["x", "y", "z", "vx", "vy", "vz", "nrcs"]
    out = {k: arr[:, i].astype(np.float32) for i, k in enumerate(keys)}
    out["origin"] = tuple(float(o) for o in origin)
    out["area"] = float(area)
    return out


def random_spectra(n_spectra: int, n_gates: int, n_doppler: int, seed: int) -> np.ndarray:
    """i.i.d. circular complex Gaussian spectra, shape [S, N_g, N_d], complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal((n_spectra, n_gates, n_doppler))
    im = rng.standard_normal((n_spectra, n_gates, n_doppler))
    return (re + 1j * im) / math.sqrt(2.0)


def random_iq(n_pulses: int, n_gates: int, seed: int) -> np.ndarray:
    """i.i.d. circular complex Gaussian IQ block [P, N_g], complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal((n_pulses, n_gates))
    im = rng.standard_normal((n_pulses, n_gates))
    return (re + 1j * im) / math.sqrt(2.0)


def target_waveform(n_pulses: int, n_gates: int, seed: int, mean_power) -> np.ndarray:
    """Seeded target waveform power P*[x, g] = mean_power[g] * Exp(1) (float64).

    ``mean_power`` is a scalar or a length-N_g profile.  Stands in for a
    measured waveform in the adjoint (inversion) workload.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    e = rng.standard_exponential((n_pulses, n_gates))
    return e * np.broadcast_to(np.asarray(mean_power, dtype=np.float64), (n_gates,))[None, :]


def cfg3_sides(n_real: int = 128, seed: int = 3, lo: int = 1024, hi: int = 4096) -> np.ndarray:
    """Side lengths of the uneven batched realizations, uniform on {lo..hi}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n_real)


def _cfg(name, L, n_pulses, seed, mode, fast=None, note=""):
    return {"name": name, "L": L, "n_pulses": n_pulses, "seed": seed, "mode": mode,
            "fast": fast, "note": note}


CONFIGS = {
    0: _cfg("regular_256x256_p64", 256, 64, 0, "regular",
            note="65,536 scatterers, 64 pulses, FP64 direct summation"),
    1: _cfg("fast_2048x2048_p4096", 2048, 4096, 1, "fast",
            FastParams(64, 64, "sqrt_raised_cosine"),
            note="4.19M scatterers, 65 spectra of 128 gates x 64 bins, 4096 pulses"),
    2: _cfg("fast_4096x4096_p8192", 4096, 8192, 2, "fast",
            FastParams(64, 64, "sqrt_raised_cosine"),
            note="16.8M scatterers, 129 spectra, precision study"),
    3: _cfg("batched_128_uneven_100km", None, None, 1000, "batched",
            FastParams(64, 64, "sqrt_raised_cosine"),
            note="128 realizations of side U{1024..4096}, 100 km track"),
    4: _cfg("adjoint_1024x1024_p256", 1024, 256, 4, "fast",
            FastParams(64, 64, "sqrt_raised_cosine"),
            note="1.05M scatterers, 256 pulses, waveform-power loss"),
}


def config(idx: int) -> dict:
    """Return a copy of configuration ``idx`` with radar and platform filled in."""
    c = dict(CONFIGS[idx])
    c["radar"] = RadarParams()
    if c["n_pulses"] is not None:
        c["platform"] = nadir_track(c["n_pulses"])
    return c
