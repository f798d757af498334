"""Spectral update of the sea surface, FP64 numpy restatement (Algorithm 1's
update_simulation, Sections III.A and IV: the surface is regenerated at every update
instead of being moved along straight lines).

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).

Linear deep-water waves from one-sided complex coefficients A(k) on the L x L wave-number
grid k = 2 pi fftfreq(L, spacing) (index [iy, ix]): with omega = sqrt(g |k|),

    eta(x, t) = s Re IFFT2[A e^{-j omega t}]                 (height)
    v_z(x, t) = s Re IFFT2[-j omega A e^{-j omega t}]        (= d eta / dt)
    v_x(x, t) = s Re IFFT2[omega (k_x/|k|) A e^{-j omega t}] (orbital velocity along k)
    v_y(x, t) = s Re IFFT2[omega (k_y/|k|) A e^{-j omega t}]

IFFT2 normalised by 1 / L^2 (numpy's convention), s the amplitude scale of the spectrum
description.  The facet grid (x, y) is fixed; at t = 0 these are the fields the seeded
surface generator returns.
"""
from __future__ import annotations

import math

import numpy as np

G_EARTH = 9.81


def wave_numbers(L: int, spacing: float):
    k1 = 2.0 * math.pi * np.fft.fftfreq(L, d=spacing)
    return k1[None, :], k1[:, None]


def surface_at(spectrum, t: float, g: float = G_EARTH):
    """Heights and velocities (float64, length L*L, row-major like the facet grid) at time t."""
    A = np.asarray(spectrum["coef"], dtype=np.complex128)
    L = A.shape[0]
    kx, ky = wave_numbers(L, spectrum["spacing"])
    kmag = np.sqrt(kx ** 2 + ky ** 2)
    omega = np.sqrt(g * kmag)
    with np.errstate(invalid="ignore", divide="ignore"):
        ux = np.where(kmag > 0, kx / np.where(kmag > 0, kmag, 1.0), 0.0)
        uy = np.where(kmag > 0, ky / np.where(kmag > 0, kmag, 1.0), 0.0)
    At = A * np.exp(-1j * omega * t)
    s = spectrum["scale"]

    def field(mult):
        return (s * np.real(np.fft.ifft2(mult * At))).ravel()

    return {"z": field(1.0), "vz": field(-1j * omega), "vx": field(omega * ux),
            "vy": field(omega * uy)}


def scene_at(spectrum, t: float, g: float = G_EARTH):
    """A scene dict (float32 arrays, state epoch t0 = t) of the surface at time t."""
    f = surface_at(spectrum, t, g)
    out = {k: np.asarray(v, dtype=np.float32) for k, v in f.items()}
    out.update(x=spectrum["x"], y=spectrum["y"], nrcs=spectrum["nrcs"], origin=spectrum["origin"],
               area=spectrum["area"], t0=float(t))
    return out
