"""Vectorised numpy restatement of the oracle for tiny inputs (N <= a few thousand).

TEST INFRASTRUCTURE ONLY.  Written independently of ``rsim_oracle.c`` (numpy
array code, ``numpy.fft`` as the transform, ``np.add.at`` as the scatter-add)
so that a slip in either restatement (an index, a sign, a transposed operand)
shows up as a disagreement between the two.

Readings are the same as the C oracle's (see its header): stop-and-hop timing,
linear kinematics, flat earth, nadir Gaussian two-way pattern, unnormalised
inverse transform, nearest Doppler bin with ties upward, periodic segments.
"""
from __future__ import annotations

import math

import numpy as np


def _scene_arrays(scene):
    f = {k: np.asarray(scene[k], dtype=np.float32).astype(np.float64)
         for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs")}
    o = np.asarray(scene.get("origin", (0.0, 0.0, 0.0)), dtype=np.float64)
    return f, o, float(scene.get("area", 1.0))


def pattern(antenna, u, v):
    """Tabulated two-way pattern at direction cosines (u, v): bilinear in the real and
    imaginary parts between the grid nodes, 0 outside [u0, u0 + (nu-1) du) x [v0, ...)."""
    tab = np.asarray(antenna.gain, dtype=np.complex128)
    nv, nu = tab.shape
    x = (np.asarray(u, dtype=np.float64) - antenna.u0) / antenna.du
    y = (np.asarray(v, dtype=np.float64) - antenna.v0) / antenna.dv
    col, row = np.floor(x), np.floor(y)
    inside = (col >= 0) & (col <= nu - 2) & (row >= 0) & (row <= nv - 2)
    c = np.where(inside, col, 0).astype(np.int64)
    r = np.where(inside, row, 0).astype(np.int64)
    fx, fy = x - col, y - row
    top = tab[r, c] + fx * (tab[r, c + 1] - tab[r, c])          # at v = v_row
    bottom = tab[r + 1, c] + fx * (tab[r + 1, c + 1] - tab[r + 1, c])
    return np.where(inside, top + fy * (bottom - top), 0.0)


def echo(radar, platform, scene, t):
    """Complex amplitude, range excess and range of every scatterer at time t."""
    f, o, area = _scene_arrays(scene)
    ts = t - float(scene.get("t0", 0.0))   # the state is given at epoch t0
    pos = np.stack([o[0] + f["x"] + f["vx"] * ts, o[1] + f["y"] + f["vy"] * ts,
                    o[2] + f["z"] + f["vz"] * ts])
    plat = np.asarray(platform.p0, dtype=np.float64) + np.asarray(platform.v, dtype=np.float64) * t
    d = plat[:, None] - pos
    horiz = np.hypot(d[0], d[1])
    rng = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    r_ref = platform.r_ref0 + platform.r_ref_rate * t
    lam = radar.c_mps / radar.carrier_hz
    off_nadir = np.arctan2(horiz, d[2])
    if getattr(radar, "antenna", None) is not None:
        # direction cosines of the line of sight platform -> scatterer
        gain = pattern(radar.antenna, -d[0] / rng, -d[1] / rng)
    else:
        # Gaussian two-way pattern whose power is halved at theta = beamwidth / 2.
        gain = 0.5 ** ((2.0 * off_nadir / radar.beamwidth_rad) ** 2 / 2.0)
    amp = np.sqrt(f["nrcs"] * area) * gain * (r_ref / rng) ** 2
    cycles = 2.0 * rng / lam
    frac = cycles - np.round(cycles)
    C = amp * np.exp(-2j * np.pi * frac)
    return C, rng - r_ref, rng


def gates(radar, dR):
    return np.floor(dR / radar.gate_width_m + radar.n_gates / 2.0).astype(np.int64)


def doppler_bins(radar, C1, C2, n_doppler):
    """Nearest bin of the pulse-pair frequency of C (cycles / pulse)."""
    freq = np.angle(C2 * np.conj(C1)) / (2.0 * np.pi)  # phase advance per pulse
    return np.mod(np.floor(freq * n_doppler + 0.5).astype(np.int64), n_doppler)


def direct_sum(radar, platform, scene, pulse0, n_pulses):
    G = radar.n_gates
    Y = np.zeros((n_pulses, G), dtype=np.complex128)
    for p in range(n_pulses):
        C, dR, _ = echo(radar, platform, scene, (pulse0 + p) / radar.prf_hz)
        g = gates(radar, dR)
        ok = (g >= 0) & (g < G)
        np.add.at(Y[p], g[ok], C[ok])
    return Y


def doppler_spectra(radar, platform, scene, update0, n_updates, n_fast, n_doppler):
    G = radar.n_gates
    T = np.zeros((n_updates, G, n_doppler), dtype=np.complex128)
    for u in range(n_updates):
        p = (update0 + u) * n_fast
        C1, dR, _ = echo(radar, platform, scene, p / radar.prf_hz)
        C2, _, _ = echo(radar, platform, scene, (p + 1) / radar.prf_hz)
        g = gates(radar, dR)
        k = doppler_bins(radar, C1, C2, n_doppler)
        ok = (g >= 0) & (g < G)
        np.add.at(T[u], (g[ok], k[ok]), C1[ok])
    return T


def weights(window, dist):
    """Blend weight at normalised distance |p_i - x| / n_fast (zero beyond 1)."""
    dist = np.abs(np.asarray(dist, dtype=np.float64))
    inside = dist <= 1.0
    dd = np.minimum(dist, 1.0)
    if window == "sqrt_linear":
        w = np.sqrt(1.0 - dd)
    elif window == "sqrt_raised_cosine":
        w = np.sqrt(0.5 * (1.0 + np.cos(np.pi * dd)))  # squared weight is a raised cosine
    elif window == "linear":
        w = 1.0 - dd
    else:
        raise ValueError(window)
    return np.where(inside, w, 0.0)


def synth(T, update0, n_fast, pulse0, n_pulses, window):
    S, G, K = T.shape
    seg = np.fft.ifft(T, axis=-1) * K  # unnormalised inverse transform per gate
    Y = np.zeros((n_pulses, G), dtype=np.complex128)
    x = pulse0 + np.arange(n_pulses)
    for s in range(S):
        p_i = (update0 + s) * n_fast
        w = weights(window, (x - p_i) / n_fast)
        m = np.mod(x - p_i, K)
        Y += w[:, None] * seg[s][:, m].T
    return Y
