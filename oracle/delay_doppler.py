"""Delay-Doppler focusing of simulated IQ, FP64 numpy restatement (Section IV.C).

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``): used by the tests and by
the CPU-baseline leg of the benchmark; the library never imports it.

The paper focuses its raw data with a delay-Doppler algorithm: the pulses are split into
bursts of 64, and per burst (1) the Doppler centroid shift of a trajectory that is not
tangent to the surface is corrected, (2) an along-track FFT forms Doppler beams, (3) the
range migration of the scatterers seen in each beam is corrected with delay phase
coefficients; multi-look then averages the Doppler beams.  The paper gives no formulas;
the readings taken here (flat earth, constant platform velocity V, reference range R_0 of
the burst's centre pulse):

    burst b: pulses x_b + k, k = 0 .. N_b - 1, x_b = pulse0 + b N_b
    (1) y_k <- y_k exp(-j 2 pi nu_c k),  nu_c = -2 V_z / (lambda PRF)
        (the phase advance per pulse of the nadir echo, whose range changes at V_z)
    (2) B_f = sum_k y_k exp(-j 2 pi nu_f k),  nu_f = (f - N_b/2) / N_b,  f = 0 .. N_b - 1
    (3) a facet at along-track offset x has nu = 2 V_h x / (lambda R_0 PRF)
        (V_h = horizontal speed), so beam f looks at x_f = nu_f lambda R_0 PRF / (2 V_h),
        whose range exceeds the nadir's by x_f^2 / (2 R_0), s_f = x_f^2 / (2 R_0 gw) gates;
        the beam's waveform is advanced by s_f gates with the shift theorem over the
        n_gates-point range transform (signed frequencies q' in [-N_g/2, N_g/2)):
        Y_f = IDFT( DFT(B_f) exp(+j 2 pi q' s_f / N_g) ) (IDFT normalised by 1 / N_g)
    (4) multi-look: W_b[g] = (1 / N_b) sum_f |Y_f[g]|^2
"""
from __future__ import annotations

import math

import numpy as np


def centroid(radar, platform) -> float:
    """Doppler centroid nu_c of the nadir echo, cycles per pulse."""
    lam = radar.c_mps / radar.carrier_hz
    return -2.0 * float(platform.v[2]) / (lam * radar.prf_hz)


def migration_gates(radar, platform, burst: int, r0: float) -> np.ndarray:
    """Range-migration shift s_f (gates) of every Doppler beam f = 0 .. burst - 1."""
    lam = radar.c_mps / radar.carrier_hz
    vh = math.hypot(float(platform.v[0]), float(platform.v[1]))
    nu = (np.arange(burst) - burst // 2) / burst
    if vh == 0.0:
        return np.zeros(burst)
    x = nu * lam * r0 * radar.prf_hz / (2.0 * vh)
    return x * x / (2.0 * r0 * radar.gate_width_m)


def focus(radar, platform, iq, pulse0: int, burst: int):
    """Focused beams Y [n_bursts, burst, n_gates] (complex128) and multi-looked
    waveforms W [n_bursts, n_gates] of iq [n_pulses, n_gates] (pulses pulse0 ..)."""
    iq = np.asarray(iq, dtype=np.complex128)
    n_pulses, G = iq.shape
    nb = n_pulses // burst
    k = np.arange(burst)
    nu_c = centroid(radar, platform)
    corr = np.exp(-2j * np.pi * nu_c * k)                 # (1)
    nu_f = (np.arange(burst) - burst // 2) / burst
    dft = np.exp(-2j * np.pi * np.outer(nu_f, k))         # (2) [f, k]
    qs = np.fft.fftfreq(G) * G                            # signed range frequencies
    Y = np.zeros((nb, burst, G), dtype=np.complex128)
    W = np.zeros((nb, G))
    for b in range(nb):
        x_c = pulse0 + b * burst + burst // 2
        r0 = platform.r_ref0 + platform.r_ref_rate * x_c / radar.prf_hz
        s = migration_gates(radar, platform, burst, r0)
        y = iq[b * burst:(b + 1) * burst] * corr[:, None]
        B = dft @ y                                        # [f, g]
        ramp = np.exp(2j * np.pi * np.outer(s, qs) / G)    # (3)
        Y[b] = np.fft.ifft(np.fft.fft(B, axis=1) * ramp, axis=1)
        W[b] = (np.abs(Y[b]) ** 2).mean(axis=0)            # (4)
    return Y, W
