"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets a plausible slip in the oracle: phase sign, gate index,
dropped amplitude factors, Doppler sign, transform direction or normalisation,
segment time origin, window exponent, spectrum/gate transposition.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import scenegen as sg
from oracle import bruteforce as bf
from oracle import n_spectra

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
H = 800e3


def static_platform(z=H, x=0.0):
    return sg.PlatformParams(p0=(x, 0.0, z), v=(0.0, 0.0, 0.0), r_ref0=H, r_ref_rate=0.0)


def frac_cycles_exact(radar, rng_exact):
    """Fractional part of 2 R / lambda = 2 R f_c / c in exact rational arithmetic."""
    cyc = 2 * rng_exact * Fraction(radar.carrier_hz) / Fraction(radar.c_mps)
    return float(cyc - round(cyc))


def wrap_angle(a):
    return (a + math.pi) % (2 * math.pi) - math.pi


# --------------------------------------------------------------------------- geometry
@pytest.mark.parametrize("h", [0.1, -1.0, 3.3, -7.77])
def test_point_scatterer_at_nadir_closed_form(orc, h):
    """Single scatterer under a static platform: R = H - h, gate = floor(-h/dRg + Ng/2),
    phase = -4 pi R / lambda, amplitude = sqrt(sigma A) (H / R)^2 (Sec. II.A radar equation)."""
    rd = sg.RadarParams()
    pf = static_platform()
    sigma, area = 0.25, 2.0
    sc = sg.point_scene([(0.0, 0.0, h, 0.0, 0.0, 0.0, sigma)], area=area)
    hz = Fraction(float(np.float32(h)))
    R_exact = Fraction(H) - hz
    e = orc.echo(rd, pf, sc, 0.0)
    assert e["R"][0] == pytest.approx(float(R_exact), abs=1e-9)
    amp = math.sqrt(float(np.float32(sigma)) * area) * (H / float(R_exact)) ** 2
    assert abs(e["C"][0]) == pytest.approx(amp, rel=1e-13)
    phase_expected = -2 * math.pi * frac_cycles_exact(rd, R_exact)
    assert abs(wrap_angle(np.angle(e["C"][0]) - phase_expected)) < 2e-7
    gate = math.floor(-hz / Fraction(rd.gate_width_m) + Fraction(rd.n_gates, 2))
    Y = orc.direct_sum(rd, pf, sc, 0, 1)
    nz = np.nonzero(np.abs(Y[0]) > 0)[0]
    assert list(nz) == [gate]
    assert Y[0, gate] == pytest.approx(e["C"][0], rel=1e-14)


def test_antenna_half_power_at_half_beamwidth(orc):
    """Two-way Gaussian pattern: power halves at theta = theta_b/2, 1/16 at theta_b."""
    rd = sg.RadarParams()
    pf = static_platform()
    pts = []
    for th in (0.5 * rd.beamwidth_rad, rd.beamwidth_rad):
        pts.append((float(np.float32(H * math.tan(th))), 0.0, 0.0, 0.0, 0.0, 0.0, 1.0))
    sc = sg.point_scene(pts, area=1.0)
    e = orc.echo(rd, pf, sc, 0.0)
    for j, want in enumerate((0.5, 1.0 / 16.0)):
        x = float(sc["x"][j])
        R = math.hypot(x, H)
        theta = math.atan2(x, H)
        gain_power = (abs(e["C"][j]) / (H / R) ** 2) ** 2
        # theta differs from the exact fraction of the beamwidth only by float32 rounding of x
        expect = want ** ((theta / (rd.beamwidth_rad * (0.5 if j == 0 else 1.0))) ** 2)
        assert gain_power == pytest.approx(expect, rel=1e-12)
        assert gain_power == pytest.approx(want, rel=1e-6)


def test_gate_boundaries(orc):
    """Scatterers just inside / outside gate edges land in the gate floor() gives."""
    rd = sg.RadarParams()
    pf = static_platform()
    pts, expect = [], []
    for j in (0, 1, 37, 64, 65, 100, 127):
        edge = (j - rd.n_gates // 2) * rd.gate_width_m   # dR at the lower edge of gate j
        for eps in (-2e-5, 2e-5):
            h = np.float32(-(edge + eps))
            hz = Fraction(float(h))
            g = math.floor(-hz / Fraction(rd.gate_width_m) + Fraction(rd.n_gates, 2))
            pts.append((0.0, 0.0, float(h), 0.0, 0.0, 0.0, 1.0))
            expect.append(g)
    sc = sg.point_scene(pts)
    gate, _, _, _ = orc.cells(rd, pf, sc, 0, 64)
    assert list(gate) == expect
    # out-of-window scatterers are dropped from the sum
    far = sg.point_scene([(0.0, 0.0, 40.0, 0, 0, 0, 1.0), (0.0, 0.0, -40.0, 0, 0, 0, 1.0)])
    assert np.all(orc.direct_sum(rd, pf, far, 0, 2) == 0)


# --------------------------------------------------------------------------- fast mode
def _small_scene(L=48, seed=11):
    return sg.sea_surface(L, seed)


@pytest.mark.parametrize("window", ["sqrt_linear", "sqrt_raised_cosine", "linear"])
def test_update_pulse_identity(orc, window):
    """At x = p_i the blend is W_i = 1, W_{i+1} = 0 and m = 0, so the fast-mode pulse
    equals the regular-mode pulse exactly (Eq. (1), Sec. III.B steps 2-4)."""
    rd = sg.RadarParams()
    n_pulses, nf, nd = 256, 64, 64
    pf = sg.nadir_track(n_pulses)
    sc = _small_scene()
    T, Y = orc.simulate_fast(rd, pf, sc, n_pulses, nf, nd, window)
    for i in range(n_pulses // nf):
        yr = orc.direct_sum(rd, pf, sc, i * nf, 1)[0]
        np.testing.assert_allclose(Y[i * nf], yr, rtol=0, atol=1e-12 * np.abs(yr).max())
    # ... while between updates the two modes differ (the method is an approximation)
    yr = orc.direct_sum(rd, pf, sc, 32, 1)[0]
    assert np.abs(Y[32] - yr).max() > 1e-6 * np.abs(yr).max()


@pytest.mark.parametrize("window", ["sqrt_linear", "sqrt_raised_cosine", "linear"])
def test_static_scene(orc, window):
    """Nothing moves: every spectrum is a DC line, every segment is constant, so
    Y_fast[x] = (W_i(x) + W_{i+1}(x)) Y_reg[x]; exact for the linear window."""
    rd = sg.RadarParams()
    sc = _small_scene(32, 5)
    for k in ("vx", "vy", "vz"):
        sc[k] = np.zeros_like(sc[k])
    pf = static_platform()
    nf, nd, P = 16, 16, 48
    T, Y = orc.simulate_fast(rd, pf, sc, P, nf, nd, window)
    assert np.all(T[..., 1:] == 0)
    yr = orc.direct_sum(rd, pf, sc, 0, 1)[0]
    for x in range(P):
        u = (x % nf) / nf
        if window == "sqrt_linear":
            w = math.sqrt(1 - u) + math.sqrt(u)
        elif window == "sqrt_raised_cosine":
            w = math.cos(math.pi * u / 2) + math.sin(math.pi * u / 2)
        else:
            w = 1.0
        np.testing.assert_allclose(Y[x], w * yr, rtol=0, atol=1e-12 * np.abs(yr).max())


@pytest.mark.parametrize("k0", [5, -5, 1, -3, 31, -32])
@pytest.mark.parametrize("window", ["sqrt_linear", "linear"])
def test_on_bin_tone(orc, k0, window):
    """One scatterer whose phase advances by exactly k0/N_d cycles per pulse: the spectrum
    is a single line in bin k0 mod N_d and the segments reproduce the true signal, so
    Y_fast = (W_i + W_{i+1}) Y_reg.  Pins the Doppler sign, the inverse-transform sign
    and the segment time origin."""
    rd = sg.RadarParams()
    nd, nf = 64, 64
    P = 192 if abs(k0) <= 8 else 64
    lam = rd.c_mps / rd.carrier_hz
    vz = k0 * lam * rd.prf_hz / (2 * nd)   # R = H - z - vz t: phase advance 2 vz/(lam PRF) cyc/pulse
    # start so that the scatterer stays inside gate 64 over the P pulses it is simulated
    travel = abs(vz) * (P / rd.prf_hz) / rd.gate_width_m
    gc0 = 64.5 + math.copysign(travel / 2, k0)
    z0 = -(gc0 - 64) * rd.gate_width_m
    sc = sg.point_scene([(0.0, 0.0, z0, 0.0, 0.0, vz, 0.3)])
    pf = static_platform()
    T, Y = orc.simulate_fast(rd, pf, sc, P, nf, nd, window)
    nzs = np.argwhere(np.abs(T) > 0)
    assert {tuple(v[1:]) for v in nzs} == {(64, k0 % nd)}
    Yr = orc.direct_sum(rd, pf, sc, 0, P)
    for x in range(P):
        u = (x % nf) / nf
        w = (math.sqrt(1 - u) + math.sqrt(u)) if window == "sqrt_linear" else 1.0
        np.testing.assert_allclose(Y[x, 64], w * Yr[x, 64], rtol=2e-5)


def test_parseval_and_dft_vs_numpy(orc):
    """Unnormalised inverse transform: equals N_d * numpy.fft.ifft, and
    sum_m |s|^2 = N_d sum_k |T|^2; its adjoint is numpy.fft.fft."""
    T = sg.random_spectra(3, 5, 64, seed=7)
    s = orc.ifft(T)
    np.testing.assert_allclose(s, np.fft.ifft(T, axis=-1) * 64, atol=1e-12)
    np.testing.assert_allclose((np.abs(s) ** 2).sum(-1), 64 * (np.abs(T) ** 2).sum(-1), rtol=1e-12)
    np.testing.assert_allclose(orc.dft(s), np.fft.fft(s, axis=-1), atol=1e-10)
    T8 = sg.random_spectra(2, 3, 8, seed=8)
    np.testing.assert_allclose(orc.ifft(T8), np.fft.ifft(T8, axis=-1) * 8, atol=1e-13)


def test_incoherent_power_proportional_to_summed_nrcs(orc):
    """Random heights (sigma_h >> lambda) make the phases uniform, so the mean gate power
    over realizations equals the summed NRCS x area of the scatterers in the window
    (Sec. II.A: raw data as a sum of many illuminated scatterers)."""
    rd = sg.RadarParams()
    pf = static_platform()
    M, L = 192, 24
    rng = np.random.Generator(np.random.PCG64(99))
    ratio = []
    xs = (np.arange(L) - (L - 1) / 2).astype(np.float32)
    for _ in range(M):
        z = rng.normal(0.0, 1.0, size=L * L).astype(np.float32)
        sigma = np.exp(rng.normal(-2, 0.5, size=L * L)).astype(np.float32)
        sc = {"x": np.tile(xs, L), "y": np.repeat(xs, L), "z": z, "vx": np.zeros(L * L, np.float32),
              "vy": np.zeros(L * L, np.float32), "vz": np.zeros(L * L, np.float32), "nrcs": sigma,
              "origin": (0, 0, 0), "area": 1.0}
        Y = orc.direct_sum(rd, pf, sc, 0, 1)[0]
        ratio.append(((np.abs(Y) ** 2).sum(), float(sigma.astype(np.float64).sum())))
    p, s = np.array(ratio).T
    r = p.sum() / s.sum()
    # ~10 occupied gates x M exponential draws: relative std ~ 1/sqrt(10 M) ~ 2.3 %
    assert abs(r - 1.0) < 0.1


@pytest.mark.parametrize("window,flat", [("sqrt_linear", True), ("sqrt_raised_cosine", True),
                                         ("linear", False)])
def test_variance_conservation_eq1(orc, window, flat):
    """Remark after Eq. (1): the 1/2 power keeps the total variance constant on average.
    With independent random spectra E|Y[x]|^2 = N_d (W_i^2 + W_{i+1}^2): flat for the
    power-complementary windows, halved mid-segment for a linear amplitude crossfade."""
    nd, nf, S, G = 16, 16, 33, 64
    T = sg.random_spectra(S, G, nd, seed=3)
    Y = orc.synth(T, 0, nf, 0, (S - 1) * nf, window)
    pw = (np.abs(Y) ** 2).reshape(S - 1, nf, G).mean(axis=(0, 2)) / nd
    if flat:
        assert np.all(np.abs(pw - 1.0) < 0.12)
    else:
        assert abs(pw[nf // 2] - 0.5) < 0.06 and abs(pw[0] - 1.0) < 0.12


def test_window_golden_eq1(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "eq1_weights.txt"))
            if l.strip() and not l.startswith("#")]
    for nf, dist, w in rows:
        assert orc.window("sqrt_linear", int(dist) / int(nf)) == pytest.approx(float(w), abs=1e-15)
    for d in np.linspace(0, 1, 11):
        for win in ("sqrt_linear", "sqrt_raised_cosine"):
            w0, w1 = orc.window(win, d), orc.window(win, 1 - d)
            assert w0 ** 2 + w1 ** 2 == pytest.approx(1.0, abs=1e-15)
    assert orc.window("sqrt_raised_cosine", 1.0) == 0.0 and orc.window("sqrt_linear", 1.5) == 0.0


def test_paper_scenario_golden():
    g = json.load(open(os.path.join(GOLDEN, "paper_scenario.json")))
    assert abs(g["n_tiles"] * g["tile_side"] ** 2 - g["n_scatterers"]) / g["n_scatterers"] < 1e-3
    # pulses over the track at the satellite speed implied by PRF and track length
    speed = g["track_km"] * 1e3 / (g["n_pulses"] / g["prf_hz_scenario"])
    assert 6500 < speed < 7000
    for nf in g["n_fast_sweep"][1:]:
        S = n_spectra(g["n_pulses"], nf)
        assert S == math.ceil(1 + g["n_pulses"] / nf) or S == 1 + g["n_pulses"] // nf + 1
        assert S >= 1 + g["n_pulses"] / nf


# --------------------------------------------------------------------------- brute force
def test_c_oracle_matches_numpy_bruteforce(orc):
    rd = sg.RadarParams(n_gates=64)
    n_pulses, nf, nd = 96, 32, 32
    pf = sg.nadir_track(n_pulses)
    sc = _small_scene(40, 21)
    Yc = orc.direct_sum(rd, pf, sc, 5, 7)
    Yb = bf.direct_sum(rd, pf, sc, 5, 7)
    np.testing.assert_allclose(Yc, Yb, rtol=0, atol=1e-12 * np.abs(Yb).max())
    Tc = orc.doppler_spectra(rd, pf, sc, 0, 4, nf, nd)
    Tb = bf.doppler_spectra(rd, pf, sc, 0, 4, nf, nd)
    np.testing.assert_allclose(Tc, Tb, rtol=0, atol=1e-12 * np.abs(Tb).max())
    for w in ("sqrt_linear", "sqrt_raised_cosine", "linear"):
        np.testing.assert_allclose(orc.synth(Tc, 0, nf, 3, 90, w), bf.synth(Tc, 0, nf, 3, 90, w),
                                   rtol=0, atol=1e-12 * np.abs(Tc).max() * nd)
    gate, bins, gc, bc = orc.cells(rd, pf, sc, 17, nd)
    C1, dR, _ = bf.echo(rd, pf, sc, 17 / rd.prf_hz)
    C2, _, _ = bf.echo(rd, pf, sc, 18 / rd.prf_hz)
    np.testing.assert_array_equal(gate, bf.gates(rd, dR))
    np.testing.assert_array_equal(bins, bf.doppler_bins(rd, C1, C2, nd))


def test_empty_scene(orc):
    rd = sg.RadarParams()
    pf = sg.nadir_track(64)
    sc = {k: np.zeros(0, np.float32) for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs")}
    assert np.all(orc.direct_sum(rd, pf, sc, 0, 3) == 0)
    assert np.all(orc.doppler_spectra(rd, pf, sc, 0, 2, 64, 64) == 0)


def test_decided_cell_variants_reproduce_the_oracle(orc):
    """With the oracle's own decisions, the decided-cell variants give the same sums."""
    rd = sg.RadarParams()
    P, nf, nd = 128, 32, 32
    pf = sg.nadir_track(P)
    sc = _small_scene(40, 9)
    gates = np.stack([orc.cells(rd, pf, sc, p, nd)[0] for p in range(3, 9)])
    np.testing.assert_array_equal(orc.direct_sum_cells(rd, pf, sc, 3, gates),
                                  orc.direct_sum(rd, pf, sc, 3, 6))
    cells = [orc.cells(rd, pf, sc, u * nf, nd) for u in range(1, 4)]
    G = np.stack([c[0] for c in cells])
    B = np.stack([c[1] for c in cells])
    np.testing.assert_array_equal(orc.doppler_spectra_cells(rd, pf, sc, 1, nf, nd, G, B),
                                  orc.doppler_spectra(rd, pf, sc, 1, 3, nf, nd))


def test_state_epoch(orc):
    """A state given at epoch t0 is the same physical surface as the state moved back to
    epoch 0 (r - v t0): identical sums up to the rounding of the moved positions."""
    rd = sg.RadarParams()
    pf = sg.nadir_track(512)
    sc = _small_scene(32, 31)
    t0 = 0.0123
    moved = dict(sc)
    for k, vk in (("x", "vx"), ("y", "vy"), ("z", "vz")):
        moved[k] = (sc[k].astype(np.float64) - sc[vk].astype(np.float64) * t0)
    shifted = dict(sc, t0=t0)
    # the moved positions are float32 inputs too: compare through the brute force in float64
    Yb = bf.direct_sum(rd, pf, {**moved, **{k: moved[k] for k in ("x", "y", "z")}}, 200, 3)
    Ys = orc.direct_sum(rd, pf, shifted, 200, 3)
    Yb2 = bf.direct_sum(rd, pf, shifted, 200, 3)
    np.testing.assert_allclose(Ys, Yb2, rtol=0, atol=1e-12 * np.abs(Ys).max())
    # moved positions rounded to float32 differ by <= 3e-8 m: phase within ~2e-5 rad
    assert np.abs(Ys - Yb).max() < 1e-4 * np.abs(Ys).max()


def test_galilean_invariance_of_the_stop_and_hop_geometry(orc):
    """Only the platform-to-scatterer vector d(t) = P(t) - s(t) enters an echo (range, gate,
    phase, pattern angle, pulse-pair Doppler), so a static scene under a platform moving at
    V and a static platform over a scene moving at -V give the same cells, the same IQ and
    the same spectra.  The scene sits 2 km along track, so its echoes carry a Doppler of
    several bins (about 2 V sin(theta) / lambda = 1.6 kHz)."""
    rd = sg.RadarParams()
    V = 7000.0
    sc = sg.sea_surface(20, 3)
    static = dict(sc, vx=np.zeros_like(sc["vx"]), vy=np.zeros_like(sc["vy"]),
                  vz=np.zeros_like(sc["vz"]))
    moving = dict(static, vx=np.full_like(sc["vx"], -V))
    pf_moving = sg.PlatformParams(p0=(-2000.0, 0.0, H), v=(V, 0.0, 0.0), r_ref0=H, r_ref_rate=0.0)
    pf_static = sg.PlatformParams(p0=(-2000.0, 0.0, H), v=(0.0, 0.0, 0.0), r_ref0=H,
                                  r_ref_rate=0.0)
    nf, nd = 8, 64
    for p in (0, 24, 57):
        ga, ba, _, _ = orc.cells(rd, pf_moving, static, p, nd)
        gb, bb, _, _ = orc.cells(rd, pf_static, moving, p, nd)
        np.testing.assert_array_equal(ga, gb)
        np.testing.assert_array_equal(ba, bb)
        assert (ga >= 0).all() and (ga < rd.n_gates).all()
        assert 3 <= np.median(ba) <= 8           # about nu N_d = 1.6 kHz / 18 kHz x 64 = 5.6
    Ya = orc.direct_sum(rd, pf_moving, static, 0, 64)
    Yb = orc.direct_sum(rd, pf_static, moving, 0, 64)
    assert np.abs(Ya).max() > 0
    assert np.linalg.norm(Ya - Yb) < 1e-6 * np.linalg.norm(Ya)
    Ta = orc.doppler_spectra(rd, pf_moving, static, 0, 8, nf, nd)
    Tb = orc.doppler_spectra(rd, pf_static, moving, 0, 8, nf, nd)
    assert np.linalg.norm(Ta - Tb) < 1e-6 * np.linalg.norm(Ta)
    # the platform's motion is really seen: the echo changes along the run
    assert np.linalg.norm(Ya[0] - Ya[-1]) > 0.1 * np.linalg.norm(Ya[0])


def test_sums_do_not_depend_on_the_thread_count():
    """The oracle sums over a fixed number of scatterer chunks and merges them in chunk
    order, so its results are the same bits however many threads run."""
    import oracle
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    sc = sg.sea_surface(150, 17)                      # 22,500 scatterers over all the chunks
    orc = oracle.Oracle()
    before = orc.threads                              # the thread count is process-wide
    out = []
    try:
        for threads in (1, 4):
            orc.set_threads(threads)
            assert orc.threads == threads
            out.append((orc.direct_sum(rd, pf, sc, 2040, 3),
                        orc.doppler_spectra(rd, pf, sc, 31, 2, fp.n_fast, fp.n_doppler)))
    finally:
        orc.set_threads(before)
    assert np.abs(out[0][0]).max() > 0 and np.abs(out[0][1]).max() > 0
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


# --------------------------------------------------------------------------- index coordinates
def _decimal_coords(radar, platform, scene, idx, pulse, n_doppler):
    """Gate coordinate dR / gate_width + N_g / 2 at `pulse` and pulse-pair bin coordinate
    nu N_d + 1/2 of Algorithm 1 (nu = phase advance of C over the pair (pulse, pulse + 1),
    cycles, wrapped to [-1/2, 1/2)) for the scatterers `idx`, in 60-digit decimal arithmetic
    straight from the definitions: positions, ranges and phases psi = 2 R / lambda at both
    pulses, and the difference psi1 - psi2 of the two phases.  The float inputs convert to
    decimal exactly."""
    import decimal
    from decimal import Decimal as D
    ctx = decimal.Context(prec=60)
    prf, lam = D(radar.prf_hz), ctx.divide(D(radar.c_mps), D(radar.carrier_hz))
    t0 = D(float(scene.get("t0", 0.0)))
    org = [D(float(v)) for v in scene.get("origin", (0.0, 0.0, 0.0))]

    def state(n, p):
        t = ctx.divide(D(p), prf)
        ts = t - t0
        s = [org[0] + D(float(scene["x"][n])) + D(float(scene["vx"][n])) * ts,
             org[1] + D(float(scene["y"][n])) + D(float(scene["vy"][n])) * ts,
             org[2] + D(float(scene["z"][n])) + D(float(scene["vz"][n])) * ts]
        P = [D(platform.p0[i]) + D(platform.v[i]) * t for i in range(3)]
        R = ctx.sqrt(sum((P[i] - s[i]) * (P[i] - s[i]) for i in range(3)))
        rref = D(platform.r_ref0) + D(platform.r_ref_rate) * t
        return R, rref

    gc, bc = [], []
    for n in idx:
        R1, rref = state(n, pulse)
        R2, _ = state(n, pulse + 1)
        gc.append(float(ctx.divide(R1 - rref, D(radar.gate_width_m)) + D(radar.n_gates) / 2))
        nu = ctx.divide(2 * (R1 - R2), lam)                 # psi1 - psi2
        nu -= (nu + D("0.5")).to_integral_value(rounding=decimal.ROUND_FLOOR)
        bc.append(float(nu * n_doppler + D("0.5")))
    return np.array(gc), np.array(bc)


@pytest.mark.parametrize("pulse", [0, 1984, 4095])
def test_index_coordinates_against_high_precision(orc, pulse):
    """The oracle's pre-floor gate and Doppler-bin coordinates (the quantities whose floors
    are Algorithm 1's rasterisation indices) against a 60-digit evaluation of their
    definitions on a moving sea surface seen along the cfg1 track: gate to 1e-11, bin to
    1e-10 (mod N_d).  A dropped velocity component, a flipped or halved phase difference,
    or a range change taken over the wrong interval fails it; so would the rounding noise
    of a difference of two FP64 ranges of ~8e5 m (~5e-10 gates) or of the two ~7e7-cycle
    phases (~1e-6 bins), which the oracle's rewritten differences avoid."""
    c = sg.config(1)
    rd, pf, nd = c["radar"], c["platform"], c["fast"].n_doppler
    sc = sg.sea_surface(64, 31)
    g, b, gc, bc = orc.cells(rd, pf, sc, pulse, nd)
    idx = np.random.Generator(np.random.PCG64(pulse + 5)).choice(sc["x"].size, 60, replace=False)
    gx, bx = _decimal_coords(rd, pf, sc, idx, pulse, nd)
    assert np.abs(gc[idx] - gx).max() < 1e-11
    db = np.abs(bc[idx] - bx)
    db = np.minimum(db, nd - db)
    assert db.max() < 1e-10
    assert np.array_equal(g[idx], np.floor(gx).astype(np.int64))
    assert np.array_equal(b[idx], np.mod(np.floor(bx).astype(np.int64), nd))
    # the scene's Doppler spreads over several bins, so the bin coordinate is exercised
    assert np.ptp(np.mod(np.floor(bx), nd)) >= 1
