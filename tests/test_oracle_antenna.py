"""Pins of the oracle's tabulated antenna pattern (Section II.A: every antenna pattern is
recorded on a u-v grid and its complex value at each facet is obtained by interpolation in
that grid).  Reading: bilinear interpolation of the real and imaginary parts at the facet's
direction cosines u = (s - P)_x / R, v = (s - P)_y / R; zero outside the grid."""
import math
from fractions import Fraction

import dataclasses
import numpy as np
import pytest

import scenegen as sg
from oracle import bruteforce as bf

H = 800e3


def _table(fn, u0, v0, du, dv, nu, nv):
    u = u0 + du * np.arange(nu)
    v = v0 + dv * np.arange(nv)
    return sg.AntennaTable(gain=fn(u[None, :], v[:, None]), u0=u0, du=du, v0=v0, dv=dv)


def test_bilinear_reproduces_linear_tables(orc):
    """A pattern linear in u and v is interpolated exactly, with its slopes as derivatives;
    outside the grid the gain is zero."""
    a, b, c = 0.7 - 0.2j, 3.0 + 1.5j, -2.0 + 0.25j
    tab = _table(lambda u, v: a + b * u + c * v, -0.5, -0.25, 0.125, 0.0625, 9, 11)
    rd = sg.RadarParams(antenna=tab)
    rng = np.random.Generator(np.random.PCG64(3))
    for u, v in zip(rng.uniform(-0.5, 0.5, 50), rng.uniform(-0.25, 0.375, 50)):
        g, gu, gv = orc.antenna_gain(rd, u, v)
        assert g == pytest.approx(a + b * u + c * v, abs=1e-14)
        assert gu == pytest.approx(b, abs=1e-12) and gv == pytest.approx(c, abs=1e-12)
    for u, v in ((-0.5 - 1e-9, 0.0), (0.5, 0.0), (0.0, -0.25 - 1e-9), (0.0, 0.375), (2.0, 2.0)):
        assert orc.antenna_gain(rd, u, v) == (0j, 0j, 0j)


def test_bilinear_at_nodes_and_cell_centres(orc):
    rng = np.random.Generator(np.random.PCG64(7))
    g = rng.standard_normal((6, 5)) + 1j * rng.standard_normal((6, 5))
    tab = sg.AntennaTable(gain=g, u0=-1.0, du=0.25, v0=0.5, dv=0.5)
    rd = sg.RadarParams(antenna=tab)
    for j in range(5):
        for i in range(4):
            u, v = -1.0 + 0.25 * i, 0.5 + 0.5 * j
            assert orc.antenna_gain(rd, u, v)[0] == g[j, i]
            centre = orc.antenna_gain(rd, u + 0.125, v + 0.25)[0]
            assert centre == pytest.approx((g[j, i] + g[j, i + 1] + g[j + 1, i] + g[j + 1, i + 1]) / 4,
                                           abs=1e-15)


def test_point_scatterers_see_the_pattern_at_their_direction_cosines(orc):
    """Static platform at (0, 0, H): a facet at (x, y, 0) has u = x / R, v = y / R.  With
    G = 1 + kappa u + j mu v (exact under bilinear interpolation) the echo is
    sqrt(sigma A) (H/R)^2 G e^{-j 4 pi R / lambda}: pins the orientation and sign of u, v."""
    kappa, mu = 40.0, -25.0
    tab = _table(lambda u, v: 1.0 + kappa * u + 1j * mu * v, -0.02, -0.02, 0.001, 0.001, 41, 41)
    rd = sg.RadarParams(antenna=tab)
    pf = sg.PlatformParams(p0=(0.0, 0.0, H), v=(0.0, 0.0, 0.0), r_ref0=H, r_ref_rate=0.0)
    pts = [(1500.0, 0.0, 0.0), (0.0, -900.0, 0.0), (-700.0, 1100.0, 0.0), (250.0, 333.0, 0.0)]
    sigma, area = 0.5, 1.0
    sc = sg.point_scene([(x, y, z, 0.0, 0.0, 0.0, sigma) for x, y, z in pts], area=area)
    e = orc.echo(rd, pf, sc, 0.0)
    for j, (x, y, _) in enumerate(pts):
        xf, yf = float(np.float32(x)), float(np.float32(y))
        R_exact = Fraction(xf) ** 2 + Fraction(yf) ** 2 + Fraction(H) ** 2
        R = math.sqrt(float(R_exact))
        u, v = xf / R, yf / R
        cyc = Fraction(2) * Fraction(R) * Fraction(rd.carrier_hz) / Fraction(rd.c_mps)
        phase = -2 * math.pi * float(cyc - round(cyc))
        want = math.sqrt(float(np.float32(sigma)) * area) * (H / R) ** 2 * (1 + kappa * u + 1j * mu * v)
        want *= complex(math.cos(phase), math.sin(phase))
        # amplitude to rounding; phase within the rounding of a 7e7-cycle two-way range
        assert abs(e["C"][j]) == pytest.approx(abs(want), rel=1e-12)
        dphi = (np.angle(e["C"][j]) - np.angle(want) + math.pi) % (2 * math.pi) - math.pi
        assert abs(dphi) < 2e-7


def test_table_sampled_from_the_gaussian_pattern_matches_it(orc):
    """Nodes sampled from the analytic two-way pattern exp(-2 ln2 theta^2 / theta_b^2),
    theta = asin(sqrt(u^2 + v^2)): the direct sum with the table differs from the analytic
    one only by the bilinear interpolation error, at most du^2/8 |w_uu| + dv^2/8 |w_vv|."""
    rd0 = sg.RadarParams()
    c = 2.0 * math.log(2.0) / rd0.beamwidth_rad ** 2
    d = 1e-4

    def w(u, v):
        return np.exp(-c * np.arcsin(np.sqrt(u ** 2 + v ** 2)) ** 2) + 0j

    tab = _table(w, -0.004, -0.004, d, d, 81, 81)
    rd = dataclasses.replace(rd0, antenna=tab)
    P = 32
    pf = sg.nadir_track(P)
    sc = sg.sea_surface(48, 9)
    Y0 = orc.direct_sum(rd0, pf, sc, 0, P)
    Y1 = orc.direct_sum(rd, pf, sc, 0, P)
    bound = 2 * d * d / 8 * 2 * c * 1.01           # |w_uu|, |w_vv| <= 2c near boresight
    err = np.abs(Y1 - Y0).max() / np.abs(Y0).max()
    assert 0 < err < bound


def test_c_oracle_matches_numpy_bruteforce_with_table(orc):
    rd = sg.RadarParams(n_gates=64, antenna=sg.antenna_table(5, n=65, half_width=0.01))
    n_pulses, nf, nd = 96, 32, 32
    pf = sg.nadir_track(n_pulses)
    sc = sg.sea_surface(40, 21)
    Yc = orc.direct_sum(rd, pf, sc, 5, 7)
    Yb = bf.direct_sum(rd, pf, sc, 5, 7)
    np.testing.assert_allclose(Yc, Yb, rtol=0, atol=1e-12 * np.abs(Yb).max())
    Tc = orc.doppler_spectra(rd, pf, sc, 0, 4, nf, nd)
    Tb = bf.doppler_spectra(rd, pf, sc, 0, 4, nf, nd)
    np.testing.assert_allclose(Tc, Tb, rtol=0, atol=1e-12 * np.abs(Tb).max())
    # the table changes the result (the pattern is not the analytic one)
    Yg = orc.direct_sum(dataclasses.replace(rd, antenna=None), pf, sc, 5, 7)
    assert np.abs(Yg - Yc).max() > 1e-3 * np.abs(Yc).max()


def test_pulse_pair_bin_carries_the_pattern_phase_change(orc):
    """Algorithm 1 takes D_i from arg(conj(C_{i+1}) C_i), and C carries the pattern, so the
    pattern's own phase change between the facet's directions at the two pulses is part of
    the Doppler.  A table whose phase ramps in u (G = e^{j 2 pi kappa u}, ~0.2 bins of phase
    change per PRI along the track): the oracle's bin coordinate against the numpy
    restatement's literal angle of C_{i+1} conj(C_i), to 2e-5 bins (that difference of two
    ~7e7-cycle phases carries ~1e-6); the pattern's share is ~0.2 bins, so a dropped or
    reversed pattern term fails."""
    kappa, nd = 1.29e4, 32
    tab = _table(lambda u, v: np.exp(2j * np.pi * kappa * u) + 0.0 * v, -2e-4, -2e-4, 4e-6, 4e-6,
                 101, 101)
    rd = sg.RadarParams(antenna=tab)
    pf = sg.nadir_track(96)
    sc = sg.sea_surface(40, 22)
    for p in (0, 47, 95):
        _, _, _, bc = orc.cells(rd, pf, sc, p, nd)
        C1, _, _ = bf.echo(rd, pf, sc, p / rd.prf_hz)
        C2, _, _ = bf.echo(rd, pf, sc, (p + 1) / rd.prf_hz)
        lit = np.angle(C2 * np.conj(C1)) / (2 * np.pi) * nd + 0.5
        d = np.mod(bc - lit, nd)
        assert np.minimum(d, nd - d).max() < 2e-5
        _, _, _, bc_g = orc.cells(dataclasses.replace(rd, antenna=None), pf, sc, p, nd)
        d = np.mod(bc - bc_g, nd)
        share = np.minimum(d, nd - d)
        assert 0.1 < share.min() and share.max() < 0.3


def test_gradient_with_table_vs_central_differences(orc):
    rd = sg.RadarParams(antenna=sg.antenna_table(11, n=65, half_width=0.01))
    P, nf, nd = 128, 64, 64
    pf = sg.nadir_track(P)
    sc = sg.sea_surface(24, 4)
    S = (P - 1) // nf + 2

    def forward(scene):
        T = orc.doppler_spectra(rd, pf, scene, 0, S, nf, nd)
        return orc.synth(T, 0, nf, 0, P, "sqrt_raised_cosine")

    Y = forward(sc)
    target = sg.target_waveform(P, rd.n_gates, 4242, (np.abs(Y) ** 2).mean(axis=0))

    def loss(Yx):
        return float(((np.abs(Yx) ** 2 - target) ** 2).sum())

    GY = 4.0 * (np.abs(Y) ** 2 - target) * Y
    GT = orc.synth_grad(GY, S, 0, nf, nd, 0, "sqrt_raised_cosine")
    gz, gs = orc.fast_grad(rd, pf, sc, 0, nf, GT)
    ok = np.ones(sc["x"].size, bool)
    for i in range(S):
        g, b, gc, bc = orc.cells(rd, pf, sc, i * nf, nd)
        ok &= (g >= 0) & (g < rd.n_gates)
        ok &= (np.abs(gc - np.round(gc)) > 2e-3) & (np.abs(bc - np.round(bc)) > 2e-2)
    picks = np.random.Generator(np.random.PCG64(6)).choice(np.nonzero(ok)[0], 6, replace=False)
    h = 2.0 ** -16
    for n in picks:
        for key, grad, step in (("z", gz, h), ("nrcs", gs, None)):
            v0 = sc[key][n]
            vp = np.float32(v0 + step) if step else np.float32(v0 * (1 + 2 ** -10))
            vm = np.float32(v0 - step) if step else np.float32(v0 * (1 - 2 ** -10))
            sp, sm = dict(sc), dict(sc)
            sp[key] = sc[key].copy()
            sm[key] = sc[key].copy()
            sp[key][n], sm[key][n] = vp, vm
            fd = (loss(forward(sp)) - loss(forward(sm))) / (float(vp) - float(vm))
            # central differences of a ~600 rad/m phase carry ~1e-5 of the largest gradient
            assert grad[n] == pytest.approx(fd, rel=2e-4, abs=5e-5 * np.abs(grad).max())


def test_pattern_term_of_the_adjoint(orc):
    """With one scatterer, L = sum_p |Y_p|^2 = sum_p |C_p|^2 does not see the phase, so its
    z-gradient is 2 sum |C|^2 d ln|C|/dz = 2 sum |C|^2 (2 d_z / R^2 + Re(dG/dz / G)).  A
    pattern G = 1 + kappa u with a steep slope makes the pattern term a large part of it;
    the adjoint must match central differences of L."""
    kappa = 800.0
    tab = _table(lambda u, v: (1.0 + kappa * u) + 0.0 * v, -0.01, -0.01, 0.0005, 0.0005, 41, 41)
    rd = sg.RadarParams(antenna=tab)
    pf = sg.PlatformParams(p0=(-50.0, 0.0, H), v=(7000.0, 0.0, 0.0), r_ref0=H - 0.3, r_ref_rate=0.0)
    sc = sg.point_scene([(900.0, 150.0, 0.2, 0.1, 0.0, 0.3, 0.8)], area=1.0)
    P = 16

    def loss(z):
        s = dict(sc)
        s["z"] = np.array([z], np.float32)
        return float((np.abs(orc.direct_sum(rd, pf, s, 0, P)) ** 2).sum())

    Y = orc.direct_sum(rd, pf, sc, 0, P)
    gz, _ = orc.direct_grad(rd, pf, sc, 0, 2.0 * Y)
    h = 2.0 ** -8
    z0 = float(sc["z"][0])
    fd = (loss(np.float32(z0 + h)) - loss(np.float32(z0 - h))) / (2 * h)
    assert gz[0] == pytest.approx(fd, rel=1e-5)
    # without the pattern term the gradient would be the range term alone
    R = np.hypot(np.hypot(900.0 - (-50.0), 150.0), H)
    range_only = 2 * float((np.abs(Y) ** 2).sum()) * 2 * (H - 0.2) / R ** 2
    assert abs(gz[0] - range_only) > 0.1 * abs(gz[0])
