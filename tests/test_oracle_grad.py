"""Pins of the oracle's adjoint: dot-product test of the post-processing adjoint and
central finite differences of a waveform-power loss w.r.t. heights and NRCS."""
import numpy as np
import pytest

import scenegen as sg


def _loss_and_grad_y(Y, target):
    pw = np.abs(Y) ** 2
    return float(((pw - target) ** 2).sum()), 4.0 * (pw - target) * Y


def _safe_scatterers(orc, rd, pf, sc, pulses, nd, count, seed):
    """Scatterers whose gate and bin coordinates stay well away from integer edges."""
    ok = np.ones(sc["x"].size, bool)
    for p in pulses:
        g, b, gc, bc = orc.cells(rd, pf, sc, p, nd)
        ok &= (g >= 0) & (g < rd.n_gates)
        ok &= np.abs(gc - np.round(gc)) > 2e-3
        ok &= np.abs(bc - np.round(bc)) > 2e-2
    idx = np.nonzero(ok)[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.choice(idx, size=count, replace=False)


def _perturbed(sc, key, n, value):
    s2 = dict(sc)
    a = sc[key].copy()
    a[n] = value
    s2[key] = a
    return s2


def test_synth_adjoint_dot_product(orc):
    """<G_Y, synth(T)> = <synth_grad(G_Y), T> (real inner product Re sum conj(a) b)."""
    S, G, nd, nf = 5, 7, 16, 12
    T = sg.random_spectra(S, G, nd, seed=1)
    P = (S - 2) * nf + 5
    GY = sg.random_iq(P, G, seed=2)
    for w in ("sqrt_linear", "sqrt_raised_cosine", "linear"):
        Y = orc.synth(T, 0, nf, 3, P, w)
        GT = orc.synth_grad(GY, S, 0, nf, nd, 3, w)
        lhs = np.real(np.vdot(GY, Y))
        rhs = np.real(np.vdot(GT, T))
        assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("mode", ["fast", "regular"])
def test_gradient_vs_central_differences(orc, mode):
    rd = sg.RadarParams()
    P, nf, nd = 128, 64, 64
    pf = sg.nadir_track(P)
    sc = sg.sea_surface(24, 4)
    S = (P - 1) // nf + 2

    def forward(scene):
        if mode == "fast":
            T = orc.doppler_spectra(rd, pf, scene, 0, S, nf, nd)
            return orc.synth(T, 0, nf, 0, P, "sqrt_raised_cosine")
        return orc.direct_sum(rd, pf, scene, 0, P)

    Y = forward(sc)
    target = sg.target_waveform(P, rd.n_gates, 4242, (np.abs(Y) ** 2).mean(axis=0))
    L0, GY = _loss_and_grad_y(Y, target)
    if mode == "fast":
        GT = orc.synth_grad(GY, S, 0, nf, nd, 0, "sqrt_raised_cosine")
        gz, gs = orc.fast_grad(rd, pf, sc, 0, nf, GT)
        pulses = [i * nf for i in range(S)]
    else:
        gz, gs = orc.direct_grad(rd, pf, sc, 0, GY)
        pulses = list(range(0, P, 7))
    picks = _safe_scatterers(orc, rd, pf, sc, pulses, nd, 6, seed=5)
    h = 2.0 ** -16
    for n in picks:
        z0 = sc["z"][n]
        zp, zm = np.float32(z0 + h), np.float32(z0 - h)
        Lp, _ = _loss_and_grad_y(forward(_perturbed(sc, "z", n, zp)), target)
        Lm, _ = _loss_and_grad_y(forward(_perturbed(sc, "z", n, zm)), target)
        fd = (Lp - Lm) / (float(zp) - float(zm))
        assert gz[n] == pytest.approx(fd, rel=2e-4, abs=1e-6 * np.abs(gz).max())
        s0 = sc["nrcs"][n]
        sp, sm = np.float32(s0 * (1 + 2 ** -10)), np.float32(s0 * (1 - 2 ** -10))
        Lp, _ = _loss_and_grad_y(forward(_perturbed(sc, "nrcs", n, sp)), target)
        Lm, _ = _loss_and_grad_y(forward(_perturbed(sc, "nrcs", n, sm)), target)
        fd = (Lp - Lm) / (float(sp) - float(sm))
        assert gs[n] == pytest.approx(fd, rel=2e-4, abs=1e-6 * np.abs(gs).max())


@pytest.mark.parametrize("x0", [0.0, 6000.0, 10000.0])
def test_amplitude_derivative_of_a_lone_scatterer(orc, x0):
    """The amplitude part of dC/dz is about 1e-8 of the phase part, so the waveform-power
    finite differences above cannot see it.  For one scatterer alone in its gate the loss
    L = |Y|^2 = a^2 carries no phase: the adjoint with dL/dY = 2 Y returns 2 a^2 d ln a / dz
    exactly, which central differences of L check here -- at nadir (range factor
    (r_ref / R)^2 alone) and 6 and 10 km off nadir, where the beam term
    d ln w / dz = -4 ln2 theta rho / (theta_b^2 R^2) reaches 15 % and 40 % of it."""
    rd = sg.RadarParams()
    H = 800e3
    z0, h = 0.25, 2.0 ** -8                              # z0 +- h exact in float32
    R = float(np.hypot(x0, H - z0))
    pf = sg.PlatformParams(p0=(0.0, 0.0, H), v=(0.0, 0.0, 0.0), r_ref0=R + 0.2, r_ref_rate=0.0)

    def scene(z):
        return sg.point_scene([(x0, 0.0, z, 0.0, 0.0, 0.0, 0.3)])

    def loss(z):
        return float((np.abs(orc.direct_sum(rd, pf, scene(z), 0, 1)) ** 2).sum())

    Y = orc.direct_sum(rd, pf, scene(z0), 0, 1)
    assert np.count_nonzero(Y) == 1                       # one gate, mid-gate
    gz, gs = orc.direct_grad(rd, pf, scene(z0), 0, 2.0 * Y)
    fd = (loss(z0 + h) - loss(z0 - h)) / (2.0 * h)
    assert gz[0] == pytest.approx(fd, rel=1e-4)
    # and d L / d sigma = L / sigma for L = a^2, a proportional to sqrt(sigma)
    assert gs[0] == pytest.approx(loss(z0) / 0.3, rel=1e-6)
