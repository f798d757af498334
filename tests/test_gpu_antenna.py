"""Tabulated antenna pattern (rsim_antenna, Section II.A: the pattern recorded on a u-v grid
and interpolated per facet) through the C ABI: per-scatterer echo, both summation modes,
batched sets and the adjoint, each against the FP64 oracle with the same table."""
import dataclasses

import numpy as np
import pytest
import torch

import scenegen as sg
from helpers import DELTA_BIN, DELTA_GATE, TOL, gpu_cells, np_, rel_l2

pytestmark = pytest.mark.gpu
PRECISIONS = ["fp64", "split"]


@pytest.fixture(scope="module")
def rsim():
    import paper_2408_11472_gb300 as m
    return m


def _radar():
    # a grid fine enough that the 256 m scene spans several cells around boresight, and
    # wide enough that no facet of these tests comes near the grid's border
    return sg.RadarParams(antenna=sg.antenna_table(31, n=129, half_width=0.004, width=0.002))


@pytest.fixture(scope="module")
def scene():
    return sg.sea_surface(256, 12)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_echo_with_table_matches_oracle(rsim, orc, scene, precision):
    rd = _radar()
    pf = sg.nadir_track(64)
    dev = rsim.Scatterers.from_arrays(scene)
    for p in (0, 37):
        C_o = orc.echo(rd, pf, scene, p / rd.prf_hz)["C"]
        C = np_(rsim.scatterer_echo(rd, pf, dev, p, precision)).astype(np.complex128)
        rel = np.abs(C - C_o) / np.abs(C_o).max()
        assert rel.max() < (1e-6 if precision == "fp64" else 1e-3)
        assert np.sqrt(np.mean(rel ** 2)) < (2e-7 if precision == "fp64" else 1e-4)
    # the table is in effect: the Gaussian pattern gives something else
    C_g = np_(rsim.scatterer_echo(dataclasses.replace(rd, antenna=None), pf, dev, 0, precision))
    assert np.abs(C_g - np_(rsim.scatterer_echo(rd, pf, dev, 0, precision))).max() > 1e-2 * np.abs(C_g).max()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_regular_mode_with_table(rsim, orc, scene, precision):
    rd = _radar()
    P = 24
    pf = sg.nadir_track(P)
    dev = rsim.Scatterers.from_arrays(scene)
    Y = np_(rsim.direct_sum(rd, pf, dev, 0, P, precision))
    G, _ = gpu_cells(rsim, rd, pf, dev, range(P), 1, precision)
    Yref = orc.direct_sum_cells(rd, pf, scene, 0, G)
    assert rel_l2(Y, Yref) <= TOL[precision]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_fast_mode_with_table(rsim, orc, scene, precision):
    rd = _radar()
    c = sg.config(1)
    fp = c["fast"]
    P = 512
    pf = sg.nadir_track(P)
    dev = rsim.Scatterers.from_arrays(scene)
    u0, S = rsim.spectra_range(0, P, fp.n_fast)
    T = np_(rsim.doppler_accumulate(rd, pf, dev, u0, S, fp.n_fast, fp.n_doppler, precision))
    G, B = gpu_cells(rsim, rd, pf, dev, [(u0 + s) * fp.n_fast for s in range(S)], fp.n_doppler,
                     precision)
    Tref = orc.doppler_spectra_cells(rd, pf, scene, u0, fp.n_fast, fp.n_doppler, G, B)
    assert rel_l2(T, Tref) <= TOL[precision]


def test_batched_sets_with_table_equal_single_calls(rsim):
    rd = _radar()
    pf = sg.nadir_track(512)
    scats = [rsim.Scatterers.from_arrays(sg.sea_surface(L, 40 + L)) for L in (40, 96, 64)]
    outs = rsim.doppler_accumulate_batched(rd, pf, scats, 2, 4, 64, 64)
    for s, T in zip(scats, outs):
        assert torch.equal(T, rsim.doppler_accumulate(rd, pf, s, 2, 4, 64, 64))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_adjoint_with_table_vs_oracle_gradient(rsim, orc, precision):
    rd = _radar()
    c = sg.config(4)
    fp = c["fast"]
    P = 256
    pf = sg.nadir_track(P)
    sc = sg.sea_surface(128, 8)
    dev = rsim.Scatterers.from_arrays(sc)
    u0, S = rsim.spectra_range(0, P, fp.n_fast)
    _, Y = rsim.simulate_fast(rd, pf, dev, P, fp.n_fast, fp.n_doppler, fp.window, precision)
    Yn = np_(Y).astype(np.complex128)
    target = sg.target_waveform(P, rd.n_gates, 4242, (np.abs(Yn) ** 2).mean(axis=0))
    GY = 4.0 * (np.abs(Yn) ** 2 - target) * Yn
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    GT = rsim.synth_pulses_backward(rd, torch.as_tensor(GY).to("cuda", cdt), S, u0, fp.n_fast,
                                    fp.n_doppler, 0, fp.window)
    gz, gs = rsim.doppler_accumulate_backward(rd, pf, dev, u0, fp.n_fast, GT)
    GTref = orc.synth_grad(GY, S, u0, fp.n_fast, fp.n_doppler, 0, fp.window)
    gz_o, gs_o = orc.fast_grad(rd, pf, sc, u0, fp.n_fast, GTref)
    ok = np.ones(sc["x"].size, bool)
    for s in range(S):
        g, b, gc, bc = orc.cells(rd, pf, sc, (u0 + s) * fp.n_fast, fp.n_doppler)
        ok &= (np.abs(gc - np.round(gc)) > 10 * DELTA_GATE) & (np.abs(bc - np.round(bc)) > 10 * DELTA_BIN)
    assert ok.mean() > 0.99
    tol = 1e-5 if precision == "fp64" else 2e-3
    assert rel_l2(np_(gz)[ok], gz_o[ok]) <= tol
    assert rel_l2(np_(gs)[ok], gs_o[ok]) <= tol


def test_bad_tables_are_rejected(rsim):
    import paper_2408_11472_gb300 as m
    pf = sg.nadir_track(8)
    dev = m.Scatterers.from_arrays(sg.sea_surface(16, 1))
    good = sg.antenna_table(1, n=9)
    for ant in (dataclasses.replace(good, du=0.0), dataclasses.replace(good, dv=-1.0),
                dataclasses.replace(good, gain=good.gain[:1, :]),
                dataclasses.replace(good, u0=float("nan"))):
        with pytest.raises(m.RsimError):
            m.direct_sum(sg.RadarParams(antenna=ant), pf, dev, 0, 1, "split")
