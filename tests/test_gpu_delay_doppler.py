"""Delay-Doppler focusing (rsim_delay_doppler, Section IV.C) through the C ABI against the
FP64 numpy restatement, on random and on simulated IQ."""
import dataclasses

import numpy as np
import pytest
import torch

import scenegen as sg
from helpers import np_, rel_l2
from oracle import delay_doppler as dd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsim():
    import paper_2408_11472_gb300 as m
    return m


# a cluster of up to eight CTAs per burst splits its gates and beams; small bursts or gate
# counts take smaller clusters (down to one gate or one beam per CTA: (2, 2), (8, 2), (4, 4))
@pytest.mark.parametrize("burst,n_gates,n_pulses,pulse0", [(64, 128, 1000, 0), (16, 32, 256, 333),
                                                           (128, 64, 384, 7), (2, 2, 9, 0),
                                                           (4, 4, 41, 1), (8, 2, 24, 3),
                                                           (1024, 8, 2048, 0)])
def test_random_iq_matches_oracle(rsim, burst, n_gates, n_pulses, pulse0):
    rd = sg.RadarParams(n_gates=n_gates)
    pf = dataclasses.replace(sg.nadir_track(n_pulses), v=(7000.0, 450.0, 2.5), r_ref_rate=1.7)
    iq = sg.random_iq(n_pulses, n_gates, seed=burst + n_gates)
    ml, beams = rsim.delay_doppler(rd, pf, torch.as_tensor(iq).to("cuda", torch.complex64),
                                   pulse0, burst, focused=True)
    Y, W = dd.focus(rd, pf, iq.astype(np.complex64), pulse0, burst)
    assert beams.shape == Y.shape and ml.shape == W.shape
    assert rel_l2(np_(beams), Y) <= 5e-6
    assert rel_l2(np_(ml), W) <= 1e-5


def test_simulated_iq_focuses_like_the_oracle(rsim):
    c = sg.config(1)
    rd, fp = c["radar"], c["fast"]
    P = 1024
    pf = sg.nadir_track(P)
    dev = rsim.Scatterers.from_arrays(sg.sea_surface(256, 3))
    _, Y = rsim.simulate_fast(rd, pf, dev, P, fp.n_fast, fp.n_doppler, fp.window, "split")
    ml, beams = rsim.delay_doppler(rd, pf, Y, 0, 64, focused=True)
    Yo, Wo = dd.focus(rd, pf, np_(Y), 0, 64)
    assert rel_l2(np_(beams), Yo) <= 5e-6
    assert rel_l2(np_(ml), Wo) <= 1e-5
    # energy: each burst's multi-look sums to the burst's IQ energy
    e = (np.abs(np_(Y)[:16 * 64].reshape(16, 64, -1)) ** 2).sum(axis=(1, 2))
    np.testing.assert_allclose(np_(ml).sum(axis=1), e, rtol=1e-5)
    # without beams the multi-look is the same
    ml2, none = rsim.delay_doppler(rd, pf, Y, 0, 64)
    assert none is None and torch.equal(ml2, ml)


def test_shapes_and_rejections(rsim):
    rd = sg.RadarParams(n_gates=128)
    pf = sg.nadir_track(64)
    iq = torch.zeros((63, 128), dtype=torch.complex64, device="cuda")
    ml, _ = rsim.delay_doppler(rd, pf, iq, 0, 64)
    assert ml.shape == (0, 128)
    with pytest.raises(rsim.RsimError):
        rsim.delay_doppler(sg.RadarParams(n_gates=96), pf,
                           torch.zeros((64, 96), dtype=torch.complex64, device="cuda"), 0, 64)
    with pytest.raises(rsim.RsimError):
        rsim.delay_doppler(rd, pf, torch.zeros((256, 128), dtype=torch.complex64, device="cuda"), 0, 128)
    with pytest.raises(rsim.RsimError):
        rsim.delay_doppler(rd, pf, torch.zeros((64, 128), dtype=torch.complex64, device="cuda"), 0, 48)
    with pytest.raises(rsim.RsimError):      # bursts longer than 1024 pulses
        rsim.delay_doppler(sg.RadarParams(n_gates=2), pf,
                           torch.zeros((2048, 2), dtype=torch.complex64, device="cuda"), 0, 2048)
