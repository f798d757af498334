"""Batched realizations (many independent surfaces of uneven size along one track, one
launch per group), culling of out-of-window samples, and CUDA-graph replay of the update loop."""
import numpy as np
import pytest
import torch

import scenegen as sg
from helpers import TOL, check_decisions, np_, rel_l2

pytestmark = pytest.mark.gpu
PRECISIONS = ["split", "fp64"]


@pytest.fixture(scope="module")
def rsim():
    import paper_2408_11472_gb300 as m
    return m


def _sets(rsim, sides, seed0=500, shift=0.0):
    out = []
    for i, L in enumerate(sides):
        if L == 0:
            out.append(rsim.Scatterers.from_arrays(
                {k: np.zeros(0, np.float32) for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs")}))
            continue
        d = sg.sea_surface(L, seed0 + i)
        d["origin"] = (shift * i, -0.5 * shift * i, 0.0)
        out.append(rsim.Scatterers.from_arrays(d))
    return out


@pytest.mark.parametrize("precision", PRECISIONS)
def test_batched_equals_individual_calls_bitwise(rsim, precision):
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    scats = _sets(rsim, [48, 100, 0, 64, 130, 20], shift=37.0)
    u0, S = 29, 6
    outs = rsim.doppler_accumulate_batched(rd, pf, scats, u0, S, fp.n_fast, fp.n_doppler, precision)
    for s, T in zip(scats, outs):
        if s.n == 0:
            assert torch.count_nonzero(T) == 0
            continue
        T1 = rsim.doppler_accumulate(rd, pf, s, u0, S, fp.n_fast, fp.n_doppler, precision)
        assert torch.equal(T, T1)


def test_every_launch_plan_gives_the_same_bits(rsim):
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    scats = _sets(rsim, [40, 0, 72, 33, 90, 16, 64, 25, 51, 12], seed0=700, shift=11.0)
    u0, S = 30, 9
    ref = rsim.doppler_accumulate_batched(rd, pf, scats, u0, S, fp.n_fast, fp.n_doppler)
    for sets, spg, pers in ((1, 0, 0), (3, 1, 0), (8, 4, 0), (96, 9, 0), (0, 2, 0), (5, 100, 0),
                            (0, 0, 4), (3, 1, 4), (96, 9, 1), (8, 2, 8)):
        t = rsim.Tuning(sets, spg, pers)
        outs = rsim.doppler_accumulate_batched(rd, pf, scats, u0, S, fp.n_fast, fp.n_doppler,
                                               tuning=t)
        for a, b in zip(outs, ref):
            assert torch.equal(a, b), (sets, spg, pers)
    # the FP64 path ignores the persistent form
    ref64 = rsim.doppler_accumulate_batched(rd, pf, scats, u0, S, fp.n_fast, fp.n_doppler, "fp64")
    outs = rsim.doppler_accumulate_batched(rd, pf, scats, u0, S, fp.n_fast, fp.n_doppler, "fp64",
                                           tuning=rsim.Tuning(0, 0, 4))
    for a, b in zip(outs, ref64):
        assert torch.equal(a, b)


def test_persistent_form_on_a_culled_long_track(rsim):
    """The persistent form on the 100 km track, where most (block, update) items are culled:
    the same bits as one call per set."""
    rd = sg.RadarParams()
    P = 257_143
    pf = sg.nadir_track(P)
    scats = []
    for i, L in enumerate((96, 40, 130)):
        d = sg.sea_surface(L, 950 + i)
        d["t0"] = P / (2 * rd.prf_hz)
        d["origin"] = (300.0 * i, 0.0, 0.0)
        scats.append(rsim.Scatterers.from_arrays(d))
    mid = P // 2 // 64
    u0, S = mid - 300, 64          # the sets enter the range window 250-285 updates before nadir
    outs = rsim.doppler_accumulate_batched(rd, pf, scats, u0, S, 64, 64,
                                           tuning=rsim.Tuning(0, 8, 4))
    nonzero = 0
    for s, T in zip(scats, outs):
        T1 = rsim.doppler_accumulate(rd, pf, s, u0, S, 64, 64)
        assert torch.equal(T, T1)
        nonzero += int(torch.count_nonzero(T1))
    assert nonzero > 0


def test_autotune_returns_a_valid_plan(rsim):
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    scats = _sets(rsim, [64, 100, 48, 80], seed0=710, shift=5.0)
    u0, S = 30, 8
    ref = rsim.doppler_accumulate_batched(rd, pf, scats, u0, S, fp.n_fast, fp.n_doppler)
    t, ms = rsim.autotune_batched(rd, pf, scats, u0, S, fp.n_fast, fp.n_doppler, reps=2)
    assert ms > 0.0
    assert 1 <= t.sets_per_launch <= 96 and t.samples_per_group >= 0
    assert 0 <= t.persistent <= 8 and list(t.reserved) == [0] * 5
    outs = rsim.doppler_accumulate_batched(rd, pf, scats, u0, S, fp.n_fast, fp.n_doppler, tuning=t)
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
    # the batched driver tunes on its first block and keeps the results unchanged
    bfm = rsim.BatchedFastMode(rd, pf, scats, u0 * fp.n_fast, 6 * fp.n_fast, fp.n_fast,
                               fp.n_doppler, update_block=4)
    y_default = [y.clone() for y in bfm.run()]
    bfm.autotune(reps=1)
    for a, b in zip(bfm.run(), y_default):
        assert torch.equal(a, b)


def test_bad_tuning_is_rejected(rsim):
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    scats = _sets(rsim, [16], seed0=720)
    for t in (rsim.Tuning(97, 0), rsim.Tuning(-1, 0), rsim.Tuning(4, -2), rsim.Tuning(4, 0, 9),
              rsim.Tuning(4, 0, -1)):
        with pytest.raises(rsim.RsimError):
            rsim.doppler_accumulate_batched(rd, pf, scats, 0, 1, fp.n_fast, fp.n_doppler, tuning=t)
    t = rsim.Tuning(4, 0)
    t.reserved[2] = 1
    with pytest.raises(rsim.RsimError):
        rsim.doppler_accumulate_batched(rd, pf, scats, 0, 1, fp.n_fast, fp.n_doppler, tuning=t)


def test_more_sets_than_one_launch_holds(rsim):
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    scats = _sets(rsim, [8 + (i % 7) for i in range(150)], seed0=900)
    outs = rsim.doppler_accumulate_batched(rd, pf, scats, 31, 2, fp.n_fast, fp.n_doppler)
    for i in (0, 95, 96, 149):
        T1 = rsim.doppler_accumulate(rd, pf, scats[i], 31, 2, fp.n_fast, fp.n_doppler)
        assert torch.equal(outs[i], T1)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_culling_on_a_long_track(rsim, orc, precision):
    """100 km track (257,143 pulses), scene at the midpoint: spectra of updates outside the
    range window are empty, those crossing into it match the oracle (which sums every
    scatterer without any culling)."""
    rd = sg.RadarParams()
    P = 257_143
    pf = sg.nadir_track(P)
    sc = sg.sea_surface(96, 17)
    sc["t0"] = P / (2 * rd.prf_hz)     # surface state given at the nadir crossing
    dev = rsim.Scatterers.from_arrays(sc)
    nf, nd = 64, 64
    # the scene enters the range window about 350 updates (1.2 s, 8.7 km) before nadir:
    # empty before, partly inside (0.04 % .. 50 % of the scatterers) across these updates
    mid = P // 2 // nf
    probe = [mid - 1500, mid - 360, mid - 349, mid - 347, mid - 330, mid - 278, mid, mid + 300,
             mid + 1500]
    for u in probe:
        T = np_(rsim.doppler_accumulate(rd, pf, dev, u, 1, nf, nd, precision))
        g, b, _, _ = check_decisions(rsim, orc, rd, pf, dev, sc, u * nf, nd, precision)
        Tref = orc.doppler_spectra_cells(rd, pf, sc, u, nf, nd, g[None], b[None])
        Tor = orc.doppler_spectra(rd, pf, sc, u, 1, nf, nd)
        if np.abs(Tref).max() == 0:
            assert np.abs(T).max() == 0 and np.abs(Tor).max() == 0
        else:
            assert rel_l2(T, Tref) <= TOL[precision]
            assert rel_l2(T, Tor) <= TOL[precision]
    T_far = np_(rsim.doppler_accumulate(rd, pf, dev, mid - 1500, 3, nf, nd, precision))
    assert np.abs(T_far).max() == 0
    T_in = np_(rsim.doppler_accumulate(rd, pf, dev, mid, 1, nf, nd, precision))
    assert np.abs(T_in).max() > 0


def test_batched_fast_mode_graph_replay(rsim):
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    scats = _sets(rsim, [40, 72, 56], seed0=700, shift=11.0)
    run = rsim.BatchedFastMode(rd, pf, scats, 1000, 300, fp.n_fast, fp.n_doppler, fp.window,
                               update_block=3)
    eager = [y.clone() for y in run.run()]
    run.capture()
    for y in run.iq:
        y.zero_()
    replayed = run.replay()
    torch.cuda.synchronize()
    for a, b, s in zip(eager, replayed, scats):
        assert torch.equal(a, b)
        _, Y1 = rsim.simulate_fast(rd, pf, s, 300, fp.n_fast, fp.n_doppler, fp.window, "split", 1000)
        assert torch.equal(a, Y1)
