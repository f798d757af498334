"""GPU parity of the fast mode (Algorithm 1 spectra + Section III.B post-processing)
against the FP64 oracle, through the C ABI, from small scenes to the full cfg1 scene."""
import numpy as np
import pytest
import torch

import scenegen as sg
from helpers import TOL, check_decisions, gpu_cells, np_, rel_l2

pytestmark = pytest.mark.gpu
PRECISIONS = ["fp64", "split"]


@pytest.fixture(scope="module")
def rsim():
    import paper_2408_11472_gb300 as m
    return m


@pytest.fixture(scope="module")
def small():
    c = sg.config(1)
    return c, sg.sea_surface(256, 1)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_spectra_parity_small(rsim, orc, small, precision):
    """256 x 256 surface on the cfg1 track; 9 updates from update 30 (several CTAs, ragged
    sample blocks, Doppler on both sides of zero).  Every update's index decisions against
    the oracle's; the spectra against the oracle summed over the GPU's decisions and, end to
    end, against the oracle with its own decisions, both at the path's tolerance."""
    c, sc = small
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    dev = rsim.Scatterers.from_arrays(sc)
    u0, S = 30, 9
    T = np_(rsim.doppler_accumulate(rd, pf, dev, u0, S, fp.n_fast, fp.n_doppler, precision))
    G, B = [], []
    for s in range(S):
        g, b, fg, fb = check_decisions(rsim, orc, rd, pf, dev, sc, (u0 + s) * fp.n_fast,
                                       fp.n_doppler, precision)
        assert fg < 1e-6 and fb < 1e-6
        G.append(g)
        B.append(b)
    Tref = orc.doppler_spectra_cells(rd, pf, sc, u0, fp.n_fast, fp.n_doppler, np.stack(G),
                                     np.stack(B))
    assert rel_l2(T, Tref) <= TOL[precision]
    Tor = orc.doppler_spectra(rd, pf, sc, u0, S, fp.n_fast, fp.n_doppler)
    assert rel_l2(T, Tor) <= TOL[precision]


def test_spectra_deterministic(rsim, small):
    c, sc = small
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    dev = rsim.Scatterers.from_arrays(sc)
    for precision in PRECISIONS:
        a = rsim.doppler_accumulate(rd, pf, dev, 3, 5, fp.n_fast, fp.n_doppler, precision)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            b = rsim.doppler_accumulate(rd, pf, dev, 3, 5, fp.n_fast, fp.n_doppler, precision)
        s.synchronize()
        assert torch.equal(a, b)


def test_single_bin_spectra_equal_regular_mode_bitwise(rsim, small):
    """With one Doppler bin the spectrum of update i is the regular-mode pulse p_i: the
    same contributions in the same cells give identical fixed-point sums."""
    c, sc = small
    rd, pf = c["radar"], c["platform"]
    dev = rsim.Scatterers.from_arrays(sc)
    for precision in PRECISIONS:
        T = rsim.doppler_accumulate(rd, pf, dev, 2, 3, 64, 1, precision)
        for s in range(3):
            Y = rsim.direct_sum(rd, pf, dev, (2 + s) * 64, 1, precision)
            assert torch.equal(T[s, :, 0], Y[0])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_simulate_fast_ragged_pulse_range(rsim, orc, small, precision):
    """A pulse range that starts and ends mid-segment: spectra and blended pulses, against
    the oracle with the GPU's checked decisions and end to end with its own."""
    c, sc = small
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    dev = rsim.Scatterers.from_arrays(sc)
    p0, P = 1000, 301
    T, Y = rsim.simulate_fast(rd, pf, dev, P, fp.n_fast, fp.n_doppler, fp.window, precision, p0)
    u0, S = rsim.spectra_range(p0, P, fp.n_fast)
    Tn = np_(T)
    G, B = [], []
    for s in range(S):
        g, b, _, _ = check_decisions(rsim, orc, rd, pf, dev, sc, (u0 + s) * fp.n_fast,
                                     fp.n_doppler, precision)
        G.append(g)
        B.append(b)
    Tref = orc.doppler_spectra_cells(rd, pf, sc, u0, fp.n_fast, fp.n_doppler, np.stack(G),
                                     np.stack(B))
    assert rel_l2(Tn, Tref) <= TOL[precision]
    Yref = orc.synth(Tref, u0, fp.n_fast, p0, P, fp.window)
    assert rel_l2(np_(Y), Yref) <= TOL[precision]
    Tor, Yor = orc.simulate_fast(rd, pf, sc, P, fp.n_fast, fp.n_doppler, fp.window, p0)
    assert rel_l2(Tn, Tor) <= TOL[precision]
    assert rel_l2(np_(Y), Yor) <= TOL[precision]


def test_fast_mode_equals_regular_at_update_pulses(rsim, small):
    c, sc = small
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    dev = rsim.Scatterers.from_arrays(sc)
    T, Y = rsim.simulate_fast(rd, pf, dev, 256, fp.n_fast, fp.n_doppler, fp.window, "fp64", 128)
    for x in (128, 192, 256, 320):
        Yr = rsim.direct_sum(rd, pf, dev, x, 1, "fp64")[0]
        # same contributions, summed per (gate, bin) then over bins vs per gate: equal up
        # to the 2^-32 fixed-point quantisation of the emitted partial sums
        assert rel_l2(np_(Y[x - 128]), np_(Yr)) < 1e-9


def test_large_cell_grids(rsim, orc):
    """4096 gates x 16 bins against the oracle; the largest grid (128 x 4096 bins) through
    its index decisions and its bin-summed spectrum (= the single-bin spectrum)."""
    rd = sg.RadarParams(n_gates=4096, gate_width_m=0.05)
    pf = sg.nadir_track(4096)
    sc = sg.sea_surface(64, 12)
    dev = rsim.Scatterers.from_arrays(sc)
    for precision in PRECISIONS:
        T = np_(rsim.doppler_accumulate(rd, pf, dev, 10, 1, 64, 16, precision))
        G, B = gpu_cells(rsim, rd, pf, dev, [640], 16, precision)
        Tref = orc.doppler_spectra_cells(rd, pf, sc, 10, 64, 16, G, B)
        assert np.abs(Tref).max() > 0
        assert rel_l2(T, Tref) <= TOL[precision]
    rd = sg.RadarParams()
    for precision in PRECISIONS:
        T = rsim.doppler_accumulate(rd, pf, dev, 10, 2, 64, 4096, precision)
        T1 = rsim.doppler_accumulate(rd, pf, dev, 10, 2, 64, 1, precision)
        assert rel_l2(np_(T.sum(-1)), np_(T1[..., 0])) < 1e-6
        check_decisions(rsim, orc, rd, pf, dev, sc, 640, 4096, precision)


def test_full_cfg1(rsim, orc):
    """cfg1 at full size in the benchmark's launch configuration: 4.19M scatterers,
    65 spectra of 128 x 64, 4096 pulses, split precision.  Every update: the index
    decisions against the oracle's, the spectrum against the oracle summed over those
    decisions, and end to end against the oracle with its own decisions, all at the split
    tolerance; the pulses against the oracle's post-processing of the GPU spectra and, end
    to end, of its own."""
    c = sg.config(1)
    rd, pf, fp, P = c["radar"], c["platform"], c["fast"], c["n_pulses"]
    sc = sg.sea_surface(c["L"], c["seed"])
    dev = rsim.Scatterers.from_arrays(sc)
    T, Y = rsim.simulate_fast(rd, pf, dev, P, fp.n_fast, fp.n_doppler, fp.window, "split")
    Tn, Yn = np_(T), np_(Y)
    S = Tn.shape[0]
    assert Tn.shape == (65, 128, 64) and Yn.shape == (4096, 128)
    exempt = 0.0
    for u in range(S):
        g, b, fg, fb = check_decisions(rsim, orc, rd, pf, dev, sc, u * fp.n_fast, fp.n_doppler,
                                       "split")
        exempt += fg + fb
        Tref = orc.doppler_spectra_cells(rd, pf, sc, u, fp.n_fast, fp.n_doppler, g[None],
                                         b[None])
        assert rel_l2(Tn[u:u + 1], Tref) <= TOL["split"], u
    assert exempt / S < 1e-6
    Tor = orc.doppler_spectra(rd, pf, sc, 0, S, fp.n_fast, fp.n_doppler)
    assert rel_l2(Tn, Tor) <= TOL["split"]
    Yref = orc.synth(Tn.astype(np.complex128), 0, fp.n_fast, 0, P, fp.window)
    assert rel_l2(Yn, Yref) <= 1e-5
    Yor = orc.synth(Tor, 0, fp.n_fast, 0, P, fp.window)
    assert rel_l2(Yn, Yor) <= TOL["split"]


def test_host_streamer_overlaps_copies_and_matches(rsim):
    """Scatterers streamed from pinned host memory in blocks (copies overlapped with the
    summation, exact sums in one workspace) give the spectra of one call on the whole set;
    the IQ read back on the streamer's side stream is each run's own result."""
    import scenegen as sg_
    c = sg_.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    scene = sg_.sea_surface(300, 8)                      # 90,000 scatterers: ragged last block
    host = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).pin_memory()
            for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs")}
    host.update(origin=scene["origin"], area=scene["area"])
    P = 640
    u0, S = rsim.spectra_range(0, P, fp.n_fast)
    hs = rsim.HostStreamer(scene["x"].size, rd.n_gates, fp.n_doppler, S, chunks=3)
    assert len(hs.ranges) == 3 and hs.ranges[0][0] == 0 and hs.ranges[-1][1] == scene["x"].size
    from paper_2408_11472_gb300.sharding import block_scatterers
    assert all(a % block_scatterers() == 0 for a, _ in hs.ranges)
    T, Y = hs.run(rd, pf, host, P, fp.n_fast, fp.n_doppler, fp.window)
    dev = rsim.Scatterers.from_arrays(scene)
    T1, Y1 = rsim.simulate_fast(rd, pf, dev, P, fp.n_fast, fp.n_doppler, fp.window)
    # blockwise exact sums in one workspace: bit-identical to one call on the whole set
    assert torch.equal(T, T1)
    assert torch.equal(Y, Y1)
    T2, _ = hs.run(rd, pf, host, P, fp.n_fast, fp.n_doppler, fp.window)   # the other buffer set
    assert torch.equal(T2, T)
    T3, _ = hs.run(rd, pf, host, P, fp.n_fast, fp.n_doppler, fp.window)   # the first set again
    assert torch.equal(T3, T)
    one = rsim.HostStreamer(scene["x"].size, rd.n_gates, fp.n_doppler, S)  # default: one block
    assert len(one.ranges) == 1
    T4, _ = one.run(rd, pf, host, P, fp.n_fast, fp.n_doppler, fp.window)
    assert torch.equal(T4, T)
    # IQ read back on the side stream into alternating pinned buffers, three runs in a row
    # writing the same device IQ: each host copy holds its own run's result
    yh = [torch.empty((P, rd.n_gates), dtype=torch.complex64).pin_memory() for _ in range(2)]
    Yd = torch.empty((P, rd.n_gates), dtype=torch.complex64, device="cuda")
    host2 = dict(host, t0=0.5)                           # a different state epoch: other IQ
    for r, h in enumerate((host, host2, host)):
        one.run(rd, pf, h, P, fp.n_fast, fp.n_doppler, fp.window, out=Yd, host_out=yh[r % 2])
        if r == 1:
            one.readback_done.synchronize()
            Y2 = yh[1].clone()
    one.wait_readback()
    torch.cuda.synchronize()
    assert torch.equal(yh[0], Y1.cpu())
    assert not torch.equal(Y2, Y1.cpu())
    dev2 = rsim.Scatterers(*[getattr(dev, k) for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs")],
                           origin=dev.origin, area=dev.area, t0=0.5)
    _, Y5 = rsim.simulate_fast(rd, pf, dev2, P, fp.n_fast, fp.n_doppler, fp.window)
    assert torch.equal(Y2, Y5.cpu())
    with pytest.raises(ValueError):
        one.run(rd, pf, host, P, fp.n_fast, fp.n_doppler, fp.window,
                host_out=torch.empty((P, rd.n_gates), dtype=torch.complex64))   # not pinned
