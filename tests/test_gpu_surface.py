"""Spectral surface update on the GPU (rsim_surface_prepare / rsim_surface_at, Algorithm 1's
update_simulation) against the FP64 numpy restatement, and the fast mode with the surface
regenerated at every update against the oracle fed with the oracle's own surfaces."""
import ctypes

import numpy as np
import pytest
import torch

import scenegen as sg
from helpers import check_decisions, np_, rel_l2
from oracle import surface as sf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsim():
    import paper_2408_11472_gb300 as m
    return m


# every pass plan of the mixed-radix transforms: 4 (radix 4), 8 (8), 16 (16), 32 (16, 2),
# 64 (16, 4), 128 (16, 8), 256 (16, 16), 512 (16, 16, 2), 1024 (16, 16, 4),
# 2048 (16, 16, 8), 4096 (16, 16, 16; two columns per block)
@pytest.mark.parametrize("L,spacing", [(64, 1.0), (256, 1.0), (128, 2.5), (4, 1.0), (8, 1.0),
                                       (16, 1.0), (32, 2.0), (512, 1.0), (1024, 1.0),
                                       (2048, 1.0), (4096, 1.0)])
def test_fields_match_oracle(rsim, L, spacing):
    spec = sg.sea_spectrum(L, 40 + L, spacing=spacing)
    surf = rsim.EvolvingSurface(spec)
    for t in (0.0, 0.35, 7.0, 3600.25):
        sc = surf.at(t)
        ref = sf.surface_at(spec, t)
        assert sc.t0 == t
        for key, arr in (("z", sc.z), ("vx", sc.vx), ("vy", sc.vy), ("vz", sc.vz)):
            r = ref[key]
            err = np.abs(np_(arr).astype(np.float64) - r).max()
            assert err <= 5e-6 * max(np.abs(r).max(), 1e-30), (key, t, err)


def test_t0_surface_is_the_seeded_surface(rsim):
    spec = sg.sea_spectrum(128, 3)
    sc = rsim.EvolvingSurface(spec).at(0.0)
    ref = sg.sea_surface(128, 3)
    assert torch.equal(sc.x, torch.as_tensor(ref["x"]).cuda())
    assert torch.equal(sc.nrcs, torch.as_tensor(ref["nrcs"]).cuda())
    for key in ("z", "vx", "vy", "vz"):
        r = ref[key].astype(np.float64)
        assert np.abs(np_(getattr(sc, key)) - r).max() <= 5e-6 * np.abs(r).max()


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_fast_mode_with_evolving_surface_matches_oracle(rsim, orc, precision):
    rd = sg.RadarParams()
    P, nf, nd = 384, 64, 64
    pf = sg.nadir_track(P)
    spec = sg.sea_spectrum(128, 21)
    surf = rsim.EvolvingSurface(spec)
    T, Y = rsim.simulate_fast_evolving(rd, pf, surf, P, nf, nd, "sqrt_raised_cosine", precision)
    u0, S = rsim.spectra_range(0, P, nf)
    for s in range(S):
        t = (u0 + s) * nf / rd.prf_hz
        sc_gpu = surf.at(t)
        sc_or = sf.scene_at(spec, t)
        # the surfaces differ by the FP32 transforms (~1e-7 m of height, 2e-7 gates; the
        # velocities' error moves the bin coordinate by ~1e-8): decisions are compared
        # outside a band of 1e-5 gates and 1e-6 bins around the oracle's cell edges
        G, B, _, _ = check_decisions(rsim, orc, rd, pf, sc_gpu, sc_or, (u0 + s) * nf, nd,
                                     precision, band=(1e-5, 1e-6))
        Tref = orc.doppler_spectra_cells(rd, pf, sc_or, u0 + s, nf, nd, G[None], B[None])
        # ~1e-7 m of height is ~1e-4 of phase
        assert rel_l2(np_(T)[s], Tref[0]) <= 1e-3
        assert rel_l2(np_(T)[s], orc.doppler_spectra(rd, pf, sc_or, u0 + s, 1, nf, nd)[0]) <= 1e-3
    # the surface moves: the spectra differ from those of the frozen t = 0 surface moved
    # along straight lines
    frozen = rsim.Scatterers.from_arrays(sg.sea_surface(128, 21))
    T_lin = rsim.doppler_accumulate(rd, pf, frozen, u0, S, nf, nd, precision)
    assert rel_l2(np_(T)[-1], np_(T_lin)[-1]) > 1e-2


@pytest.mark.parametrize("precision,block", [("split", 33), ("fp64", 33), ("split", 2),
                                             ("split", 3), ("fp64", 2)])
def test_evolving_loop_graph_replay_is_bit_identical(rsim, precision, block):
    """The update loop with buffers allocated once (EvolvingFastMode): eager run and CUDA
    graph replays give the spectra and pulses of simulate_fast_evolving bit for bit, on a
    ragged pulse range (7 spectra: one block, or several blocks synthesised on two streams
    into two alternating groups of field sets while the previous block is summed)."""
    rd = sg.RadarParams()
    P, p0, nf, nd = 333, 40, 64, 64
    pf = sg.nadir_track(P + p0)
    surf = rsim.EvolvingSurface(sg.sea_spectrum(128, 22))
    T, Y = rsim.simulate_fast_evolving(rd, pf, surf, P, nf, nd, "sqrt_raised_cosine", precision,
                                       p0)
    em = rsim.EvolvingFastMode(rd, pf, surf, P, nf, nd, "sqrt_raised_cosine", precision, p0,
                               block=block)
    Te, Ye = em.run()
    assert torch.equal(Te, T) and torch.equal(Ye, Y)
    em.capture()
    for _ in range(2):
        em.spectra.fill_(7.0)
        em.iq.fill_(7.0)
        Tg, Yg = em.replay()
        torch.cuda.synchronize()
        assert torch.equal(Tg, T) and torch.equal(Yg, Y)


def test_bad_spectra_are_rejected(rsim):
    import paper_2408_11472_gb300._lib as L
    spec = sg.sea_spectrum(16, 1)
    with pytest.raises(ValueError):
        rsim.EvolvingSurface(dict(spec, coef=spec["coef"][:, :8]))
    for bad in (dict(spec, coef=np.zeros((12, 12), complex)), dict(spec, spacing=0.0),
                dict(spec, scale=float("nan"))):
        with pytest.raises(rsim.RsimError):
            rsim.EvolvingSurface(bad)
    surf = rsim.EvolvingSurface(spec)
    with pytest.raises(rsim.RsimError):
        surf.at(float("inf"))
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(rsim.RsimError):            # workspace too small
        L.check(L.lib.rsim_surface_at(ctypes.byref(surf.spec), 0.0, surf.z.data_ptr(),
                                      surf.vx.data_ptr(), surf.vy.data_ptr(), surf.vz.data_ptr(),
                                      small.data_ptr(), 16, None))


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_states_summation_equals_single_state_pass(rsim, precision):
    """rsim_doppler_accumulate_states with every update given the same state (epoch 0) is the
    one-state summation of that scene: the FP64 path bit for bit, the split path to its
    rounding (its pulse-pair constant is formed per update in FP32).  8,100 scatterers: the
    last thread's float4 group is partial."""
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    sc = sg.sea_surface(90, 27)
    dev = rsim.Scatterers.from_arrays(sc)
    u0, S = 29, 7
    ref = rsim.doppler_accumulate(rd, pf, dev, u0, S, fp.n_fast, fp.n_doppler, precision)
    G = rd.n_gates
    ws = torch.empty(rsim.workspace_size(S, G, fp.n_doppler), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(ref)
    from paper_2408_11472_gb300 import _lib
    st = torch.cuda.current_stream().cuda_stream
    nbytes = ws.numel()
    _lib.check(_lib.lib.rsim_workspace_clear(S, G, fp.n_doppler, ws.data_ptr(), nbytes, st))
    states = [(dev.z, dev.vx, dev.vy, dev.vz, 0.0)] * S
    rsim.doppler_accumulate_states(rd, pf, dev, u0, states[:4], fp.n_fast, fp.n_doppler,
                                   precision, workspace=ws)
    slot = rsim.workspace_size(1, G, fp.n_doppler)
    rsim.doppler_accumulate_states(rd, pf, dev, u0 + 4, states[4:], fp.n_fast, fp.n_doppler,
                                   precision, workspace=ws[4 * slot:])
    prec = 0 if precision == "fp64" else 1
    _lib.check(_lib.lib.rsim_workspace_finalize(S, G, fp.n_doppler, prec, ws.data_ptr(), nbytes,
                                                out.data_ptr(), st))
    torch.cuda.synchronize()
    assert np.abs(np_(ref)).max() > 0
    if precision == "fp64":
        assert torch.equal(out, ref)
    else:
        assert rel_l2(np_(out), np_(ref)) <= 1e-5


def test_states_summation_rejects_bad_arguments(rsim):
    rd = sg.RadarParams()
    pf = sg.nadir_track(256)
    dev = rsim.Scatterers.from_arrays(sg.sea_surface(64, 3))
    ws = torch.empty(rsim.workspace_size(65, rd.n_gates, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        rsim.doppler_accumulate_states(rd, pf, dev, 0, [(dev.z, dev.vx, dev.vy, dev.vz, 0.0)] * 65,
                                       64, 64, workspace=ws)
    shifted = torch.empty(dev.n + 1, dtype=torch.float32, device="cuda")[1:]
    with pytest.raises(rsim.RsimError):
        rsim.doppler_accumulate_states(rd, pf, dev, 0, [(shifted, dev.vx, dev.vy, dev.vz, 0.0)],
                                       64, 64, workspace=ws)
    with pytest.raises(rsim.RsimError):
        rsim.doppler_accumulate_states(rd, pf, dev, 0, [(dev.z, dev.vx, dev.vy, dev.vz, 0.0)],
                                       64, 64, workspace=ws[:16])
