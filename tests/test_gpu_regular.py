"""GPU parity of the regular mode (rsim_direct_sum) and of the index decisions against
the FP64 oracle, through the C ABI."""
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
def cfg0():
    c = sg.config(0)
    return c, sg.sea_surface(c["L"], c["seed"])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_cells_match_oracle_cfg0(rsim, orc, cfg0, precision):
    c, sc = cfg0
    dev = rsim.Scatterers.from_arrays(sc)
    rd, pf = c["radar"], c["platform"]
    for p in (0, 31, 63):
        _, _, fg, fb = check_decisions(rsim, orc, rd, pf, dev, sc, p, 64, precision)
        assert fg < 1e-6 and fb < 1e-6
        # coordinates themselves: FP64 path to rounding, split path to FP32 level
        g_o, b_o, gc_o, bc_o = orc.cells(rd, pf, sc, p, 64)
        g, b, gc, bc = rsim.scatterer_cells(rd, pf, dev, p, 64, precision)
        tol_g = 1e-9 if precision == "fp64" else 5e-6
        assert np.abs(np_(gc) - gc_o).max() < tol_g


@pytest.mark.parametrize("precision", PRECISIONS)
def test_scatterer_echo_matches_oracle(rsim, orc, cfg0, precision):
    """Per-scatterer complex amplitude: FP64 path to rounding; split path within its FP32
    phase error (a few 1e-6 cycles of two-way phase) and amplitude rounding."""
    c, sc = cfg0
    dev = rsim.Scatterers.from_arrays(sc)
    rd, pf = c["radar"], c["platform"]
    for p in (0, 40):
        C_o = orc.echo(rd, pf, sc, p / rd.prf_hz)["C"]
        C = np_(rsim.scatterer_echo(rd, pf, dev, p, precision)).astype(np.complex128)
        assert C.dtype == np.complex128 and C.shape == C_o.shape
        rel = np.abs(C - C_o) / np.abs(C_o)
        assert rel.max() < (1e-6 if precision == "fp64" else 1e-3)
        assert np.sqrt(np.mean(rel ** 2)) < (2e-7 if precision == "fp64" else 1e-4)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_direct_sum_parity_cfg0(rsim, orc, cfg0, precision):
    """cfg0 at full size: 65,536 scatterers x 64 pulses."""
    c, sc = cfg0
    rd, pf, P = c["radar"], c["platform"], c["n_pulses"]
    dev = rsim.Scatterers.from_arrays(sc)
    Y = np_(rsim.direct_sum(rd, pf, dev, 0, P, precision))
    gates = np.stack([check_decisions(rsim, orc, rd, pf, dev, sc, p, 1, precision)[0]
                      for p in range(P)])
    Yref = orc.direct_sum_cells(rd, pf, sc, 0, gates)
    err = rel_l2(Y, Yref)
    assert err <= TOL[precision], err
    if precision == "fp64":
        # element-wise: the oracle's phase of a ~7e7-cycle two-way range carries ~1e-8-cycle
        # FP64 rounding (~1e-7 relative per contribution), the GPU's sums 2^-32 fixed point
        np.testing.assert_allclose(Y, Yref, rtol=0, atol=1e-6 * np.abs(Yref).max())
    # end to end against the oracle's own decisions
    Yor = orc.direct_sum(rd, pf, sc, 0, P)
    assert rel_l2(Y, Yor) <= TOL[precision]


def test_direct_sum_accumulates_and_is_deterministic(rsim, cfg0):
    c, sc = cfg0
    rd, pf = c["radar"], c["platform"]
    dev = rsim.Scatterers.from_arrays(sc)
    for precision in PRECISIONS:
        a = rsim.direct_sum(rd, pf, dev, 5, 9, precision)
        b = rsim.direct_sum(rd, pf, dev, 5, 9, precision)
        assert torch.equal(a, b)
        rsim.direct_sum(rd, pf, dev, 5, 9, precision, out=b)
        assert torch.equal(b, 2 * a)


@pytest.mark.parametrize("n", [1, 1023, 1025, 4097])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_direct_sum_ragged_sizes(rsim, orc, precision, n):
    rd = sg.RadarParams()
    pf = sg.nadir_track(64)
    full = sg.sea_surface(72, 3)
    sc = {k: (v[:n] if isinstance(v, np.ndarray) else v) for k, v in full.items()}
    dev = rsim.Scatterers.from_arrays(sc)
    Y = np_(rsim.direct_sum(rd, pf, dev, 2, 7, precision))
    gates, _ = gpu_cells(rsim, rd, pf, dev, range(2, 9), 1, precision)
    Yref = orc.direct_sum_cells(rd, pf, sc, 2, gates)
    assert rel_l2(Y, Yref) <= TOL[precision]
    assert rel_l2(Y, orc.direct_sum(rd, pf, sc, 2, 7)) <= TOL[precision]


def test_misaligned_arrays_give_identical_results(rsim):
    """Arrays that are not 16-byte aligned take the scalar-load path: same bits."""
    rd = sg.RadarParams()
    pf = sg.nadir_track(64)
    sc = sg.sea_surface(48, 4)
    dev = rsim.Scatterers.from_arrays(sc)
    shifted = {}
    for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs"):
        t = torch.empty(dev.n + 1, dtype=torch.float32, device="cuda")
        t[1:] = getattr(dev, k)
        shifted[k] = t[1:]
    dev2 = rsim.Scatterers(**shifted)
    assert dev2.x.data_ptr() % 16 != 0
    for precision in PRECISIONS:
        a = rsim.direct_sum(rd, pf, dev, 0, 4, precision)
        b = rsim.direct_sum(rd, pf, dev2, 0, 4, precision)
        assert torch.equal(a, b)


def test_empty_scene_and_zero_pulses(rsim):
    rd = sg.RadarParams()
    pf = sg.nadir_track(64)
    e = {k: np.zeros(0, np.float32) for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs")}
    dev = rsim.Scatterers.from_arrays(e)
    out = torch.full((3, rd.n_gates), 1 + 2j, dtype=torch.complex64, device="cuda")
    rsim.direct_sum(rd, pf, dev, 0, 3, "split", out=out)
    assert torch.all(out == 1 + 2j)
    sc = rsim.Scatterers.from_arrays(sg.sea_surface(16, 1))
    z = rsim.direct_sum(rd, pf, sc, 0, 0, "split")
    assert z.shape == (0, rd.n_gates)


@pytest.mark.parametrize("n_gates", [1, 7, 4096])
def test_gate_counts(rsim, orc, n_gates):
    rd = sg.RadarParams(n_gates=n_gates, gate_width_m=0.47 if n_gates < 4096 else 0.05)
    pf = sg.nadir_track(64)
    sc = sg.sea_surface(64, 8)
    dev = rsim.Scatterers.from_arrays(sc)
    for precision in PRECISIONS:
        Y = np_(rsim.direct_sum(rd, pf, dev, 10, 3, precision))
        gates, _ = gpu_cells(rsim, rd, pf, dev, range(10, 13), 1, precision)
        Yref = orc.direct_sum_cells(rd, pf, sc, 10, gates)
        if np.abs(Yref).max() == 0:
            assert np.abs(Y).max() == 0
        else:
            assert rel_l2(Y, Yref) <= TOL[precision]
            assert rel_l2(Y, orc.direct_sum(rd, pf, sc, 10, 3)) <= TOL[precision]


def test_long_track_and_moving_window(rsim, orc):
    """Pulse indices ~ 2.5e5 (t ~ 14 s, a 100 km track) and a drifting range window."""
    rd = sg.RadarParams()
    P = 257_143
    pf0 = sg.nadir_track(P)
    pf = sg.PlatformParams(p0=pf0.p0, v=pf0.v, r_ref0=pf0.r_ref0 - 0.3, r_ref_rate=0.05)
    sc = sg.sea_surface(96, 6)
    sc["t0"] = P / (2 * rd.prf_hz) - 0.25   # surface state given a quarter second before
    dev = rsim.Scatterers.from_arrays(sc)
    p0 = P // 2 - 3
    for precision in PRECISIONS:
        Y = np_(rsim.direct_sum(rd, pf, dev, p0, 6, precision))
        gates, _ = gpu_cells(rsim, rd, pf, dev, range(p0, p0 + 6), 1, precision)
        Yref = orc.direct_sum_cells(rd, pf, sc, p0, gates)
        assert np.abs(Yref).max() > 0
        assert rel_l2(Y, Yref) <= TOL[precision]
        assert rel_l2(Y, orc.direct_sum(rd, pf, sc, p0, 6)) <= TOL[precision]
