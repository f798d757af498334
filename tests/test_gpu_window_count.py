"""The optional out-of-window counter of rsim_direct_sum and rsim_doppler_accumulate: per
sample, the scatterers whose gate lies outside the range window (Section II.A's box-car gate
model leaves them out).  Checked against the oracle's own gate decisions (exact away from the
window's two edges), against the GPU's per-scatterer decisions (exact), on a long track whose
sets enter the window part-way (culled, partial and full samples, ragged blocks and sample
groups); the counter changes nothing in the sums."""
import numpy as np
import pytest
import torch

import scenegen as sg
from helpers import DELTA_GATE, np_

pytestmark = pytest.mark.gpu
PRECISIONS = ["split", "fp64"]


@pytest.fixture(scope="module")
def rsim():
    import paper_2408_11472_gb300 as m
    return m


P_TRACK = 257_143


def _track_case(L=96, seed=950):
    """A set on the 100 km nadir track, epoch at mid-track: its scatterers enter the range
    window 250-285 updates (of 64 pulses) before nadir."""
    rd = sg.RadarParams()
    pf = sg.nadir_track(P_TRACK)
    d = sg.sea_surface(L, seed)
    d["t0"] = P_TRACK / (2 * rd.prf_hz)
    return rd, pf, d


def _oracle_counts(orc, rd, pf, scene, pulses):
    """Per pulse: (scatterers the oracle leaves out, scatterers whose gate coordinate lies
    within DELTA_GATE of either window edge, where a correct decision may go either way)."""
    out, near = [], []
    for p in pulses:
        g, _, gc, _ = orc.cells(rd, pf, scene, int(p), 1)
        out.append(int(((g < 0) | (g >= rd.n_gates)).sum()))
        near.append(int(((np.abs(gc) < DELTA_GATE) | (np.abs(gc - rd.n_gates) < DELTA_GATE)).sum()))
    return np.array(out), np.array(near)


def _gpu_cell_counts(rsim, rd, pf, scat, pulses, precision):
    c = []
    for p in pulses:
        g, _, _, _ = rsim.scatterer_cells(rd, pf, scat, int(p), 1, precision)
        g = np_(g)
        c.append(int(((g < 0) | (g >= rd.n_gates)).sum()))
    return np.array(c)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_fast_mode_counts_on_a_track_entering_the_window(rsim, orc, precision):
    rd, pf, d = _track_case()
    scat = rsim.Scatterers.from_arrays(d)
    mid = P_TRACK // 2 // 64
    u0, S, nf, nd = mid - 300, 40, 64, 64     # 40 updates: one full group of 32 and a ragged one
    oow = torch.zeros(S, dtype=torch.int64, device="cuda")
    T = rsim.doppler_accumulate(rd, pf, scat, u0, S, nf, nd, precision, out_of_window=oow)
    T0 = rsim.doppler_accumulate(rd, pf, scat, u0, S, nf, nd, precision)
    assert torch.equal(T, T0)
    got = np_(oow)
    pulses = [(u0 + s) * nf for s in range(S)]
    want, near = _oracle_counts(orc, rd, pf, d, pulses)
    n = scat.n
    assert got.max() == n and got.min() < n // 2     # culled, partial and mostly-inside updates
    assert (np.abs(got - want) <= near).all(), (got, want, near)
    assert np.array_equal(got, _gpu_cell_counts(rsim, rd, pf, scat, pulses, precision))
    # accumulated, not overwritten
    rsim.doppler_accumulate(rd, pf, scat, u0, S, nf, nd, precision, out_of_window=oow)
    assert np.array_equal(np_(oow), 2 * got)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_regular_mode_counts(rsim, orc, precision):
    rd, pf, d = _track_case(L=40, seed=951)
    scat = rsim.Scatterers.from_arrays(d)
    mid = P_TRACK // 2
    p0, n_p = mid - 285 * 64 + 3, 37           # pulses through the set's entry into the window
    oow = torch.zeros(n_p, dtype=torch.int64, device="cuda")
    Y = rsim.direct_sum(rd, pf, scat, p0, n_p, precision, out_of_window=oow)
    assert torch.equal(Y, rsim.direct_sum(rd, pf, scat, p0, n_p, precision))
    got = np_(oow)
    pulses = list(range(p0, p0 + n_p))
    want, near = _oracle_counts(orc, rd, pf, d, pulses)
    assert (np.abs(got - want) <= near).all(), (got, want, near)
    assert np.array_equal(got, _gpu_cell_counts(rsim, rd, pf, scat, pulses, precision))
    assert 0 < got.min() and got.max() < scat.n    # partly inside at every pulse


def test_counts_with_a_tabulated_pattern_and_a_ragged_block(rsim, orc):
    """The tabulated-pattern kernels count the same gates (the pattern weights C, it does not
    move the gate); 130^2 scatterers end in a partly filled block."""
    rd, pf, d = _track_case(L=130, seed=952)
    rd_t = sg.RadarParams(antenna=sg.antenna_table(31, n=129, half_width=0.02, width=0.01))
    scat = rsim.Scatterers.from_arrays(d)
    mid = P_TRACK // 2 // 64
    u0, S = mid + 280, 24                      # the set leaves the window
    a = torch.zeros(S, dtype=torch.int64, device="cuda")
    b = torch.zeros(S, dtype=torch.int64, device="cuda")
    rsim.doppler_accumulate(rd, pf, scat, u0, S, 64, 64, "split", out_of_window=a)
    rsim.doppler_accumulate(rd_t, pf, scat, u0, S, 64, 64, "split", out_of_window=b)
    assert torch.equal(a, b)
    got = np_(a)
    want, near = _oracle_counts(orc, rd, pf, d, [(u0 + s) * 64 for s in range(S)])
    assert (np.abs(got - want) <= near).all(), (got, want, near)
    assert got.min() < scat.n and got.max() > 0


def test_counter_with_empty_inputs(rsim):
    rd, pf, d = _track_case(L=8)
    scat = rsim.Scatterers.from_arrays(d)
    oow = torch.zeros(0, dtype=torch.int64, device="cuda")
    T = rsim.doppler_accumulate(rd, pf, scat, 10, 0, 64, 64, out_of_window=oow)
    assert T.shape == (0, rd.n_gates, 64)
    empty = rsim.Scatterers.from_arrays({k: np.zeros(0, np.float32)
                                         for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs")})
    oow = torch.zeros(3, dtype=torch.int64, device="cuda")
    rsim.doppler_accumulate(rd, pf, empty, 10, 3, 64, 64, out_of_window=oow)
    assert int(oow.sum()) == 0
    with pytest.raises(ValueError):
        rsim.doppler_accumulate(rd, pf, scat, 10, 3, 64, 64,
                                out_of_window=torch.zeros(2, dtype=torch.int64, device="cuda"))
