"""The summation evaluates two scatterers per paired FP32 instruction (fma/add/mul .f32x2);
the per-scatterer outputs and the exact re-evaluation of flagged scatterers use the scalar
evaluation.  Each lane of the paired form must round exactly as the scalar form, so on a
scene where many (gate, bin) cells hold a single scatterer, every such cell of the spectra
(and of the regular-mode IQ) is that scatterer's own C after the workspace's fixed-point
round trip, bit for bit."""
import numpy as np
import pytest

import scenegen as sg
from helpers import np_

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsim():
    import paper_2408_11472_gb300 as m
    return m


def fixed_round_trip(v):
    """float32 -> the workspace's 64-bit fixed point (value q 2^-32: integer part, then the
    fraction rounded to 2^-31) -> float32 (|q| split in 32-bit halves, lo 2^-32 + hi)."""
    v = np.asarray(v, dtype=np.float32)
    t = np.trunc(v)
    r = (v - t).astype(np.float32)                       # exact
    lo = np.rint((r * np.float32(2.0 ** 31)).astype(np.float32)).astype(np.int64)
    q = t.astype(np.int64) * (1 << 32) + lo * 2
    a = np.abs(q)
    lo_f = (a & 0xFFFFFFFF).astype(np.float64).astype(np.float32).astype(np.float64)
    # lo_f 2^-32 + hi is exact in float64 for |v| < 2^20; one rounding to float32, as the fma
    out = (lo_f * 2.0 ** -32 + (a >> 32).astype(np.float64)).astype(np.float32)
    return np.where(q < 0, -out, out)


def _scene(n, seed):
    """n scatterers within 30 m of the track's nadir point, heights over +-28 m (about 120
    of the 128 gates) and vertical speeds over +-25 m/s (about 17 Doppler bins), so that a
    good share of the occupied cells hold one scatterer."""
    rng = np.random.default_rng(seed)
    f = lambda a: np.asarray(a, dtype=np.float32)
    return {"x": f(rng.uniform(-30, 30, n)), "y": f(rng.uniform(-30, 30, n)),
            "z": f(rng.uniform(-28, 28, n)), "vx": f(rng.uniform(-1, 1, n)),
            "vy": f(rng.uniform(-1, 1, n)), "vz": f(rng.uniform(-25, 25, n)),
            "nrcs": f(rng.lognormal(-2.0, 0.5, n)), "origin": (0.0, 0.0, 0.0), "area": 1.0}


def _single_cells(g, b, n_gates, n_doppler):
    inwin = (g >= 0) & (g < n_gates)
    key = np.where(inwin, g.astype(np.int64) * n_doppler + b, -1)
    uniq, counts = np.unique(key[inwin], return_counts=True)
    idx = np.nonzero(inwin & np.isin(key, uniq[counts == 1]))[0]
    return idx, key[idx]


def _radars():
    return [sg.RadarParams(),
            sg.RadarParams(antenna=sg.antenna_table(31, n=129, half_width=0.004, width=0.002))]


@pytest.mark.parametrize("ant", [0, 1])
def test_fast_mode_cells_bit_identical_to_scalar(rsim, ant):
    rd = _radars()[ant]
    n_fast, n_doppler, P = 64, 64, 512
    pf = sg.nadir_track(P)
    dev = rsim.Scatterers.from_arrays(_scene(3001, 5))   # 3 blocks, the last one ragged
    u0, S = rsim.spectra_range(0, P, n_fast)
    T = np_(rsim.doppler_accumulate(rd, pf, dev, u0, S, n_fast, n_doppler, "split"))
    checked = 0
    for i in range(S):
        p = (u0 + i) * n_fast
        g, b, _, _ = rsim.scatterer_cells(rd, pf, dev, p, n_doppler, "split")
        c = np_(rsim.scatterer_echo(rd, pf, dev, p, "split"))
        idx, key = _single_cells(np_(g), np_(b), rd.n_gates, n_doppler)
        got = T[i].reshape(-1)[key]
        np.testing.assert_array_equal(got.real, fixed_round_trip(c.real[idx]))
        np.testing.assert_array_equal(got.imag, fixed_round_trip(c.imag[idx]))
        checked += idx.size
    assert checked > 1000


@pytest.mark.parametrize("ant", [0, 1])
def test_regular_mode_cells_bit_identical_to_scalar(rsim, ant):
    rd = _radars()[ant]
    P = 6
    pf = sg.nadir_track(P)
    dev = rsim.Scatterers.from_arrays(_scene(203, 6))     # about 1.7 per occupied gate
    Y = np_(rsim.direct_sum(rd, pf, dev, 0, P, "split"))
    checked = 0
    for p in range(P):
        g, _, _, _ = rsim.scatterer_cells(rd, pf, dev, p, 1, "split")
        c = np_(rsim.scatterer_echo(rd, pf, dev, p, "split"))
        idx, key = _single_cells(np_(g), np.zeros(dev.n, np.int64), rd.n_gates, 1)
        np.testing.assert_array_equal(Y[p][key].real, fixed_round_trip(c.real[idx]))
        np.testing.assert_array_equal(Y[p][key].imag, fixed_round_trip(c.imag[idx]))
        checked += idx.size
    assert checked > 50
