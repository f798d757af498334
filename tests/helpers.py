"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np

# Tolerances (relative L2 against the FP64 oracle).
TOL = {"fp64": 1e-5, "split": 1e-3}
# Index decisions (Algorithm 1's rasterisation indices: the floors of the gate and pulse-pair
# bin coordinates).  The oracle evaluates both coordinates without cancellation (pinned to
# 1e-11 gates and 1e-10 bins against 60-digit arithmetic); the GPU's FP64 path carries about
# 1.3e-10 gates (FP64 rounding of d_z near 8e5 m) and ~1e-14 bins.  Decisions are compared
# exactly except where the oracle's coordinate lies within these distances of a cell edge;
# inside that band the split path must take the decision of the GPU's own FP64 path.
DELTA_GATE = 2e-9
DELTA_BIN = 1e-9


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def np_(t):
    return t.detach().cpu().numpy()


def gpu_cells(rsim, radar, platform, scat, pulses, n_doppler, precision):
    G, B = [], []
    for p in pulses:
        g, b, _, _ = rsim.scatterer_cells(radar, platform, scat, int(p), n_doppler, precision)
        G.append(np_(g))
        B.append(np_(b))
    return np.stack(G), np.stack(B)


def _edge_dist(c):
    return np.abs(c - np.round(c))


def _mod_dist(a, b, n):
    d = np.mod(a - b, n)
    return np.minimum(d, n - d)


def check_decisions(rsim, orc, radar, platform, scat, scene, pulse, n_doppler, precision,
                    band=(DELTA_GATE, DELTA_BIN)):
    """Index decisions of `precision` at one pulse (gate at `pulse`, bin of the pair
    (pulse, pulse + 1)) against the oracle's own decisions on `scene`:

    * outside `band` of a cell edge (measured on the oracle's coordinate), gates of every
      scatterer that either side puts in the range window, and bins of every scatterer in
      the window, are equal to the oracle's;
    * inside the band the GPU's decision is the floor of its own FP64 coordinate (for
      RSIM_SPLIT: the decision of rsim_scatterer_cells(..., "fp64"));
    * with the default band, the GPU's FP64 coordinates lie within half the band of the
      oracle's, so that floor is a correct decision there.

    Returns the GPU's gates and bins (numpy) and the fractions inside the band."""
    g, b, _, _ = (np_(t) for t in rsim.scatterer_cells(radar, platform, scat, int(pulse),
                                                         n_doppler, precision))
    g64, b64, gc64, bc64 = (np_(t) for t in rsim.scatterer_cells(radar, platform, scat, int(pulse),
                                                                 n_doppler, "fp64"))
    g_o, b_o, gc_o, bc_o = orc.cells(radar, platform, scene, int(pulse), n_doppler)
    ng = radar.n_gates
    win_o = (g_o >= 0) & (g_o < ng)
    win = win_o | ((g >= 0) & (g < ng))
    near_g = _edge_dist(gc_o) < band[0]
    near_b = _edge_dist(bc_o) < band[1]
    bad = win & ~near_g & (g != g_o)
    assert not bad.any(), "gate mismatch outside the band: %d of %d" % (bad.sum(), win.sum())
    bad = win & near_g & (g != g64)
    assert not bad.any(), "gate inside the band differs from the FP64 decision: %d" % bad.sum()
    bad = win_o & ~near_b & (b != b_o)
    assert not bad.any(), "bin mismatch outside the band: %d of %d" % (bad.sum(), win_o.sum())
    bad = win_o & near_b & (b != b64)
    assert not bad.any(), "bin inside the band differs from the FP64 decision: %d" % bad.sum()
    if band == (DELTA_GATE, DELTA_BIN):
        assert np.abs(gc64[win_o] - gc_o[win_o]).max(initial=0.0) < 0.5 * DELTA_GATE
        if n_doppler > 1:   # one bin (regular mode): the bin coordinate carries no decision
            assert _mod_dist(bc64[win_o], bc_o[win_o], n_doppler).max(initial=0.0) \
                < 0.5 * DELTA_BIN
    return g, b, float(near_g[win].mean()) if win.any() else 0.0, \
        float(near_b[win_o].mean()) if win_o.any() else 0.0
