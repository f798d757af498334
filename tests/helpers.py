"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np

# Tolerances (relative L2 against the FP64 oracle summed over the same index decisions).
TOL = {"fp64": 1e-5, "split": 1e-3}
# Index decisions are compared bit-exactly except where the oracle's own pre-floor coordinate
# lies within this distance of an integer edge (the oracle's FP64 rounding noise is ~1e-10
# gates and ~1e-6 bins -- the bin coordinate comes from the difference of two ~7e7-cycle phases).
DELTA_GATE = 1e-7
DELTA_BIN = 2e-5


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


def index_agreement(g_gpu, b_gpu, gc_or, bc_or, g_or, b_or, n_doppler, check_bins=True):
    """Assert exact agreement outside the delta bands, +-1 inside; return exempt fractions."""
    near_g = np.abs(gc_or - np.round(gc_or)) < DELTA_GATE
    assert np.array_equal(g_gpu[~near_g], g_or[~near_g]), \
        "gate mismatch outside band: %d" % int((g_gpu[~near_g] != g_or[~near_g]).sum())
    assert np.all(np.abs(g_gpu[near_g].astype(np.int64) - g_or[near_g]) <= 1)
    fb = 0.0
    if check_bins:
        near_b = np.abs(bc_or - np.round(bc_or)) < DELTA_BIN
        assert np.array_equal(b_gpu[~near_b], b_or[~near_b]), \
            "bin mismatch outside band: %d" % int((b_gpu[~near_b] != b_or[~near_b]).sum())
        d = np.mod(b_gpu[near_b].astype(np.int64) - b_or[near_b], n_doppler)
        assert np.all((d == 0) | (d == 1) | (d == n_doppler - 1))
        fb = float(near_b.mean())
    return float(near_g.mean()), fb
