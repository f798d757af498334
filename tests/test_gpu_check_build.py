"""The -DRSIM_CHECK debug build (librsim_check.so) on the GPU: on in-range work its kernel
checks all pass and its results are bit-identical to librsim.so's; a contribution beyond the
fixed-point range (|value| >= 2^30, which librsim.so adds with wrap-around) is skipped by its
check and reported as RSIM_ERR_CHECK, and the next call is clean again."""
import contextlib

import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsim():
    import paper_2408_11472_gb300 as m
    return m


@pytest.fixture(scope="module")
def checklib():
    from paper_2408_11472_gb300 import _lib
    lib = _lib.load(_lib.CHECK_LIB_PATH)
    assert lib.rsim_check_build() == 1
    return lib


@contextlib.contextmanager
def _using(lib):
    """Route the Python binding's calls through `lib` (marshalling is unchanged)."""
    from paper_2408_11472_gb300 import _lib
    saved = _lib.lib
    _lib.lib = lib
    try:
        yield
    finally:
        _lib.lib = saved


def _scene(L=72, seed=5):
    d = sg.sea_surface(L, seed)   # 5184 scatterers: five full blocks and a ragged one
    return d


def test_in_range_work_passes_every_check(rsim, checklib):
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    scat = rsim.Scatterers.from_arrays(_scene())
    u0, S = 30, 5
    for prec in ("split", "fp64"):
        T = rsim.doppler_accumulate(rd, pf, scat, u0, S, fp.n_fast, fp.n_doppler, prec)
        Y = rsim.direct_sum(rd, pf, scat, u0 * fp.n_fast, 7, prec)
        oow = torch.zeros(S, dtype=torch.int64, device="cuda")
        with _using(checklib):
            Tc = rsim.doppler_accumulate(rd, pf, scat, u0, S, fp.n_fast, fp.n_doppler, prec,
                                         out_of_window=oow)
            Yc = rsim.direct_sum(rd, pf, scat, u0 * fp.n_fast, 7, prec)
            g = torch.randn(T.shape, dtype=T.dtype, device="cuda")
            gz_c, gs_c = rsim.doppler_accumulate_backward(rd, pf, scat, u0, fp.n_fast, g)
        assert torch.equal(T, Tc) and torch.equal(Y, Yc), prec
        gz, gs = rsim.doppler_accumulate_backward(rd, pf, scat, u0, fp.n_fast, g)
        assert torch.equal(gz, gz_c) and torch.equal(gs, gs_c), prec
        oow_n = torch.zeros(S, dtype=torch.int64, device="cuda")
        rsim.doppler_accumulate(rd, pf, scat, u0, S, fp.n_fast, fp.n_doppler, prec,
                                out_of_window=oow_n)
        assert torch.equal(oow, oow_n)


def test_fixed_point_overflow_is_reported(rsim, checklib):
    from paper_2408_11472_gb300 import _lib
    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    d = _scene(L=40, seed=6)
    d["nrcs"] = d["nrcs"].copy()
    d["nrcs"][123] = np.float32(1e30)     # sqrt(nrcs area) ~ 1e15: beyond 2^30
    scat = rsim.Scatterers.from_arrays(d)
    u0, S = 30, 3
    with _using(checklib):
        with pytest.raises(_lib.RsimError) as ei:
            rsim.doppler_accumulate(rd, pf, scat, u0, S, fp.n_fast, fp.n_doppler, "split")
        assert ei.value.status == 6
        assert "fixed-point range" in str(ei.value)
        # the record was cleared: in-range work right after is clean
        ok = rsim.Scatterers.from_arrays(_scene(L=40, seed=6))
        T = rsim.doppler_accumulate(rd, pf, ok, u0, S, fp.n_fast, fp.n_doppler, "split")
    assert torch.equal(T, rsim.doppler_accumulate(rd, pf, ok, u0, S, fp.n_fast, fp.n_doppler))
