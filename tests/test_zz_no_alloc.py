"""rsim_doppler_accumulate_noalloc -- the spectrum pass for callers that cannot allocate
device memory where they run (allocation-free real-time loops, plug-ins inside a host
process whose allocator they do not own).  Its scratch is a device array built into the
library, so the caller passes only inputs and outputs.

Checked through the C ABI against rsim_doppler_accumulate (with a caller workspace).  The
sums are exact 64-bit fixed point, so the two entry points must give the same bits: on two
calls in a row (the second reuses the array the first one left dirty, which the pass must
clear itself), on the 65-update track of the benchmark's spectra, and on a request of exactly
the array's size.  This file is collected last so that a failure here stops a -x run only
after every other test has run; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu

LIMIT = 16 << 20   # bytes of the built-in scratch array


def _call(rsim, _lib, rd, pf, dev, u0, S, nf, nd, prec_id, cdt):
    B = ctypes.byref
    R, PF, SC = _lib.make_radar(rd), _lib.make_platform(pf), dev.c_struct()
    out = torch.zeros((S, rd.n_gates, nd), dtype=cdt, device="cuda")
    st = _lib.lib.rsim_doppler_accumulate_noalloc(B(R), B(PF), B(SC), u0, S, nf, nd, prec_id,
                                                  out.data_ptr(), None)
    assert st == 0, _lib.lib.rsim_last_error()
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_workspace_entry_point_twice():
    import paper_2408_11472_gb300 as rsim
    from paper_2408_11472_gb300 import _lib

    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    dev = rsim.Scatterers.from_arrays(sg.sea_surface(192, 21))
    for precision, prec_id, cdt in (("split", 1, torch.complex64), ("fp64", 0, torch.complex128)):
        u0, S = 28, 9
        ref = rsim.doppler_accumulate(rd, pf, dev, u0, S, fp.n_fast, fp.n_doppler, precision)
        assert np.abs(ref.cpu().numpy()).max() > 0
        for _ in range(2):
            out = _call(rsim, _lib, rd, pf, dev, u0, S, fp.n_fast, fp.n_doppler, prec_id, cdt)
            assert torch.equal(out, ref)


def test_noalloc_full_track_and_exact_limit():
    """65 updates of 128 gates x 64 bins (8.5 MB of scratch, the benchmark's spectra), then
    128 updates (exactly the 16 MiB the array holds): same bits as the workspace entry
    point."""
    import paper_2408_11472_gb300 as rsim
    from paper_2408_11472_gb300 import _lib

    c = sg.config(1)
    rd, pf, fp = c["radar"], c["platform"], c["fast"]
    dev = rsim.Scatterers.from_arrays(sg.sea_surface(128, 23))
    for S in (65, 128):
        need = _lib.lib.rsim_workspace_size(S, rd.n_gates, fp.n_doppler)
        assert need <= LIMIT and (S != 128 or need == LIMIT)
        ref = rsim.doppler_accumulate(rd, pf, dev, 0, S, fp.n_fast, fp.n_doppler, "split")
        out = _call(rsim, _lib, rd, pf, dev, 0, S, fp.n_fast, fp.n_doppler, 1, torch.complex64)
        assert torch.equal(out, ref)
        assert np.abs(out.cpu().numpy()).max() > 0


def test_noalloc_rejects_requests_beyond_its_scratch():
    import paper_2408_11472_gb300 as rsim
    from paper_2408_11472_gb300 import _lib

    rd = sg.RadarParams()
    pf = sg.nadir_track(4096)
    dev = rsim.Scatterers.from_arrays(sg.sea_surface(32, 2))
    B = ctypes.byref
    R, PF, SC = _lib.make_radar(rd), _lib.make_platform(pf), dev.c_struct()
    # 129 updates x 128 gates x 64 bins x 16 B = 16 MiB + 128 KiB
    out = torch.zeros((129, rd.n_gates, 64), dtype=torch.complex64, device="cuda")
    st = _lib.lib.rsim_doppler_accumulate_noalloc(B(R), B(PF), B(SC), 0, 129, 64, 64, 1,
                                                  out.data_ptr(), None)
    assert st == 5
    assert b"built-in" in _lib.lib.rsim_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(out) == 0
