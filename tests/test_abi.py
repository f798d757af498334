"""CPU-side checks of the C ABI: every function include/rsim.h declares is exported by the
built library, and argument validation rejects bad calls before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsim.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    names = re.findall(r"\b(rsim_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_2408_11472_gb300 import _lib
    return _lib


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rsim_direct_sum", "rsim_doppler_accumulate", "rsim_synth_pulses",
                 "rsim_direct_sum_backward", "rsim_doppler_accumulate_backward",
                 "rsim_synth_pulses_backward", "rsim_workspace_size", "rsim_last_error",
                 "rsim_version", "rsim_scatterer_cells"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L.lib, name), name
        assert name in L.PROTOTYPES, "binding lacks a prototype for %s" % name


def test_check_build_flag(L):
    """librsim_check.so is the same library compiled with -DRSIM_CHECK: it says so, exports
    the whole boundary and validates arguments on the host exactly as librsim.so does."""
    assert L.lib.rsim_check_build() == 0
    chk = L.load(L.CHECK_LIB_PATH)
    assert chk.rsim_check_build() == 1
    assert chk.rsim_version() == L.lib.rsim_version()
    for name in declared_functions():
        assert hasattr(chk, name), name
    B = ctypes.byref
    rd, pf, sc = _structs(L)
    assert chk.rsim_direct_sum(None, B(pf), B(sc), 0, 4, 1, 0x1000, 0x1000, 1 << 20, None,
                               None) == 1
    assert b"radar" in chk.rsim_last_error()
    assert chk.rsim_workspace_size(65, 128, 64) == L.lib.rsim_workspace_size(65, 128, 64)


def test_version_and_workspace_size(L):
    assert L.lib.rsim_version() == 2
    assert L.lib.rsim_workspace_size(65, 128, 64) == 65 * 128 * 64 * 16
    assert L.lib.rsim_workspace_size(4096, 128, 1) == 4096 * 128 * 16
    assert L.lib.rsim_workspace_size(4, 128, 3) == 0      # not a power of two
    assert L.lib.rsim_workspace_size(-1, 128, 1) == 0
    assert L.lib.rsim_workspace_size(4, 0, 1) == 0


def _structs(L, n=16, **radar_kw):
    import paper_2408_11472_gb300 as rsim
    rd = L.make_radar(rsim.Radar(**radar_kw))
    pf = L.make_platform(rsim.Platform())
    fake = 0x100000  # never dereferenced: every call below fails validation first
    sc = L.Scatterers(n, *([fake] * 7), (ctypes.c_double * 3)(0, 0, 0), 1.0)
    return rd, pf, sc


def test_invalid_arguments_are_rejected(L):
    B = ctypes.byref
    rd, pf, sc = _structs(L)
    lib = L.lib
    # missing structs
    assert lib.rsim_direct_sum(None, B(pf), B(sc), 0, 4, 1, 0x1000, 0x1000, 1 << 20, None, None) == 1
    assert b"radar" in lib.rsim_last_error()
    # bad radar
    bad, _, _ = _structs(L, n_gates=0)
    assert lib.rsim_direct_sum(B(bad), B(pf), B(sc), 0, 4, 1, 0x1000, 0x1000, 1 << 20, None, None) == 1
    # bad precision
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc), 0, 4, 7, 0x1000, 0x1000, 1 << 20, None, None) == 1
    # negative pulse / count
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc), -1, 4, 1, 0x1000, 0x1000, 1 << 20, None, None) == 1
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc), 0, -4, 1, 0x1000, 0x1000, 1 << 20, None, None) == 1
    # fast mode: n_fast = 0 is regular mode, n_doppler must be a power of two
    assert lib.rsim_doppler_accumulate(B(rd), B(pf), B(sc), 0, 2, 0, 64, 1, 0x1000, 0x1000,
                                       1 << 24, None, None) == 1
    assert lib.rsim_doppler_accumulate(B(rd), B(pf), B(sc), 0, 2, 64, 48, 1, 0x1000, 0x1000,
                                       1 << 24, None, None) == 1
    # null scatterer arrays with n > 0
    sc_null = L.Scatterers(16, *([None] * 7), (ctypes.c_double * 3)(0, 0, 0), 1.0)
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc_null), 0, 4, 1, 0x1000, 0x1000, 1 << 20, None, None) == 1


def test_workspace_errors(L):
    B = ctypes.byref
    rd, pf, sc = _structs(L)
    lib = L.lib
    need = lib.rsim_workspace_size(4, 128, 1)
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc), 0, 4, 1, 0x1000, None, need, None, None) == 5
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc), 0, 4, 1, 0x1000, 0x1000, need - 1, None, None) == 5
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc), 0, 4, 1, 0x1000, 0x1008, need, None, None) == 5
    assert b"workspace" in lib.rsim_last_error()


def test_out_of_window_counter_must_be_aligned(L):
    """The optional out-of-window counter of the two summation calls is checked on the host
    (8-byte alignment) before any CUDA call."""
    B = ctypes.byref
    rd, pf, sc = _structs(L)
    lib = L.lib
    need = lib.rsim_workspace_size(4, 128, 1)
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc), 0, 4, 1, 0x1000, 0x1000, need, 0x2004,
                               None) == 1
    assert b"out_of_window" in lib.rsim_last_error()
    need = lib.rsim_workspace_size(2, 128, 64)
    assert lib.rsim_doppler_accumulate(B(rd), B(pf), B(sc), 0, 2, 64, 64, 1, 0x1000, 0x1000,
                                       need, 0x2002, None) == 1
    assert b"out_of_window" in lib.rsim_last_error()


def test_noalloc_size_limit_is_checked_on_the_host(L):
    """The allocation-free pass rejects a request just over its 16 MiB built-in scratch
    (129 updates x 128 gates x 64 bins x 16 B) before any CUDA call, so this runs without a
    GPU; exactly 16 MiB (128 updates) is accepted (checked on a GPU in test_zz_no_alloc)."""
    B = ctypes.byref
    rd, pf, sc = _structs(L)
    lib = L.lib
    assert lib.rsim_workspace_size(128, 128, 64) == 16 << 20
    assert lib.rsim_doppler_accumulate_noalloc(B(rd), B(pf), B(sc), 0, 129, 64, 64, 1, 0x1000,
                                               None) == 5
    assert b"built-in" in lib.rsim_last_error()
    assert lib.rsim_doppler_accumulate_noalloc(None, B(pf), B(sc), 0, 4, 64, 64, 1, 0x1000,
                                               None) == 1


def test_states_summation_validates_on_the_host(L):
    """rsim_doppler_accumulate_states checks its states before any CUDA call: at most 64 per
    call, a states array when there are updates, 16-byte aligned fields."""
    B = ctypes.byref
    rd, pf, sc = _structs(L)
    lib = L.lib
    st = (L.SurfaceState * 1)(L.SurfaceState(0x1000, 0x1000, 0x1000, 0x1000, 0.0))
    assert lib.rsim_doppler_accumulate_states(B(rd), B(pf), B(sc), 0, 65, st, 64, 64, 1,
                                              0x1000, 1 << 30, None) == 1
    assert lib.rsim_doppler_accumulate_states(B(rd), B(pf), B(sc), 0, 1, None, 64, 64, 1,
                                              0x1000, 1 << 30, None) == 1
    bad = (L.SurfaceState * 1)(L.SurfaceState(0x1004, 0x1000, 0x1000, 0x1000, 0.0))
    assert lib.rsim_doppler_accumulate_states(B(rd), B(pf), B(sc), 0, 1, bad, 64, 64, 1,
                                              0x1000, 1 << 30, None) == 1
    assert b"16-byte" in lib.rsim_last_error()
    assert lib.rsim_doppler_accumulate_states(B(rd), B(pf), B(sc), 0, 1, st, 64, 64, 1,
                                              0x1000, 16, None) == 5


def test_empty_work_is_a_noop(L):
    B = ctypes.byref
    rd, pf, sc = _structs(L, n=0)
    lib = L.lib
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc), 0, 4, 1, None, None, 0, None, None) == 0
    rd, pf, sc = _structs(L)
    assert lib.rsim_direct_sum(B(rd), B(pf), B(sc), 0, 0, 1, None, None, 0, None, None) == 0
    assert lib.rsim_synth_pulses(B(rd), None, 0, 0, 64, 64, 0, 0, 1, 1, None, None) == 0


def test_synth_checks_spectrum_coverage(L):
    B = ctypes.byref
    rd, _, _ = _structs(L)
    lib = L.lib
    # pulses 0..127 with n_fast 64 need spectra of updates 0, 1, 2
    assert lib.rsim_synth_pulses(B(rd), 0x1000, 2, 0, 64, 64, 0, 128, 1, 1, 0x1000, None) == 1
    assert b"need spectra" in lib.rsim_last_error()
    assert lib.rsim_synth_pulses(B(rd), 0x1000, 3, 1, 64, 64, 0, 128, 1, 1, 0x1000, None) == 1
    # n_doppler must be a power of two >= 2, window known
    assert lib.rsim_synth_pulses(B(rd), 0x1000, 3, 0, 64, 48, 0, 128, 1, 1, 0x1000, None) == 1
    assert lib.rsim_synth_pulses(B(rd), 0x1000, 3, 0, 64, 64, 0, 128, 9, 1, 0x1000, None) == 1


def test_python_layer_requires_cuda_tensors():
    import numpy as np
    import torch
    import paper_2408_11472_gb300 as rsim
    with pytest.raises(TypeError):
        rsim.Scatterers(*[torch.zeros(4) for _ in range(7)])
    assert rsim.spectra_range(0, 4096, 64) == (0, 65)
    assert rsim.spectra_range(100, 28, 64) == (1, 2)
    assert rsim.spectra_range(100, 29, 64) == (1, 3)
    del np


def test_missing_library_fails_loudly(tmp_path):
    """Without the built CUDA library the binding refuses to load: there is no CPU fallback."""
    from paper_2408_11472_gb300 import _lib
    with pytest.raises(ImportError, match="no CPU fallback"):
        _lib.load(str(tmp_path / "librsim.so"))
