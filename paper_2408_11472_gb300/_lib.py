"""ctypes view of librsim.so (the C ABI declared in include/rsim.h).

Argument marshalling only: structs mirroring the header, prototypes, status
checking.  Importing this module loads the in-tree library and raises if it is
missing -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import weakref

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsim.so")
# the same library compiled with -DRSIM_CHECK (kernel bounds checks; for tests)
CHECK_LIB_PATH = os.path.join(_HERE, "librsim_check.so")

RSIM_OK = 0
STATUS_NAMES = {0: "RSIM_OK", 1: "RSIM_ERR_INVALID_ARG", 2: "RSIM_ERR_CUDA",
                3: "RSIM_ERR_UNSUPPORTED", 4: "RSIM_ERR_TIMEOUT", 5: "RSIM_ERR_WORKSPACE",
                6: "RSIM_ERR_CHECK"}
PRECISIONS = {"fp64": 0, "split": 1}
WINDOWS = {"sqrt_linear": 0, "sqrt_raised_cosine": 1, "linear": 2}


class RsimError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))


class Antenna(ctypes.Structure):
    _fields_ = [("gain", ctypes.c_void_p), ("nu", ctypes.c_int32), ("nv", ctypes.c_int32),
                ("u0", ctypes.c_double), ("du", ctypes.c_double),
                ("v0", ctypes.c_double), ("dv", ctypes.c_double)]


class Radar(ctypes.Structure):
    _fields_ = [("carrier_hz", ctypes.c_double), ("prf_hz", ctypes.c_double),
                ("c_mps", ctypes.c_double), ("gate_width_m", ctypes.c_double),
                ("beamwidth_rad", ctypes.c_double), ("n_gates", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("antenna", ctypes.POINTER(Antenna))]


class Platform(ctypes.Structure):
    _fields_ = [("p0", ctypes.c_double * 3), ("v", ctypes.c_double * 3),
                ("r_ref0", ctypes.c_double), ("r_ref_rate", ctypes.c_double)]


class Scatterers(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, ctypes.c_void_p) for k in
                                          ("x", "y", "z", "vx", "vy", "vz", "nrcs")] + [
        ("origin", ctypes.c_double * 3), ("facet_area_m2", ctypes.c_double),
        ("t0", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("sets_per_launch", ctypes.c_int32), ("samples_per_group", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]

    def __repr__(self):
        return "Tuning(sets_per_launch=%d, samples_per_group=%d, persistent=%d)" % (
            self.sets_per_launch, self.samples_per_group, self.persistent)


class SurfaceState(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("z", "vx", "vy", "vz")] + [("t0", ctypes.c_double)]


MAX_STATES = 64


class WaveSpectrum(ctypes.Structure):
    _fields_ = [("coef", ctypes.c_void_p), ("L", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("spacing", ctypes.c_double), ("scale", ctypes.c_double), ("g", ctypes.c_double)]


_P = ctypes.c_void_p
_RP = ctypes.POINTER(Radar)
_PP = ctypes.POINTER(Platform)
_SP = ctypes.POINTER(Scatterers)
_I32, _I64 = ctypes.c_int32, ctypes.c_int64

PROTOTYPES = {
    "rsim_version": ([], ctypes.c_int),
    "rsim_check_build": ([], ctypes.c_int),
    "rsim_last_error": ([], ctypes.c_char_p),
    "rsim_block_scatterers": ([], ctypes.c_int),
    "rsim_workspace_size": ([_I32, _I32, _I32], ctypes.c_size_t),
    "rsim_direct_sum": ([_RP, _PP, _SP, _I64, _I32, ctypes.c_int, _P, _P, ctypes.c_size_t, _P,
                         _P], ctypes.c_int),
    "rsim_doppler_accumulate": ([_RP, _PP, _SP, _I64, _I32, _I32, _I32, ctypes.c_int, _P, _P,
                                 ctypes.c_size_t, _P, _P], ctypes.c_int),
    "rsim_synth_pulses": ([_RP, _P, _I32, _I64, _I32, _I32, _I64, _I32, ctypes.c_int,
                           ctypes.c_int, _P, _P], ctypes.c_int),
    "rsim_scatterer_cells": ([_RP, _PP, _SP, _I64, _I32, ctypes.c_int, _P, _P, _P, _P, _P],
                             ctypes.c_int),
    "rsim_scatterer_echo": ([_RP, _PP, _SP, _I64, ctypes.c_int, _P, _P], ctypes.c_int),
    "rsim_workspace_clear": ([_I32, _I32, _I32, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "rsim_doppler_accumulate_partial": ([_RP, _PP, _SP, _I64, _I32, _I32, _I32, ctypes.c_int, _P,
                                         ctypes.c_size_t, _P], ctypes.c_int),
    "rsim_workspace_finalize": ([_I32, _I32, _I32, ctypes.c_int, _P, ctypes.c_size_t, _P, _P],
                                ctypes.c_int),
    "rsim_delay_doppler": ([_RP, _PP, _P, _I64, _I32, _I32, _P, _P, _P], ctypes.c_int),
    "rsim_surface_workspace_size": ([_I32], ctypes.c_size_t),
    "rsim_surface_prepare": ([ctypes.POINTER(WaveSpectrum), _P, ctypes.c_size_t, _P], ctypes.c_int),
    "rsim_surface_at": ([ctypes.POINTER(WaveSpectrum), ctypes.c_double, _P, _P, _P, _P, _P,
                         ctypes.c_size_t, _P], ctypes.c_int),
    "rsim_synth_pulses_backward": ([_RP, _P, _I32, _I64, _I32, _I32, _I64, _I32, ctypes.c_int,
                                    ctypes.c_int, _P, _P], ctypes.c_int),
    "rsim_doppler_accumulate_backward": ([_RP, _PP, _SP, _I64, _I32, _I32, _I32, ctypes.c_int,
                                          _P, _P, _P, _P], ctypes.c_int),
    "rsim_direct_sum_backward": ([_RP, _PP, _SP, _I64, _I32, ctypes.c_int, _P, _P, _P, _P],
                                 ctypes.c_int),
    "rsim_batched_workspace_size": ([_I32, _I32, _I32, _I32], ctypes.c_size_t),
    "rsim_doppler_accumulate_batched": ([_RP, _PP, _I32, _SP, _I64, _I32, _I32, _I32, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Tuning),
                                         _P, ctypes.c_size_t, _P], ctypes.c_int),
    "rsim_autotune_batched": ([_RP, _PP, _I32, _SP, _I64, _I32, _I32, _I32, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_void_p), _P, ctypes.c_size_t, _I32,
                               ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_double), _P],
                              ctypes.c_int),
    "rsim_doppler_accumulate_noalloc": ([_RP, _PP, _SP, _I64, _I32, _I32, _I32, ctypes.c_int,
                                         _P, _P], ctypes.c_int),
    "rsim_doppler_accumulate_states": ([_RP, _PP, _SP, _I64, _I32, ctypes.POINTER(SurfaceState),
                                        _I32, _I32, ctypes.c_int, _P, ctypes.c_size_t, _P],
                                       ctypes.c_int),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            "librsim.so is not built (%s); run `python paper_2408_11472_gb300/build.py` "
            "(the CUDA library is required; there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (args, res) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = load()


def check(status: int) -> None:
    if status != RSIM_OK:
        msg = lib.rsim_last_error()
        raise RsimError(status, msg.decode() if msg else "")


_DEVICE_TABLES = weakref.WeakKeyDictionary()


def _device_table(ant):
    """complex64 device copy of a tabulated pattern (``ant.gain`` [nv, nu], numpy or torch),
    made once per table object and device, kept as long as the table object lives."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    per = _DEVICE_TABLES.setdefault(ant, {})
    t = per.get(dev)
    if t is None:
        g = ant.gain
        t = (g if isinstance(g, torch.Tensor) else torch.from_numpy(
            __import__("numpy").asarray(g))).to(device=dev, dtype=torch.complex64).contiguous()
        if t.dim() != 2:
            raise ValueError("antenna gain must be a 2-D [nv, nu] array")
        per[dev] = t
    return t


def make_radar(r) -> Radar:
    out = Radar(float(r.carrier_hz), float(r.prf_hz), float(r.c_mps), float(r.gate_width_m),
                float(r.beamwidth_rad), int(r.n_gates), 0, None)
    ant = getattr(r, "antenna", None)
    if ant is not None:
        t = _device_table(ant)
        a = Antenna(t.data_ptr(), int(t.shape[1]), int(t.shape[0]), float(ant.u0), float(ant.du),
                    float(ant.v0), float(ant.dv))
        out.antenna = ctypes.pointer(a)
        out._keep = (a, t)
    return out


def make_platform(p) -> Platform:
    return Platform((ctypes.c_double * 3)(*[float(v) for v in p.p0]),
                    (ctypes.c_double * 3)(*[float(v) for v in p.v]), float(p.r_ref0),
                    float(p.r_ref_rate))
