"""FP64 CPU oracle of the scatterer -> IQ summation (regular and fast mode).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the library's product path never
imports, links or runs anything here, and nothing here imports the library.

Independent restatements of the paper's method live here:

* ``rsim_oracle.c`` (plain C, OpenMP over fixed chunks, compensated sums,
  direct O(N_d^2) DFT), wrapped by :class:`Oracle` through ctypes;
* ``bruteforce.py`` (vectorised numpy, for tiny inputs), used to pin the C code;
* ``delay_doppler.py`` (numpy): delay-Doppler focusing of the IQ (Section IV.C);
* ``surface.py`` (numpy): the spectral surface update at each update time.

Pins (see ``tests/test_oracle_*.py``): closed-form point-scatterer gate, phase
and amplitude; the antenna 3 dB point; update-pulse identity; static scene;
on-bin Doppler tones of both signs; Parseval; DFT vs ``numpy.fft``;
incoherent power; Eq. (1) variance conservation; finite differences for the
adjoint; brute force on tiny inputs.  The fast-vs-regular agreement away from
update pulses is an approximation property of the method: parity unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsim_oracle.c")
_LIB = os.path.join(_HERE, "librsim_oracle.so")
_lock = threading.Lock()

WINDOWS = {"sqrt_linear": 0, "sqrt_raised_cosine": 1, "linear": 2}


# compiler and flags of the C oracle (reported beside its timings)
CC = "gcc"
CFLAGS = ["-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, IEEE double, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = [CC] + CFLAGS + ["-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class _Radar(ctypes.Structure):
    _fields_ = [("carrier_hz", ctypes.c_double), ("prf_hz", ctypes.c_double),
                ("c_mps", ctypes.c_double), ("gate_width_m", ctypes.c_double),
                ("beamwidth_rad", ctypes.c_double), ("n_gates", ctypes.c_int32),
                ("ant_nu", ctypes.c_int32), ("ant", ctypes.POINTER(ctypes.c_double)),
                ("ant_nv", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("ant_u0", ctypes.c_double), ("ant_du", ctypes.c_double),
                ("ant_v0", ctypes.c_double), ("ant_dv", ctypes.c_double)]


class _Platform(ctypes.Structure):
    _fields_ = [("p0", ctypes.c_double * 3), ("v", ctypes.c_double * 3),
                ("r_ref0", ctypes.c_double), ("r_ref_rate", ctypes.c_double)]


_FP = ctypes.POINTER(ctypes.c_float)
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int32)


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", _FP), ("y", _FP), ("z", _FP), ("vx", _FP),
                ("vy", _FP), ("vz", _FP), ("nrcs", _FP), ("origin", ctypes.c_double * 3),
                ("area", ctypes.c_double), ("t0", ctypes.c_double)]


def _radar(r) -> _Radar:
    """ctypes radar; a tabulated antenna pattern (``r.antenna``: complex ``gain[nv, nu]``,
    grid ``u0, du, v0, dv``) rides along as float64 (re, im) pairs, kept alive by the struct."""
    out = _Radar(float(r.carrier_hz), float(r.prf_hz), float(r.c_mps), float(r.gate_width_m),
                 float(r.beamwidth_rad), int(r.n_gates), 0, None, 0, 0, 0.0, 1.0, 0.0, 1.0)
    ant = getattr(r, "antenna", None)
    if ant is not None:
        g = np.asarray(ant.gain, dtype=np.complex128)
        if g.ndim != 2 or min(g.shape) < 2:
            raise ValueError("antenna gain must be [nv, nu] with nu, nv >= 2")
        buf = np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))
        out.ant = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        out.ant_nv, out.ant_nu = int(g.shape[0]), int(g.shape[1])
        out.ant_u0, out.ant_du = float(ant.u0), float(ant.du)
        out.ant_v0, out.ant_dv = float(ant.v0), float(ant.dv)
        out._keep = buf
    return out


def _platform(p) -> _Platform:
    return _Platform((ctypes.c_double * 3)(*p.p0), (ctypes.c_double * 3)(*p.v),
                     float(p.r_ref0), float(p.r_ref_rate))


_KEYS = ("x", "y", "z", "vx", "vy", "vz", "nrcs")


def _scene(s):
    arrs = [np.ascontiguousarray(np.asarray(s[k]), dtype=np.float32) for k in _KEYS]
    n = arrs[0].size
    for a in arrs:
        if a.size != n:
            raise ValueError("scene arrays differ in length")
    sc = _Scene(n, *[a.ctypes.data_as(_FP) for a in arrs],
                (ctypes.c_double * 3)(*s.get("origin", (0.0, 0.0, 0.0))), float(s.get("area", 1.0)),
                float(s.get("t0", 0.0)))
    return sc, arrs  # keep arrays alive


def _d(a):
    return a.ctypes.data_as(_DP)


def _cplx_in(a) -> np.ndarray:
    a = np.asarray(a)
    return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1), dtype=np.float64)


def _cplx_out(buf) -> np.ndarray:
    return buf[..., 0] + 1j * buf[..., 1]


class Oracle:
    """ctypes wrapper of the C oracle (all outputs float64 / complex128 numpy arrays)."""

    def __init__(self, threads: int | None = None):
        self.lib = ctypes.CDLL(build())
        L = self.lib
        L.or_echo_batch.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                    ctypes.c_int64, ctypes.c_int64] + [_DP] * 6
        L.or_cells.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.c_int32, _IP, _IP, _DP, _DP]
        L.or_direct_sum.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_int32, _DP]
        L.or_doppler_spectra.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, _DP]
        L.or_ifft.argtypes = [_DP, ctypes.c_int64, ctypes.c_int32, _DP]
        L.or_dft.argtypes = [_DP, ctypes.c_int64, ctypes.c_int32, _DP]
        L.or_window.argtypes = [ctypes.c_int32, ctypes.c_double]
        L.or_window.restype = ctypes.c_double
        L.or_synth.argtypes = [ctypes.c_int32, _DP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                               ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _DP]
        L.or_synth.restype = ctypes.c_int
        L.or_synth_grad.argtypes = [ctypes.c_int32, _DP, ctypes.c_int32, ctypes.c_int64,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_int32, _DP]
        L.or_fast_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _DP, _DP, _DP]
        L.or_direct_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_int32, _DP, _DP, _DP]
        L.or_direct_sum_cells.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_int32, _IP, _DP]
        L.or_doppler_spectra_cells.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, _IP, _IP, _DP]
        L.or_antenna_gain.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _DP, _DP, _DP]
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_get_threads.restype = ctypes.c_int
        if threads:
            L.or_set_threads(int(threads))

    @property
    def threads(self) -> int:
        return int(self.lib.or_get_threads())

    def set_threads(self, n: int) -> None:
        self.lib.or_set_threads(int(n))

    # -- per-scatterer state -------------------------------------------------
    def echo(self, radar, platform, scene, t: float):
        sc, keep = _scene(scene)
        n = sc.n
        outs = [np.empty(n) for _ in range(6)]
        rd, pf = _radar(radar), _platform(platform)
        self.lib.or_echo_batch(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), float(t), 0, n,
                               *[_d(o) for o in outs])
        R, dR, theta, amp, cr, ci = outs
        return {"R": R, "dR": dR, "theta": theta, "amp": amp, "C": cr + 1j * ci}

    def antenna_gain(self, radar, u: float, v: float):
        """Tabulated pattern of ``radar.antenna`` at (u, v): (G, dG/du, dG/dv), complex."""
        rd = _radar(radar)
        g, gu, gv = (np.zeros(2) for _ in range(3))
        self.lib.or_antenna_gain(ctypes.byref(rd), float(u), float(v), _d(g), _d(gu), _d(gv))
        return complex(*g), complex(*gu), complex(*gv)

    def cells(self, radar, platform, scene, pulse: int, n_doppler: int):
        sc, keep = _scene(scene)
        n = sc.n
        gate = np.empty(n, np.int32)
        bins = np.empty(n, np.int32)
        gc = np.empty(n)
        bc = np.empty(n)
        rd, pf = _radar(radar), _platform(platform)
        self.lib.or_cells(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(pulse),
                          int(n_doppler), gate.ctypes.data_as(_IP), bins.ctypes.data_as(_IP),
                          _d(gc), _d(bc))
        return gate, bins, gc, bc

    # -- regular mode --------------------------------------------------------
    def direct_sum(self, radar, platform, scene, pulse0: int, n_pulses: int) -> np.ndarray:
        sc, keep = _scene(scene)
        out = np.zeros((n_pulses, radar.n_gates, 2))
        rd, pf = _radar(radar), _platform(platform)
        self.lib.or_direct_sum(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(pulse0),
                               int(n_pulses), _d(out))
        return _cplx_out(out)

    def direct_sum_cells(self, radar, platform, scene, pulse0: int, gates) -> np.ndarray:
        """Regular-mode sums with gate decisions supplied, ``gates`` int32 [n_pulses, n]."""
        sc, keep = _scene(scene)
        g = np.ascontiguousarray(gates, dtype=np.int32)
        if g.ndim != 2 or g.shape[1] != sc.n:
            raise ValueError("gates must be [n_pulses, n]")
        out = np.zeros((g.shape[0], radar.n_gates, 2))
        rd, pf = _radar(radar), _platform(platform)
        self.lib.or_direct_sum_cells(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc),
                                     int(pulse0), g.shape[0], g.ctypes.data_as(_IP), _d(out))
        return _cplx_out(out)

    # -- fast mode -----------------------------------------------------------
    def doppler_spectra_cells(self, radar, platform, scene, update0: int, n_fast: int,
                              n_doppler: int, gates, bins) -> np.ndarray:
        """Algorithm 1 rasterisation with (gate, bin) decisions supplied ([n_updates, n] each)."""
        sc, keep = _scene(scene)
        g = np.ascontiguousarray(gates, dtype=np.int32)
        b = np.ascontiguousarray(bins, dtype=np.int32)
        if g.shape != b.shape or g.ndim != 2 or g.shape[1] != sc.n:
            raise ValueError("gates/bins must be [n_updates, n]")
        out = np.zeros((g.shape[0], radar.n_gates, n_doppler, 2))
        rd, pf = _radar(radar), _platform(platform)
        self.lib.or_doppler_spectra_cells(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc),
                                          int(update0), g.shape[0], int(n_fast), int(n_doppler),
                                          g.ctypes.data_as(_IP), b.ctypes.data_as(_IP), _d(out))
        return _cplx_out(out)

    def doppler_spectra(self, radar, platform, scene, update0: int, n_updates: int, n_fast: int,
                        n_doppler: int) -> np.ndarray:
        sc, keep = _scene(scene)
        out = np.zeros((n_updates, radar.n_gates, n_doppler, 2))
        rd, pf = _radar(radar), _platform(platform)
        self.lib.or_doppler_spectra(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc),
                                    int(update0), int(n_updates), int(n_fast), int(n_doppler),
                                    _d(out))
        return _cplx_out(out)

    def ifft(self, T) -> np.ndarray:
        T = np.asarray(T)
        buf = _cplx_in(T)
        out = np.empty_like(buf)
        rows = int(np.prod(T.shape[:-1]))
        self.lib.or_ifft(_d(buf), rows, int(T.shape[-1]), _d(out))
        return _cplx_out(out)

    def dft(self, s) -> np.ndarray:
        s = np.asarray(s)
        buf = _cplx_in(s)
        out = np.empty_like(buf)
        rows = int(np.prod(s.shape[:-1]))
        self.lib.or_dft(_d(buf), rows, int(s.shape[-1]), _d(out))
        return _cplx_out(out)

    def window(self, window, d: float) -> float:
        w = WINDOWS[window] if isinstance(window, str) else int(window)
        return float(self.lib.or_window(w, float(d)))

    def synth(self, T, update0: int, n_fast: int, pulse0: int, n_pulses: int, window) -> np.ndarray:
        T = np.asarray(T)
        S, G, K = T.shape
        buf = _cplx_in(T)
        out = np.zeros((n_pulses, G, 2))
        w = WINDOWS[window] if isinstance(window, str) else int(window)
        rc = self.lib.or_synth(G, _d(buf), S, int(update0), int(n_fast), K, int(pulse0),
                               int(n_pulses), w, _d(out))
        if rc != 0:
            raise ValueError("pulse range needs spectra outside the ones given")
        return _cplx_out(out)

    def synth_grad(self, G_Y, S: int, update0: int, n_fast: int, n_doppler: int, pulse0: int,
                   window) -> np.ndarray:
        G_Y = np.asarray(G_Y)
        P, G = G_Y.shape
        buf = _cplx_in(G_Y)
        out = np.zeros((S, G, n_doppler, 2))
        w = WINDOWS[window] if isinstance(window, str) else int(window)
        self.lib.or_synth_grad(G, _d(buf), int(S), int(update0), int(n_fast), int(n_doppler),
                               int(pulse0), P, w, _d(out))
        return _cplx_out(out)

    def fast_grad(self, radar, platform, scene, update0: int, n_fast: int, G_T):
        G_T = np.asarray(G_T)
        S, G, K = G_T.shape
        sc, keep = _scene(scene)
        buf = _cplx_in(G_T)
        gz = np.zeros(sc.n)
        gs = np.zeros(sc.n)
        rd, pf = _radar(radar), _platform(platform)
        self.lib.or_fast_grad(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(update0),
                              int(S), int(n_fast), int(K), _d(buf), _d(gz), _d(gs))
        return gz, gs

    def direct_grad(self, radar, platform, scene, pulse0: int, G_Y):
        G_Y = np.asarray(G_Y)
        P, G = G_Y.shape
        sc, keep = _scene(scene)
        buf = _cplx_in(G_Y)
        gz = np.zeros(sc.n)
        gs = np.zeros(sc.n)
        rd, pf = _radar(radar), _platform(platform)
        self.lib.or_direct_grad(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(pulse0),
                                int(P), _d(buf), _d(gz), _d(gs))
        return gz, gs

    # -- composite -----------------------------------------------------------
    def simulate_fast(self, radar, platform, scene, n_pulses: int, n_fast: int, n_doppler: int,
                      window, pulse0: int = 0):
        """Spectra for every update the pulse range needs, then the blended pulses."""
        u0 = pulse0 // n_fast
        u1 = (pulse0 + n_pulses - 1) // n_fast + 1
        T = self.doppler_spectra(radar, platform, scene, u0, u1 - u0 + 1, n_fast, n_doppler)
        Y = self.synth(T, u0, n_fast, pulse0, n_pulses, window)
        return T, Y


def n_spectra(n_pulses: int, n_fast: int) -> int:
    """Number of spectra for pulses 0..n_pulses-1: floor((P-1)/n_fast) + 2
    (the paper's 1 + n_pulses/n_fast when n_fast divides n_pulses)."""
    return (n_pulses - 1) // n_fast + 2
