"""GB300-native coherent summation of sea-surface scatterers into radar IQ range gates.

Hot path of the raw-data simulator of arXiv 2408.11472 (Monnier, Camus,
Hellouvry): regular mode (every scatterer into every pulse, Section II.A) and
the fast mode of Section III (one Doppler-spectrum pass per surface update,
Algorithm 1; batched per-gate inverse FFT, Eq. (1) weights and overlap-add,
Section III.B), plus the adjoints of both.

Every step runs in the hand-written sm_103a kernels of ``librsim.so`` behind
the C ABI of ``include/rsim.h``; this module only marshals torch tensors
(device memory, streams) into those calls.  There is no CPU fallback: importing
the package fails if the CUDA library has not been built.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import Optional, Tuple

import torch

from . import _lib
from ._lib import PRECISIONS, WINDOWS, RsimError

__all__ = [
    "Antenna", "Radar", "Platform", "Scatterers", "RsimError", "workspace_size", "direct_sum",
    "doppler_accumulate", "doppler_accumulate_noalloc", "doppler_accumulate_batched",
    "doppler_accumulate_states",
    "autotune_batched", "Tuning",
    "batched_workspace_size", "BatchedFastMode", "synth_pulses", "scatterer_cells", "scatterer_echo",
    "delay_doppler", "EvolvingSurface", "simulate_fast_evolving", "HostStreamer",
    "synth_pulses_backward",
    "doppler_accumulate_backward", "direct_sum_backward", "spectra_range", "simulate_fast",
    "FastMode", "RegularMode", "version", "PRECISIONS", "WINDOWS",
]

_KEYS = ("x", "y", "z", "vx", "vy", "vz", "nrcs")


@dataclasses.dataclass(frozen=True, eq=False)
class Antenna:
    """Two-way complex antenna pattern on a u-v grid (rsim_antenna): ``gain[j, i]`` at the
    direction cosines u = u0 + i du, v = v0 + j dv of the line of sight platform -> facet;
    numpy or torch, complex, [nv, nu].  Copied to the device once per device."""

    gain: object
    u0: float
    du: float
    v0: float
    dv: float


@dataclasses.dataclass(frozen=True)
class Radar:
    """Instrument constants (SI).  Defaults: Sentinel-3 SRAL-like Ku-band altimeter.
    ``antenna``: tabulated two-way pattern (any object with gain, u0, du, v0, dv), or None
    for the Gaussian pattern of ``beamwidth_rad``."""

    carrier_hz: float = 13.575e9
    prf_hz: float = 18_000.0
    c_mps: float = 299_792_458.0
    gate_width_m: float = 0.47
    beamwidth_rad: float = math.radians(1.3)
    n_gates: int = 128
    antenna: Optional[Antenna] = None


@dataclasses.dataclass(frozen=True)
class Platform:
    """Track P(t) = p0 + v t (scene frame) and range reference r_ref(t) = r_ref0 + r_ref_rate t."""

    p0: tuple = (0.0, 0.0, 800e3)
    v: tuple = (7_000.0, 0.0, 0.0)
    r_ref0: float = 800e3
    r_ref_rate: float = 0.0


class Scatterers:
    """Structure-of-arrays scatterer set on a CUDA device (float32, contiguous).

    Positions are relative to ``origin`` at the epoch ``t0`` (seconds); a scatterer moves as
    origin + r + v (t - t0)."""

    def __init__(self, x, y, z, vx, vy, vz, nrcs, origin=(0.0, 0.0, 0.0), area=1.0, t0=0.0):
        arrs = [x, y, z, vx, vy, vz, nrcs]
        n = arrs[0].numel()
        for a in arrs:
            if not isinstance(a, torch.Tensor) or a.dtype != torch.float32 or not a.is_cuda:
                raise TypeError("scatterer arrays must be float32 CUDA tensors")
            if a.numel() != n or not a.is_contiguous():
                raise ValueError("scatterer arrays must be contiguous and of equal length")
        self.x, self.y, self.z, self.vx, self.vy, self.vz, self.nrcs = arrs
        self.origin = tuple(float(o) for o in origin)
        self.area = float(area)
        self.t0 = float(t0)

    @classmethod
    def from_arrays(cls, d, device="cuda") -> "Scatterers":
        """Copy a dict of arrays (numpy or torch; keys x, y, z, vx, vy, vz, nrcs,
        optional origin and area) to ``device``."""
        t = [torch.as_tensor(d[k]).to(device=device, dtype=torch.float32).contiguous() for k in _KEYS]
        return cls(*t, origin=d.get("origin", (0.0, 0.0, 0.0)), area=d.get("area", 1.0),
                   t0=d.get("t0", 0.0))

    def replace(self, **kw) -> "Scatterers":
        arrs = {k: kw.get(k, getattr(self, k)) for k in _KEYS}
        return Scatterers(**arrs, origin=self.origin, area=self.area, t0=self.t0)

    @property
    def n(self) -> int:
        return self.x.numel()

    @property
    def device(self) -> torch.device:
        return self.x.device

    def c_struct(self) -> _lib.Scatterers:
        return _lib.Scatterers(self.n, *[getattr(self, k).data_ptr() for k in _KEYS],
                               (ctypes.c_double * 3)(*self.origin), self.area, self.t0)


def version() -> int:
    return int(_lib.lib.rsim_version())


def _prec(precision) -> int:
    try:
        return PRECISIONS[precision]
    except KeyError:
        raise ValueError("precision must be one of %s" % list(PRECISIONS)) from None


def _cdtype(precision) -> torch.dtype:
    return torch.complex128 if _prec(precision) == 0 else torch.complex64


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _need(t: torch.Tensor, dtype, shape, device, what):
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or t.device != device or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor of shape %s on %s"
                         % (what, dtype, tuple(shape), device))


def workspace_size(n_samples: int, n_gates: int, n_doppler: int = 1) -> int:
    """Bytes of fixed-point scratch a summation call needs (see rsim_workspace_size)."""
    return int(_lib.lib.rsim_workspace_size(int(n_samples), int(n_gates), int(n_doppler)))


def _workspace(workspace, nbytes, device):
    if workspace is None:
        return torch.empty(max(nbytes, 16), dtype=torch.uint8, device=device)
    if workspace.numel() * workspace.element_size() < nbytes:
        raise ValueError("workspace smaller than %d bytes" % nbytes)
    return workspace


def _counter(t: Optional[torch.Tensor], n: int, device) -> Optional[int]:
    if t is None:
        return None
    _need(t, torch.int64, (n,), device, "out_of_window")
    return t.data_ptr()


def direct_sum(radar, platform, scat: Scatterers, pulse0: int, n_pulses: int,
               precision: str = "split", out: Optional[torch.Tensor] = None,
               workspace: Optional[torch.Tensor] = None, stream=None,
               out_of_window: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Regular mode: IQ [n_pulses, n_gates] (+= into ``out`` if given, else a new zeroed tensor).
    ``out_of_window``: optional int64 [n_pulses] tensor; += the scatterers left out of each
    pulse (gate outside the window), as the summation decides."""
    shape = (n_pulses, radar.n_gates)
    if out is None:
        out = torch.zeros(shape, dtype=_cdtype(precision), device=scat.device)
    _need(out, _cdtype(precision), shape, scat.device, "out")
    oow = _counter(out_of_window, n_pulses, scat.device)
    ws = _workspace(workspace, workspace_size(n_pulses, radar.n_gates, 1), scat.device)
    rd, pf, sc = _lib.make_radar(radar), _lib.make_platform(platform), scat.c_struct()
    _lib.check(_lib.lib.rsim_direct_sum(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc),
                                        int(pulse0), int(n_pulses), _prec(precision),
                                        _ptr(out), _ptr(ws), ws.numel() * ws.element_size(),
                                        oow, _stream(stream)))
    return out


def doppler_accumulate(radar, platform, scat: Scatterers, update0: int, n_updates: int,
                       n_fast: int, n_doppler: int, precision: str = "split",
                       out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                       stream=None, out_of_window: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Fast-mode Doppler spectra [n_updates, n_gates, n_doppler] of updates update0.. (Algorithm 1).
    ``out_of_window``: optional int64 [n_updates] tensor; += the scatterers left out of each
    update's spectrum (gate outside the window at its first pulse), as the summation decides."""
    shape = (n_updates, radar.n_gates, n_doppler)
    if out is None:
        out = torch.zeros(shape, dtype=_cdtype(precision), device=scat.device)
    _need(out, _cdtype(precision), shape, scat.device, "out")
    oow = _counter(out_of_window, n_updates, scat.device)
    ws = _workspace(workspace, workspace_size(n_updates, radar.n_gates, n_doppler), scat.device)
    rd, pf, sc = _lib.make_radar(radar), _lib.make_platform(platform), scat.c_struct()
    _lib.check(_lib.lib.rsim_doppler_accumulate(
        ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(update0), int(n_updates),
        int(n_fast), int(n_doppler), _prec(precision), _ptr(out), _ptr(ws),
        ws.numel() * ws.element_size(), oow, _stream(stream)))
    return out


def doppler_accumulate_states(radar, platform, scat: Scatterers, update0: int, states,
                              n_fast: int, n_doppler: int, precision: str = "split",
                              workspace: Optional[torch.Tensor] = None, stream=None):
    """Spectra of updates update0 + s whose heights and velocities are states[s] = (z, vx, vy,
    vz, t0) (float32 [n] tensors and the epoch), the x, y and NRCS being ``scat``'s: added to
    the fixed-point workspace slots s (rsim_doppler_accumulate_states; clear and convert with
    rsim_workspace_clear / rsim_workspace_finalize).  At most 64 states per call."""
    n = len(states)
    if n > _lib.MAX_STATES:
        raise ValueError("at most %d states per call" % _lib.MAX_STATES)
    arr = (_lib.SurfaceState * max(n, 1))()
    for i, (z, vx, vy, vz, t0) in enumerate(states):
        for f in (z, vx, vy, vz):
            _need(f, torch.float32, (scat.n,), scat.device, "state field")
        arr[i] = _lib.SurfaceState(z.data_ptr(), vx.data_ptr(), vy.data_ptr(), vz.data_ptr(),
                                   float(t0))
    ws = workspace
    rd, pf, sc = _lib.make_radar(radar), _lib.make_platform(platform), scat.c_struct()
    _lib.check(_lib.lib.rsim_doppler_accumulate_states(
        ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(update0), n, arr, int(n_fast),
        int(n_doppler), _prec(precision), _ptr(ws), ws.numel() * ws.element_size(),
        _stream(stream)))


def doppler_accumulate_noalloc(radar, platform, scat: Scatterers, update0: int, n_updates: int,
                               n_fast: int, n_doppler: int, precision: str = "split",
                               out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """doppler_accumulate without a workspace, for callers that cannot allocate device
    memory where they run: the scratch is the library's built-in 16 MiB device array (calls
    that overlap on the GPU race on it).  ``out`` should be passed by such callers; without
    it a zeroed tensor is created here for convenience."""
    shape = (n_updates, radar.n_gates, n_doppler)
    if out is None:
        out = torch.zeros(shape, dtype=_cdtype(precision), device=scat.device)
    _need(out, _cdtype(precision), shape, scat.device, "out")
    rd, pf, sc = _lib.make_radar(radar), _lib.make_platform(platform), scat.c_struct()
    _lib.check(_lib.lib.rsim_doppler_accumulate_noalloc(
        ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(update0), int(n_updates),
        int(n_fast), int(n_doppler), _prec(precision), _ptr(out), _stream(stream)))
    return out


def batched_workspace_size(n_real: int, n_samples: int, n_gates: int, n_doppler: int) -> int:
    return int(_lib.lib.rsim_batched_workspace_size(int(n_real), int(n_samples), int(n_gates),
                                                    int(n_doppler)))


Tuning = _lib.Tuning


def _batched_args(radar, scats, n_updates, n_doppler, precision, outs, workspace):
    n_real = len(scats)
    shape = (n_updates, radar.n_gates, n_doppler)
    dev = scats[0].device if n_real else torch.device("cuda")
    if outs is None:
        outs = [torch.zeros(shape, dtype=_cdtype(precision), device=dev) for _ in range(n_real)]
    if len(outs) != n_real:
        raise ValueError("one output per scatterer set")
    for o in outs:
        _need(o, _cdtype(precision), shape, dev, "out")
    need = batched_workspace_size(n_real, n_updates, radar.n_gates, n_doppler)
    ws = _workspace(workspace, need, dev)
    arr = (_lib.Scatterers * max(n_real, 1))(*[s.c_struct() for s in scats])
    ptrs = (ctypes.c_void_p * max(n_real, 1))(*[o.data_ptr() for o in outs])
    return outs, ws, arr, ptrs


def doppler_accumulate_batched(radar, platform, scats, update0: int, n_updates: int, n_fast: int,
                               n_doppler: int, precision: str = "split", outs=None,
                               workspace: Optional[torch.Tensor] = None, stream=None,
                               tuning: Optional[Tuning] = None):
    """doppler_accumulate for a list of independent scatterer sets (realizations of the same
    track) in one launch per group of sets.  ``tuning``: launch plan (``autotune_batched``),
    None for the library's choice; every plan gives bit-identical spectra.  Returns the list
    of spectra (+= into ``outs``)."""
    outs, ws, arr, ptrs = _batched_args(radar, scats, n_updates, n_doppler, precision, outs,
                                        workspace)
    rd, pf = _lib.make_radar(radar), _lib.make_platform(platform)
    _lib.check(_lib.lib.rsim_doppler_accumulate_batched(
        ctypes.byref(rd), ctypes.byref(pf), len(scats), arr, int(update0), int(n_updates),
        int(n_fast), int(n_doppler), _prec(precision), ptrs,
        ctypes.byref(tuning) if tuning is not None else None, _ptr(ws),
        ws.numel() * ws.element_size(), _stream(stream)))
    return outs


def autotune_batched(radar, platform, scats, update0: int, n_updates: int, n_fast: int,
                     n_doppler: int, precision: str = "split", reps: int = 3, outs=None,
                     workspace: Optional[torch.Tensor] = None, stream=None):
    """Time candidate launch plans of ``doppler_accumulate_batched`` on these arguments
    (rsim_autotune_batched; synchronous) and return ``(tuning, ms)`` of the fastest.  The
    spectra in ``outs`` (allocated when None) receive unspecified values."""
    outs, ws, arr, ptrs = _batched_args(radar, scats, n_updates, n_doppler, precision, outs,
                                        workspace)
    rd, pf = _lib.make_radar(radar), _lib.make_platform(platform)
    best, ms = Tuning(), ctypes.c_double(0.0)
    _lib.check(_lib.lib.rsim_autotune_batched(
        ctypes.byref(rd), ctypes.byref(pf), len(scats), arr, int(update0), int(n_updates),
        int(n_fast), int(n_doppler), _prec(precision), ptrs, _ptr(ws),
        ws.numel() * ws.element_size(), int(reps), ctypes.byref(best), ctypes.byref(ms),
        _stream(stream)))
    return best, float(ms.value)


def _prec_of(t: torch.Tensor) -> str:
    if t.dtype == torch.complex128:
        return "fp64"
    if t.dtype == torch.complex64:
        return "split"
    raise TypeError("expected a complex64 or complex128 tensor")


def synth_pulses(radar, spectra: torch.Tensor, update0: int, n_fast: int, pulse0: int,
                 n_pulses: int, window: str = "sqrt_raised_cosine",
                 out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Post-processing of Section III.B: IQ [n_pulses, n_gates] from spectra [S, n_gates, N_d]."""
    precision = _prec_of(spectra)
    S, G, K = spectra.shape
    if G != radar.n_gates:
        raise ValueError("spectra gate axis does not match radar.n_gates")
    if not spectra.is_contiguous():
        raise ValueError("spectra must be contiguous")
    shape = (n_pulses, G)
    if out is None:
        out = torch.empty(shape, dtype=spectra.dtype, device=spectra.device)
    _need(out, spectra.dtype, shape, spectra.device, "out")
    rd = _lib.make_radar(radar)
    _lib.check(_lib.lib.rsim_synth_pulses(ctypes.byref(rd), _ptr(spectra), int(S), int(update0),
                                          int(n_fast), int(K), int(pulse0), int(n_pulses),
                                          WINDOWS[window], _prec(precision), _ptr(out),
                                          _stream(stream)))
    return out


def scatterer_cells(radar, platform, scat: Scatterers, pulse: int, n_doppler: int,
                    precision: str = "split", stream=None):
    """Per-scatterer gate and Doppler-bin decisions at pulse (pair (pulse, pulse+1)),
    with their pre-floor coordinates: (gate int32, bin int32, gate_coord f64, bin_coord f64)."""
    dev = scat.device
    gate = torch.empty(scat.n, dtype=torch.int32, device=dev)
    bins = torch.empty(scat.n, dtype=torch.int32, device=dev)
    gc = torch.empty(scat.n, dtype=torch.float64, device=dev)
    bc = torch.empty(scat.n, dtype=torch.float64, device=dev)
    rd, pf, sc = _lib.make_radar(radar), _lib.make_platform(platform), scat.c_struct()
    _lib.check(_lib.lib.rsim_scatterer_cells(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc),
                                             int(pulse), int(n_doppler), _prec(precision),
                                             _ptr(gate), _ptr(bins), _ptr(gc), _ptr(bc),
                                             _stream(stream)))
    return gate, bins, gc, bc


def scatterer_echo(radar, platform, scat: Scatterers, pulse: int, precision: str = "split",
                   stream=None) -> torch.Tensor:
    """Per-scatterer complex amplitude C_n at ``pulse`` (in or out of the range window), as
    the summation evaluates it in ``precision``: complex64 (split) or complex128 (fp64) [n]."""
    out = torch.empty(scat.n, dtype=_cdtype(precision), device=scat.device)
    rd, pf, sc = _lib.make_radar(radar), _lib.make_platform(platform), scat.c_struct()
    _lib.check(_lib.lib.rsim_scatterer_echo(ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc),
                                            int(pulse), _prec(precision), _ptr(out),
                                            _stream(stream)))
    return out


def delay_doppler(radar, platform, iq: torch.Tensor, pulse0: int = 0, burst: int = 64,
                  focused: bool = False, stream=None):
    """Delay-Doppler focusing of IQ [n_pulses, n_gates] complex64 (rsim_delay_doppler,
    Section IV.C): bursts of ``burst`` pulses, centroid correction, along-track beams,
    range-migration delay phases, multi-look.  Returns ``(multilook, beams)``: float32
    [bursts, n_gates] and, when ``focused``, complex64 [bursts, burst, n_gates] (else None)."""
    if iq.dtype != torch.complex64 or iq.dim() != 2 or iq.shape[1] != radar.n_gates:
        raise TypeError("iq must be complex64 [n_pulses, n_gates]")
    iq = iq.contiguous()
    nb = iq.shape[0] // int(burst)
    ml = torch.empty((nb, radar.n_gates), dtype=torch.float32, device=iq.device)
    beams = (torch.empty((nb, int(burst), radar.n_gates), dtype=torch.complex64, device=iq.device)
             if focused else None)
    rd, pf = _lib.make_radar(radar), _lib.make_platform(platform)
    _lib.check(_lib.lib.rsim_delay_doppler(ctypes.byref(rd), ctypes.byref(pf), _ptr(iq),
                                           int(pulse0), int(iq.shape[0]), int(burst),
                                           _ptr(beams) if beams is not None else None, _ptr(ml),
                                           _stream(stream)))
    return ml, beams


def synth_pulses_backward(radar, grad_iq: torch.Tensor, n_spectra: int, update0: int,
                          n_fast: int, n_doppler: int, pulse0: int,
                          window: str = "sqrt_raised_cosine", out: Optional[torch.Tensor] = None,
                          stream=None) -> torch.Tensor:
    """Adjoint of synth_pulses: dL/dT [n_spectra, n_gates, n_doppler] from dL/dY."""
    precision = _prec_of(grad_iq)
    P, G = grad_iq.shape
    shape = (n_spectra, G, n_doppler)
    if out is None:
        out = torch.empty(shape, dtype=grad_iq.dtype, device=grad_iq.device)
    _need(out, grad_iq.dtype, shape, grad_iq.device, "out")
    grad_iq = grad_iq.contiguous()
    rd = _lib.make_radar(radar)
    _lib.check(_lib.lib.rsim_synth_pulses_backward(
        ctypes.byref(rd), _ptr(grad_iq), int(n_spectra), int(update0), int(n_fast), int(n_doppler),
        int(pulse0), int(P), WINDOWS[window], _prec(precision), _ptr(out), _stream(stream)))
    return out


def _grads(scat, grad_z, grad_nrcs):
    if grad_z is None:
        grad_z = torch.zeros(scat.n, dtype=torch.float32, device=scat.device)
    if grad_nrcs is None:
        grad_nrcs = torch.zeros(scat.n, dtype=torch.float32, device=scat.device)
    for t in (grad_z, grad_nrcs):
        _need(t, torch.float32, (scat.n,), scat.device, "gradient buffer")
    return grad_z, grad_nrcs


def doppler_accumulate_backward(radar, platform, scat: Scatterers, update0: int, n_fast: int,
                                grad_spectra: torch.Tensor, grad_z=None, grad_nrcs=None,
                                stream=None) -> Tuple[torch.Tensor, torch.Tensor]:
    """Adjoint of doppler_accumulate: (dL/dz, dL/dnrcs) accumulated into float32 [n] buffers."""
    precision = _prec_of(grad_spectra)
    S, G, K = grad_spectra.shape
    grad_spectra = grad_spectra.contiguous()
    grad_z, grad_nrcs = _grads(scat, grad_z, grad_nrcs)
    rd, pf, sc = _lib.make_radar(radar), _lib.make_platform(platform), scat.c_struct()
    _lib.check(_lib.lib.rsim_doppler_accumulate_backward(
        ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(update0), int(S), int(n_fast),
        int(K), _prec(precision), _ptr(grad_spectra), _ptr(grad_z), _ptr(grad_nrcs),
        _stream(stream)))
    return grad_z, grad_nrcs


def direct_sum_backward(radar, platform, scat: Scatterers, pulse0: int, grad_iq: torch.Tensor,
                        grad_z=None, grad_nrcs=None, stream=None):
    """Adjoint of direct_sum: (dL/dz, dL/dnrcs) accumulated into float32 [n] buffers."""
    precision = _prec_of(grad_iq)
    P, G = grad_iq.shape
    grad_iq = grad_iq.contiguous()
    grad_z, grad_nrcs = _grads(scat, grad_z, grad_nrcs)
    rd, pf, sc = _lib.make_radar(radar), _lib.make_platform(platform), scat.c_struct()
    _lib.check(_lib.lib.rsim_direct_sum_backward(
        ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(pulse0), int(P),
        _prec(precision), _ptr(grad_iq), _ptr(grad_z), _ptr(grad_nrcs), _stream(stream)))
    return grad_z, grad_nrcs


def spectra_range(pulse0: int, n_pulses: int, n_fast: int) -> Tuple[int, int]:
    """(update0, n_spectra) of the updates whose spectra the pulses [pulse0, pulse0+n_pulses)
    blend: floor(pulse0/n_fast) .. floor((pulse0+n_pulses-1)/n_fast) + 1."""
    u0 = pulse0 // n_fast
    u1 = (pulse0 + n_pulses - 1) // n_fast + 1
    return u0, u1 - u0 + 1


def simulate_fast(radar, platform, scat: Scatterers, n_pulses: int, n_fast: int, n_doppler: int,
                  window: str = "sqrt_raised_cosine", precision: str = "split", pulse0: int = 0,
                  workspace=None, spectra=None, out=None, stream=None):
    """Fast mode end to end: spectra of every update the pulses need, then the blended IQ.
    Returns (spectra [S, G, N_d], iq [n_pulses, G])."""
    u0, S = spectra_range(pulse0, n_pulses, n_fast)
    if spectra is not None:
        spectra.zero_()
    T = doppler_accumulate(radar, platform, scat, u0, S, n_fast, n_doppler, precision,
                           out=spectra, workspace=workspace, stream=stream)
    Y = synth_pulses(radar, T, u0, n_fast, pulse0, n_pulses, window, out=out, stream=stream)
    return T, Y


class HostStreamer:
    """Fast mode from scatterer arrays in pinned host memory, with the host-to-device copies
    overlapped with the scatterer pass.  Device buffers come in two sets, so the copies of
    one run overlap the summation of the previous run: for a stream of runs one block
    (``chunks=1``, the default) hides the copies entirely.  For the latency of a single run
    the set can be cut into ``chunks`` blocks of whole summation blocks (1024 scatterers,
    ``rsim_block_scatterers()``; "waves": one block per full wave of CTAs), block i+1
    copied while block i is summed (the summation
    adds, so the blocks' sums make the set's; every scatterer keeps its FP64 reference
    point).  All blocks add into one fixed-point workspace, so the spectra are bit-identical to a
    single call on the whole set.  Buffers and workspace are allocated once.

    ``run(..., host_out=pinned)`` also reads the IQ back into a pinned host tensor on a
    read-back stream of its own, so the copy overlaps the scatterer pass of the next run; the
    next run's post-processing waits for it before it rewrites the device IQ.  The host
    tensor holds the result once ``readback_done`` has completed (``synchronize()`` it, or
    ``wait_readback(stream)`` to order a stream after it)."""

    def __init__(self, n: int, n_gates: int, n_doppler: int, max_spectra: int,
                 chunks=None, device="cuda", precision: str = "split"):
        self.n, self.precision = int(n), precision
        self.dev = torch.device(device)
        blk = int(_lib.lib.rsim_block_scatterers())
        nb = (self.n + blk - 1) // blk
        if chunks is None:
            chunks = 1
        elif chunks == "waves":
            # blocks of whole waves of CTAs (6 resident per SM), so no launch ends in a
            # partly filled wave
            wave = 6 * torch.cuda.get_device_properties(self.dev).multi_processor_count
            chunks = max(1, (nb + wave - 1) // wave)
        self.chunks = max(1, int(chunks))
        # two sets of device buffers: the copies of one run overlap the summation of the last
        self.sets = [{k: torch.empty(self.n, dtype=torch.float32, device=self.dev) for k in _KEYS}
                     for _ in range(2)]
        self.released = [torch.cuda.Event() for _ in range(2)]
        self.turn = 0
        self.ws = torch.empty(max(16, workspace_size(max_spectra, n_gates, n_doppler)),
                              dtype=torch.uint8, device=self.dev)
        self.copy_stream = torch.cuda.Stream(device=self.dev)
        if chunks is not None and self.chunks > 1 and nb >= self.chunks:
            edges = [min(self.n, (nb * i // self.chunks) * blk) for i in range(self.chunks + 1)]
        else:
            per = (nb + self.chunks - 1) // self.chunks          # whole waves, last one short
            edges = [min(self.n, i * per * blk) for i in range(self.chunks + 1)]
        self.ranges = [(a, b) for a, b in zip(edges[:-1], edges[1:]) if b > a]
        self.events = [torch.cuda.Event() for _ in self.ranges]
        self.readback_stream = torch.cuda.Stream(device=self.dev)
        self.readback_done = None      # event after the last IQ read-back, if any

    def wait_readback(self, stream=None):
        """Order ``stream`` (default: the current one) after the last IQ read-back."""
        if self.readback_done is not None:
            (stream or torch.cuda.current_stream(self.dev)).wait_event(self.readback_done)

    def run(self, radar, platform, host: dict, n_pulses: int, n_fast: int, n_doppler: int,
            window: str = "sqrt_raised_cosine", pulse0: int = 0, spectra=None, out=None,
            host_out=None):
        """host: pinned CPU float32 arrays x, y, z, vx, vy, vz, nrcs [n] (+ origin, area, t0).
        Returns (spectra, iq) on the device, enqueued on the current stream.  host_out: an
        optional pinned CPU tensor [n_pulses, n_gates] of the IQ dtype that receives the IQ
        through the read-back stream (complete once ``readback_done`` has completed)."""
        u0, S = spectra_range(pulse0, n_pulses, n_fast)
        if host_out is not None:
            if (host_out.device.type != "cpu" or not host_out.is_pinned()
                    or tuple(host_out.shape) != (n_pulses, radar.n_gates)
                    or host_out.dtype != _cdtype(self.precision) or not host_out.is_contiguous()):
                raise ValueError("host_out must be a contiguous pinned CPU tensor [n_pulses, "
                                 "n_gates] of the IQ dtype")
        cur = torch.cuda.current_stream(self.dev)
        T = spectra
        if T is None:
            T = torch.zeros((S, radar.n_gates, n_doppler), dtype=_cdtype(self.precision),
                            device=self.dev)
        else:
            T.zero_()
        buf, rel = self.sets[self.turn], self.released[self.turn]
        self.turn ^= 1
        self.copy_stream.wait_event(rel)          # this set's last summation has read it
        with torch.cuda.stream(self.copy_stream):
            for (a, b), ev in zip(self.ranges, self.events):
                for k in _KEYS:
                    buf[k][a:b].copy_(host[k][a:b], non_blocking=True)
                ev.record(self.copy_stream)
        origin, area, t0 = host.get("origin", (0.0, 0.0, 0.0)), host.get("area", 1.0), host.get("t0", 0.0)
        G, nbytes = radar.n_gates, self.ws.numel()
        rd, pf, prec = _lib.make_radar(radar), _lib.make_platform(platform), _prec(self.precision)
        st = _stream(cur)
        # one fixed-point workspace for all blocks: the spectra are bit-identical to
        # a single call on the whole set
        _lib.check(_lib.lib.rsim_workspace_clear(S, G, n_doppler, _ptr(self.ws), nbytes, st))
        for (a, b), ev in zip(self.ranges, self.events):
            cur.wait_event(ev)
            part = Scatterers(*[buf[k][a:b] for k in _KEYS], origin=origin, area=area, t0=t0)
            sc = part.c_struct()
            _lib.check(_lib.lib.rsim_doppler_accumulate_partial(
                ctypes.byref(rd), ctypes.byref(pf), ctypes.byref(sc), int(u0), int(S), int(n_fast),
                int(n_doppler), prec, _ptr(self.ws), nbytes, st))
        rel.record(cur)
        _lib.check(_lib.lib.rsim_workspace_finalize(S, G, n_doppler, prec, _ptr(self.ws), nbytes,
                                                    _ptr(T), st))
        self.wait_readback(cur)                   # the last read-back has left the device IQ
        Y = synth_pulses(radar, T, u0, n_fast, pulse0, n_pulses, window, out=out)
        if host_out is not None:
            ready = torch.cuda.Event()
            ready.record(cur)
            self.readback_stream.wait_event(ready)
            with torch.cuda.stream(self.readback_stream):
                host_out.copy_(Y, non_blocking=True)
            Y.record_stream(self.readback_stream)   # Y stays allocated until the copy is done
            self.readback_done = torch.cuda.Event()
            self.readback_done.record(self.readback_stream)
        return T, Y


class FastMode(torch.autograd.Function):
    """IQ of the fast mode as a differentiable function of scatterer heights z and NRCS.

    forward(z, nrcs, scat, radar, platform, pulse0, n_pulses, n_fast, n_doppler, window,
    precision) -> complex IQ [n_pulses, n_gates].  The backward pass runs the adjoint
    kernels (per-scatterer phase recomputed, not stored)."""

    @staticmethod
    def forward(ctx, z, nrcs, scat, radar, platform, pulse0, n_pulses, n_fast, n_doppler,
                window="sqrt_raised_cosine", precision="split"):
        s = scat.replace(z=z.detach().contiguous(), nrcs=nrcs.detach().contiguous())
        _, Y = simulate_fast(radar, platform, s, n_pulses, n_fast, n_doppler, window, precision,
                             pulse0)
        ctx.args = (s, radar, platform, pulse0, n_pulses, n_fast, n_doppler, window)
        return Y

    @staticmethod
    def backward(ctx, grad_y):
        s, radar, platform, pulse0, n_pulses, n_fast, n_doppler, window = ctx.args
        u0, S = spectra_range(pulse0, n_pulses, n_fast)
        gT = synth_pulses_backward(radar, grad_y.contiguous(), S, u0, n_fast, n_doppler, pulse0,
                                   window)
        gz, gs = doppler_accumulate_backward(radar, platform, s, u0, n_fast, gT)
        return gz, gs, None, None, None, None, None, None, None, None, None


class RegularMode(torch.autograd.Function):
    """IQ of the regular mode as a differentiable function of heights z and NRCS."""

    @staticmethod
    def forward(ctx, z, nrcs, scat, radar, platform, pulse0, n_pulses, precision="split"):
        s = scat.replace(z=z.detach().contiguous(), nrcs=nrcs.detach().contiguous())
        Y = direct_sum(radar, platform, s, pulse0, n_pulses, precision)
        ctx.args = (s, radar, platform, pulse0)
        return Y

    @staticmethod
    def backward(ctx, grad_y):
        s, radar, platform, pulse0 = ctx.args
        gz, gs = direct_sum_backward(radar, platform, s, pulse0, grad_y.contiguous())
        return gz, gs, None, None, None, None, None, None


class EvolvingSurface:
    """The sea surface regenerated at each update from its wave spectrum (rsim_surface_at;
    Algorithm 1's update_simulation): the facet grid and NRCS are fixed, heights and
    velocities are synthesised at time t by two packed L x L inverse transforms.

    ``spectrum``: dict with ``coef`` (one-sided complex coefficients [L, L]), ``scale``,
    ``spacing``, ``x``, ``y``, ``nrcs``, ``origin``, ``area`` (as ``scenegen.sea_spectrum``
    returns).  ``at(t)`` returns a Scatterers view of the surface at t (state epoch t0 = t)
    whose arrays are overwritten by the next call."""

    def __init__(self, spectrum: dict, device="cuda", g: float = 9.81):
        coef = torch.as_tensor(spectrum["coef"])
        L = int(coef.shape[0])
        if coef.dim() != 2 or coef.shape[1] != L:
            raise ValueError("coef must be [L, L]")
        self.L = L
        self.coef = coef.to(device=device, dtype=torch.complex64).contiguous()
        dev = self.coef.device
        f32 = dict(device=dev, dtype=torch.float32)
        self.x = torch.as_tensor(spectrum["x"]).to(**f32).contiguous()
        self.y = torch.as_tensor(spectrum["y"]).to(**f32).contiguous()
        self.nrcs = torch.as_tensor(spectrum["nrcs"]).to(**f32).contiguous()
        self.origin = tuple(spectrum.get("origin", (0.0, 0.0, 0.0)))
        self.area = float(spectrum.get("area", 1.0))
        self.z, self.vx, self.vy, self.vz = (torch.empty(L * L, **f32) for _ in range(4))
        self.spec = _lib.WaveSpectrum(self.coef.data_ptr(), L, 0, float(spectrum["spacing"]),
                                      float(spectrum["scale"]), float(g))
        n = int(_lib.lib.rsim_surface_workspace_size(L))
        self.workspace = torch.empty(n, dtype=torch.uint8, device=dev)
        _lib.check(_lib.lib.rsim_surface_prepare(ctypes.byref(self.spec), _ptr(self.workspace),
                                                 n, _stream(None)))

    def new_workspace(self) -> torch.Tensor:
        """Another prepared synthesis workspace (its own copy of the tables and of the packed
        intermediate), so that two syntheses can run at once on different streams."""
        n = self.workspace.numel()
        ws = torch.empty(n, dtype=torch.uint8, device=self.workspace.device)
        _lib.check(_lib.lib.rsim_surface_prepare(ctypes.byref(self.spec), _ptr(ws), n,
                                                 _stream(None)))
        return ws

    def at(self, t: float, stream=None, fields=None, workspace=None) -> Scatterers:
        """The surface at t; ``fields``: optional (z, vx, vy, vz) float32 [L*L] tensors to
        write instead of the surface's own (e.g. a second set from ``new_fields()``, so
        one update can be synthesised while the last one is still being read);
        ``workspace``: optional one from ``new_workspace()`` instead of the surface's own."""
        ws = self.workspace if workspace is None else workspace
        if ws.numel() < self.workspace.numel() or ws.device != self.workspace.device:
            raise ValueError("workspace must come from new_workspace()")
        z, vx, vy, vz = fields if fields is not None else (self.z, self.vx, self.vy, self.vz)
        for f in (z, vx, vy, vz):
            if f.dtype != torch.float32 or f.numel() != self.L * self.L or f.device != self.z.device \
                    or not f.is_contiguous():
                raise ValueError("fields must be contiguous float32 [L*L] tensors on the surface's device")
        _lib.check(_lib.lib.rsim_surface_at(
            ctypes.byref(self.spec), float(t), _ptr(z), _ptr(vx), _ptr(vy),
            _ptr(vz), _ptr(ws), ws.numel(), _stream(stream)))
        return Scatterers(self.x, self.y, z, vx, vy, vz, self.nrcs,
                          origin=self.origin, area=self.area, t0=float(t))

    def new_fields(self):
        """A second (z, vx, vy, vz) set of buffers for ``at(..., fields=...)``."""
        return tuple(torch.empty_like(self.z) for _ in range(4))

    def field_sets(self, k: int):
        """k (z, vx, vy, vz) sets of buffers, one per update of a block."""
        return [self.new_fields() for _ in range(k)]

    def grid(self) -> Scatterers:
        """The facet grid and NRCS as a scatterer set (heights and velocities: the surface's
        own buffers; the per-update summation takes them from its states instead)."""
        return Scatterers(self.x, self.y, self.z, self.vx, self.vy, self.vz, self.nrcs,
                          origin=self.origin, area=self.area)


# updates per summation launch of the evolving surface (each needs its own field set)
EVOLVING_BLOCK = 33


def _evolving_spectra(radar, platform, surface: EvolvingSurface, u0: int, S: int, n_fast: int,
                      n_doppler: int, precision: str, T: torch.Tensor, ws: torch.Tensor,
                      stream=None, groups=None, side=None, side2=None, ws2=None):
    """Spectra T[s] (+=) of updates u0 + s, the surface regenerated at each update, in blocks of
    K updates: the K surfaces are synthesised into K field sets, then one summation launch
    (rsim_doppler_accumulate_states) adds the block's spectra to their slots of the
    fixed-point workspace; one clear before, one conversion of all slots at the end.

    ``groups``: one or two lists of K field sets (default: one of min(S, EVOLVING_BLOCK)).
    With two and a ``side`` stream the syntheses of block b + 1 run on the side stream into
    the other group while block b is summed (same kernels and inputs: the same bits).  With a
    second side stream ``side2`` and a second synthesis workspace ``ws2``
    (``surface.new_workspace()``) the block's syntheses alternate between the two, so that
    one synthesis's passes fill the SMs the other's last wave leaves idle."""
    G = radar.n_gates
    nbytes = ws.numel() * ws.element_size()
    cur = stream if stream is not None else torch.cuda.current_stream()
    st = _stream(cur)
    _lib.check(_lib.lib.rsim_workspace_clear(S, G, n_doppler, _ptr(ws), nbytes, st))
    slot = workspace_size(1, G, n_doppler)
    if groups is None:
        groups = [surface.field_sets(max(1, min(S, EVOLVING_BLOCK)))]
    K = len(groups[0])
    overlap = len(groups) > 1 and side is not None
    grid = surface.grid()
    read = [None] * len(groups)     # event after the summation that last read a group
    sides = [side] + ([side2] if (overlap and side2 is not None and ws2 is not None) else [])
    wss = [None, ws2][:len(sides)]
    if overlap:
        fork = torch.cuda.Event()
        fork.record(cur)
        for sd in sides:
            sd.wait_event(fork)
    for b, s0 in enumerate(range(0, S, K)):
        s1 = min(S, s0 + K)
        gi = b % len(groups)
        sets = groups[gi]
        if overlap and read[gi] is not None:
            for sd in sides:
                sd.wait_event(read[gi])  # the summation two blocks back has read this group
        states = []
        for i, s in enumerate(range(s0, s1)):
            t = (u0 + s) * n_fast / radar.prf_hz
            if overlap:
                surface.at(t, stream=sides[i % len(sides)], fields=sets[i],
                           workspace=wss[i % len(sides)])
            else:
                surface.at(t, stream=cur, fields=sets[i])
            states.append(sets[i] + (t,))
        if overlap:
            for sd in sides:
                made = torch.cuda.Event()
                made.record(sd)
                cur.wait_event(made)
        doppler_accumulate_states(radar, platform, grid, u0 + s0, states, n_fast, n_doppler,
                                  precision, workspace=ws[s0 * slot:], stream=cur)
        if overlap:
            read[gi] = torch.cuda.Event()
            read[gi].record(cur)
    _lib.check(_lib.lib.rsim_workspace_finalize(S, G, n_doppler, _prec(precision), _ptr(ws), nbytes,
                                                _ptr(T), st))


def simulate_fast_evolving(radar, platform, surface: EvolvingSurface, n_pulses: int, n_fast: int,
                           n_doppler: int, window: str = "sqrt_raised_cosine",
                           precision: str = "split", pulse0: int = 0,
                           workspace: Optional[torch.Tensor] = None, stream=None):
    """Fast mode with the surface regenerated at every update (Algorithm 1 in full): for each
    update i the surface at t_i = p_i / PRF, its Doppler spectrum, then the post-processing.
    ``workspace``: at least workspace_size(S, n_gates, n_doppler) bytes for the S spectra.
    Returns (spectra, iq)."""
    u0, S = spectra_range(pulse0, n_pulses, n_fast)
    G = radar.n_gates
    dev = surface.coef.device
    T = torch.zeros((S, G, n_doppler), dtype=_cdtype(precision), device=dev)
    ws = _workspace(workspace, workspace_size(S, G, n_doppler), dev)
    _evolving_spectra(radar, platform, surface, u0, S, n_fast, n_doppler, precision, T, ws, stream)
    Y = synth_pulses(radar, T, u0, n_fast, pulse0, n_pulses, window, stream=stream)
    return T, Y


class EvolvingFastMode:
    """simulate_fast_evolving with every buffer allocated once, so the whole update loop
    (per block of updates the surface syntheses and one summation launch, then the
    post-processing) can be captured into a CUDA graph (``capture()``) and replayed
    (``replay()``).  The syntheses run on two side streams (alternately, each with its own
    synthesis workspace) into two alternating groups of field sets, overlapped with the
    summations; the results are those of simulate_fast_evolving bit for bit.  ``block``:
    updates per summation launch (each needs its own field set in both groups).  ``spectra``
    and ``iq`` hold the results; ``run()`` enqueues the same work eagerly."""

    def __init__(self, radar, platform, surface: EvolvingSurface, n_pulses: int, n_fast: int,
                 n_doppler: int, window: str = "sqrt_raised_cosine", precision: str = "split",
                 pulse0: int = 0, block: int = EVOLVING_BLOCK):
        if not 1 <= block <= _lib.MAX_STATES:
            raise ValueError("block must be in [1, %d]" % _lib.MAX_STATES)
        self.radar, self.platform, self.surface = radar, platform, surface
        self.n_pulses, self.n_fast, self.n_doppler = n_pulses, n_fast, n_doppler
        self.window, self.precision, self.pulse0 = window, precision, pulse0
        self.u0, self.S = spectra_range(pulse0, n_pulses, n_fast)
        dev = surface.coef.device
        G, cdt = radar.n_gates, _cdtype(precision)
        self.spectra = torch.zeros((self.S, G, n_doppler), dtype=cdt, device=dev)
        self.iq = torch.empty((n_pulses, G), dtype=cdt, device=dev)
        self.workspace = torch.empty(max(16, workspace_size(self.S, G, n_doppler)),
                                     dtype=torch.uint8, device=dev)
        # two groups of field sets and side streams: block b + 1 is synthesised while block b
        # is summed
        K = max(1, min(self.S, block))
        self.groups = [surface.field_sets(K), surface.field_sets(K)]
        self.side = torch.cuda.Stream(device=dev)
        # a second synthesis stream and workspace: consecutive syntheses run two at a time
        self.side2 = torch.cuda.Stream(device=dev)
        self.ws2 = surface.new_workspace()
        self.graph = None

    def _run(self):
        self.spectra.zero_()
        _evolving_spectra(self.radar, self.platform, self.surface, self.u0, self.S, self.n_fast,
                          self.n_doppler, self.precision, self.spectra, self.workspace,
                          groups=self.groups, side=self.side, side2=self.side2, ws2=self.ws2)
        synth_pulses(self.radar, self.spectra, self.u0, self.n_fast, self.pulse0, self.n_pulses,
                     self.window, out=self.iq)

    def run(self):
        self._run()
        return self.spectra, self.iq

    def capture(self):
        """Record the whole update loop into a CUDA graph (after one eager warm-up run)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._run()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._run()
        self.graph = g
        return self

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()
        return self.spectra, self.iq


class BatchedFastMode:
    """Fast mode for many independent realizations of the same track (e.g. the ~100 surface
    realizations averaged per SWH/SSH spectrum, Section IV.D).

    Per block of ``update_block`` updates one batched spectrum launch covers every
    realization (rsim_doppler_accumulate_batched: one CTA grid shared by sets of uneven
    size, out-of-window samples culled per block); then each realization's post-processing
    runs.  All buffers are allocated up front, so the whole sequence can be captured once
    into a CUDA graph (``capture()``) and replayed (``replay()``).  ``spectra[r]`` and
    ``iq[r]`` hold realization r's results."""

    def __init__(self, radar, platform, scats, pulse0: int, n_pulses: int, n_fast: int,
                 n_doppler: int, window: str = "sqrt_raised_cosine", precision: str = "split",
                 update_block: int = 64, tuning: Optional[Tuning] = None):
        self.radar, self.platform, self.scats = radar, platform, list(scats)
        self.tuning = tuning
        self.pulse0, self.n_pulses, self.n_fast, self.n_doppler = pulse0, n_pulses, n_fast, n_doppler
        self.window, self.precision = window, precision
        self.u0, self.S = spectra_range(pulse0, n_pulses, n_fast)
        self.block = max(1, min(int(update_block), self.S))
        dev = self.scats[0].device
        cdt = _cdtype(precision)
        G = radar.n_gates
        self.spectra = [torch.zeros((self.S, G, n_doppler), dtype=cdt, device=dev) for _ in self.scats]
        self.iq = [torch.empty((n_pulses, G), dtype=cdt, device=dev) for _ in self.scats]
        self.workspace = torch.empty(
            max(16, batched_workspace_size(len(self.scats), self.block, G, n_doppler)),
            dtype=torch.uint8, device=dev)
        self.graph = None

    def _run(self):
        for T in self.spectra:
            T.zero_()
        for b0 in range(0, self.S, self.block):
            b1 = min(self.S, b0 + self.block)
            doppler_accumulate_batched(self.radar, self.platform, self.scats, self.u0 + b0, b1 - b0,
                                       self.n_fast, self.n_doppler, self.precision,
                                       outs=[T[b0:b1] for T in self.spectra],
                                       workspace=self.workspace, tuning=self.tuning)
        for T, Y in zip(self.spectra, self.iq):
            synth_pulses(self.radar, T, self.u0, self.n_fast, self.pulse0, self.n_pulses,
                         self.window, out=Y)

    def run(self):
        """Run eagerly on the current stream."""
        self._run()
        return self.iq

    def autotune(self, reps: int = 3, at_update: Optional[int] = None):
        """Choose the launch plan by timing candidates on one block of updates, the one
        starting at update ``at_update`` (default: the first; pick a block where the scenes
        are in the range window), before ``capture()``.  Returns ``(tuning, ms)``."""
        n = min(self.S, self.block)
        b0 = 0 if at_update is None else min(max(int(at_update) - self.u0, 0), self.S - n)
        self.tuning, ms = autotune_batched(
            self.radar, self.platform, self.scats, self.u0 + b0, n, self.n_fast, self.n_doppler,
            self.precision, reps=reps, outs=[T[b0:b0 + n] for T in self.spectra],
            workspace=self.workspace)
        for T in self.spectra:
            T.zero_()
        return self.tuning, ms

    def capture(self):
        """Record the whole update loop into a CUDA graph (after one eager warm-up run)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._run()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._run()
        self.graph = g
        return self

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()
        return self.iq
