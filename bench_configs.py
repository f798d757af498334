"""The other concrete runs of the measurement plan, one JSON line each (``bench.py --config K``).

    cfg 0  regular mode, 256 x 256 surface (65,536 scatterers), 64 pulses, FP64: one call
           captured in a CUDA graph and replayed (the run is launch- and FP64-bound).
    cfg 2  precision study, 4096 x 4096 surface (16.8 M scatterers), 8192 pulses, 129
           spectra: split and FP64 GPU paths, each against the FP64 oracle; residual phase
           and amplitude error per scatterer (split vs FP64) on a 1 M-scatterer sample;
           regular mode on the first 512 pulses.
    cfg 3  batched realizations: 128 surfaces of uneven side U{1024..4096} at the midpoint
           of a 100 km track (257,143 pulses, an update every 64), fast mode over the
           updates whose range window can reach the scene, autotuned launch plan, whole
           update loop captured in a CUDA graph; per-realization IQ and the mean waveform
           power.
    cfg 4  adjoint, 1024 x 1024 surface, 256 pulses: waveform-power loss against a seeded
           target, forward and backward through the autograd Function; gradient against the
           FP64 oracle's.
    nfast  fast mode against regular mode over the update interval n_fast and the Doppler
           bin count (N_d = n_fast, or 2 n_fast zero-padded), 2048 x 2048 surface.
    antenna  the 2048 x 2048 fast-mode pass with a tabulated u-v antenna pattern.
    dda    delay-Doppler focusing of the fast- and regular-mode IQ of that surface.
    surface  fast mode with the surface regenerated at every update from its spectrum.

Every input is seeded and synthetic (the generator in ``scenegen``).  The FP64 oracle runs
only inside each run's ``cpu_baseline`` leg, which times it on the host cores and returns
its output; the GPU results are compared with that output.
"""
from __future__ import annotations

import math
import os
import statistics
import time

import numpy as np

import scenegen as sg

from bench import OPS_PER_PULSE_REGULAR, OPS_PER_UPDATE  # noqa: E402  (counted there)

L2_FLUSH_BYTES = 512 << 20
_PEAKS = {}


def _alu_peaks(torch):
    """Measured pipe rates of this GPU (bench.measure_alu_peaks), once per process."""
    if not _PEAKS:
        import bench
        _PEAKS.update(bench.measure_alu_peaks(torch, "cuda:%d" % torch.cuda.current_device()))
    return _PEAKS


def _fp32_peak_ops(torch):
    """FP32 lane-operations per second: measured per SM and clock, at the clock the
    microbenchmark ran at."""
    p = _alu_peaks(torch)
    per_clk = max(p["ffma"]["ops_per_clk_per_sm"], p["ffma2"]["ops_per_clk_per_sm"])
    return per_clk * p["sms"] * p["ffma2"]["sm_mhz"] * 1e6


def _fp64_peak_flops(torch):
    p = _alu_peaks(torch)
    return 2.0 * p["dfma"]["ops_per_clk_per_sm"] * p["sms"] * p["dfma"]["sm_mhz"] * 1e6


# (begin, end) epoch seconds of every timed region of the run, for the clock record
_TIMED_WINDOWS = []


def _timed(torch, fn, reps, flush=None):
    """Median CUDA-event time (ms) of fn over reps runs after one untimed run."""
    fn()
    torch.cuda.synchronize()
    out = []
    t_begin = time.time()
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    _TIMED_WINDOWS.append((t_begin, time.time()))
    return statistics.median(out)


def _rl2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _np(t):
    return t.detach().cpu().numpy()


def _cpu_leg(fn):
    """Run an oracle computation on the host cores: (result, seconds, threads).  The time is
    the best of three runs when one takes under 20 s (the three stay under a minute)."""
    import oracle
    orc = oracle.Oracle()
    t = time.perf_counter()
    res = fn(orc)
    secs = time.perf_counter() - t
    if secs < 20.0:
        for _ in range(2):
            t = time.perf_counter()
            fn(orc)
            secs = min(secs, time.perf_counter() - t)
    return res, secs, orc.threads


def _base_line(cfg_name, metric, unit, value, higher=True, dtype="f32"):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": 1,
            "higher_is_better": higher, "dtype": dtype,
            "data": "synthetic (seeded linear deep-water wave field, lognormal NRCS)",
            "config": {"workload": cfg_name}}


# ------------------------------------------------------------------------------ cfg 0
def run_cfg0(torch, rsim, args):
    c = sg.config(0)
    rd, pf, P, L = c["radar"], c["platform"], c["n_pulses"], c["L"]
    scene = sg.sea_surface(L, c["seed"])
    dev = rsim.Scatterers.from_arrays(scene)
    N, G = dev.n, rd.n_gates
    res = {}
    for prec in ("fp64", "split"):
        cdt = torch.complex128 if prec == "fp64" else torch.complex64
        Y = torch.zeros((P, G), dtype=cdt, device="cuda")
        ws = torch.empty(rsim.workspace_size(P, G, 1), dtype=torch.uint8, device="cuda")

        def call():
            Y.zero_()
            rsim.direct_sum(rd, pf, dev, 0, P, prec, out=Y, workspace=ws)

        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            call()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            call()
        reps = 1000
        for _ in range(20):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_begin = time.time()
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        _TIMED_WINDOWS.append((t_begin, time.time()))
        ms = e0.elapsed_time(e1) / reps
        res[prec] = {"ms_per_call": round(ms, 5), "contribs_per_s": round(N * P / (ms / 1e3), 1),
                     "Y": _np(Y)}
    Yo, secs, cores = _cpu_leg(lambda orc: orc.direct_sum(rd, pf, scene, 0, P))
    line = _base_line(c["name"], "regular-mode scatterer-pulse contribs/s (FP64, graph replay)",
                      "contribs/s", res["fp64"]["contribs_per_s"], dtype="f64")
    line["config"].update({"scatterers": N, "pulses": P, "gates": G, "precision": "fp64",
                           "timing": "1000 CUDA-graph replays of one call (memset + kernel + "
                                     "finalize), inputs L2-resident (6.5 MB)"})
    line["ms_per_call"] = res["fp64"]["ms_per_call"]
    line["roofline"] = {"bound": "fp64", "note": "FP64 path: geometry, phase and pattern in FP64",
                        "achieved_contribs_per_s": res["fp64"]["contribs_per_s"],
                        "fp64_peak_tflops": round(_fp64_peak_flops(torch) / 1e12, 3),
                        "peak_basis": "measured DFMA microbenchmark"}
    line["split"] = {"ms_per_call": res["split"]["ms_per_call"],
                     "contribs_per_s": res["split"]["contribs_per_s"],
                     "roofline_frac_alu": round(N * P * OPS_PER_PULSE_REGULAR /
                                                (res["split"]["ms_per_call"] / 1e3) / _fp32_peak_ops(torch), 4)}
    line["rel_l2_vs_oracle"] = {"fp64": _rl2(res["fp64"]["Y"], Yo),
                                "split": _rl2(res["split"]["Y"], Yo)}
    line["cpu_baseline"] = {"value": round(N * P / secs, 1), "unit": "contribs/s", "cores": cores,
                            "kind": "oracle", "sample": "the whole run (%d x %d)" % (N, P),
                            "seconds": round(secs, 3)}
    line["gpu_launches"] = 2 * 1000
    return line


# ------------------------------------------------------------------------------ cfg 2
def run_cfg2(torch, rsim, args):
    c = sg.config(2)
    rd, pf, fp, P, L = c["radar"], c["platform"], c["fast"], c["n_pulses"], c["L"]
    scene = sg.sea_surface(L, c["seed"], backend="torch", device="cuda")
    dev = rsim.Scatterers.from_arrays(scene)
    N, G = dev.n, rd.n_gates
    S = (P - 1) // fp.n_fast + 2
    ws = torch.empty(rsim.workspace_size(max(S, 512), G, fp.n_doppler), dtype=torch.uint8,
                     device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    for prec in ("split", "fp64"):
        cdt = torch.complex128 if prec == "fp64" else torch.complex64
        T = torch.zeros((S, G, fp.n_doppler), dtype=cdt, device="cuda")
        Y = torch.empty((P, G), dtype=cdt, device="cuda")

        def acc():
            T.zero_()
            rsim.doppler_accumulate(rd, pf, dev, 0, S, fp.n_fast, fp.n_doppler, prec, out=T,
                                    workspace=ws)

        def syn():
            rsim.synth_pulses(rd, T, 0, fp.n_fast, 0, P, fp.window, out=Y)

        reps = 5 if prec == "split" else 2
        t_acc = _timed(torch, acc, reps, flush)
        t_syn = _timed(torch, syn, reps, flush)
        acc()
        syn()
        torch.cuda.synchronize()
        out[prec] = {"accumulate_ms": round(t_acc, 3), "synth_ms": round(t_syn, 3),
                     "iq_pulses_per_s": round(P / ((t_acc + t_syn) / 1e3), 1),
                     "scatterer_updates_per_s": round(N * S / (t_acc / 1e3), 1),
                     "T": _np(T), "Y": _np(Y)}
    # per-scatterer residual error of the split path against the FP64 path (1 M sample)
    n_s = 1 << 20
    sub = rsim.Scatterers(**{k: scene[k][:n_s] for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs")},
                          origin=scene["origin"], area=scene["area"])
    hist = {}
    for p in (0, P // 2):
        Cs = rsim.scatterer_echo(rd, pf, sub, p, "split").to(torch.complex128)
        Cd = rsim.scatterer_echo(rd, pf, sub, p, "fp64")
        ph = torch.angle(Cs * Cd.conj()).abs().cpu().numpy()
        am = ((Cs.abs() - Cd.abs()) / Cd.abs()).abs().cpu().numpy()
        edges = [0, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, math.pi]
        cnt, _ = np.histogram(ph, bins=edges)
        hist["pulse_%d" % p] = {
            "phase_err_rad": {"p50": float(np.percentile(ph, 50)), "p99": float(np.percentile(ph, 99)),
                              "p99.9": float(np.percentile(ph, 99.9)), "max": float(ph.max()),
                              "rms": float(np.sqrt(np.mean(ph ** 2))),
                              "histogram_edges": edges, "histogram_counts": cnt.tolist()},
            "amp_rel_err": {"p50": float(np.percentile(am, 50)), "max": float(am.max()),
                            "rms": float(np.sqrt(np.mean(am ** 2)))}}
    # regular mode on the first 512 pulses
    Pr = 512
    reg = {}
    wsr = torch.empty(rsim.workspace_size(Pr, G, 1), dtype=torch.uint8, device="cuda")
    for prec in ("split", "fp64"):
        cdt = torch.complex128 if prec == "fp64" else torch.complex64
        Yr = torch.zeros((Pr, G), dtype=cdt, device="cuda")

        def dsum():
            Yr.zero_()
            rsim.direct_sum(rd, pf, dev, 0, Pr, prec, out=Yr, workspace=wsr)

        t = _timed(torch, dsum, 3 if prec == "split" else 1, flush)
        dsum()
        torch.cuda.synchronize()
        reg[prec] = {"ms": round(t, 3), "contribs_per_s": round(N * Pr / (t / 1e3), 1), "Y": _np(Yr)}
    # the FP64 oracle on the host cores: the whole scatterer pass and post-processing
    host = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in scene.items()}

    def oracle_run(orc):
        To = orc.doppler_spectra(rd, pf, host, 0, S, fp.n_fast, fp.n_doppler)
        Yo = orc.synth(To, 0, fp.n_fast, 0, P, fp.window)
        return To, Yo

    (To, Yo), secs, cores = _cpu_leg(oracle_run)
    # the same oracle summing over the GPU's own (gate, bin) decisions, every 8th update:
    # separates arithmetic error from cell flips of scatterers within rounding of an edge
    same_cells = {}
    for prec in ("split", "fp64"):
        num = den = 0.0
        for u in range(0, S, 8):
            g, b, _, _ = rsim.scatterer_cells(rd, pf, dev, u * fp.n_fast, fp.n_doppler, prec)
            Tc, _, _ = _cpu_leg(lambda orc: orc.doppler_spectra_cells(
                rd, pf, host, u, fp.n_fast, fp.n_doppler, _np(g)[None, :], _np(b)[None, :]))
            num += float(np.sum(np.abs(out[prec]["T"][u] - Tc[0]) ** 2))
            den += float(np.sum(np.abs(Tc[0]) ** 2))
        same_cells[prec] = math.sqrt(num / den)
    line = _base_line(c["name"], "fast-mode IQ pulses/s (split) with rel L2 vs FP64 oracle",
                      "IQ pulses/s", out["split"]["iq_pulses_per_s"])
    line["config"].update({"scatterers": N, "pulses": P, "spectra": S, "gates": G,
                           "doppler_bins": fp.n_doppler, "window": fp.window,
                           "l2": "flushed before each timed call"})
    for prec in ("split", "fp64"):
        o = out[prec]
        line[prec] = {k: o[k] for k in ("accumulate_ms", "synth_ms", "iq_pulses_per_s",
                                        "scatterer_updates_per_s")}
        line[prec]["rel_l2_vs_oracle"] = {"spectra": _rl2(o["T"], To), "iq": _rl2(o["Y"], Yo),
                                          "spectra_same_cells": same_cells[prec]}
    line["split"]["roofline_frac_alu"] = round(
        N * S * OPS_PER_UPDATE / (out["split"]["accumulate_ms"] / 1e3) / _fp32_peak_ops(torch), 4)
    line["split_vs_fp64_gpu"] = {"rel_l2_spectra": _rl2(out["split"]["T"], out["fp64"]["T"]),
                                 "rel_l2_iq": _rl2(out["split"]["Y"], out["fp64"]["Y"])}
    line["residual_error_split_vs_fp64_per_scatterer"] = dict(hist, sample="first %d scatterers" % n_s)
    line["regular_first_512_pulses"] = {
        "split_contribs_per_s": reg["split"]["contribs_per_s"], "split_ms": reg["split"]["ms"],
        "fp64_contribs_per_s": reg["fp64"]["contribs_per_s"], "fp64_ms": reg["fp64"]["ms"],
        "rel_l2_split_vs_fp64": _rl2(reg["split"]["Y"], reg["fp64"]["Y"])}
    line["cpu_baseline"] = {"value": round(P / secs, 3), "unit": "IQ pulses/s", "cores": cores,
                            "kind": "oracle", "sample": "the whole run (all %d spectra + "
                            "post-processing of %d pulses)" % (S, P), "seconds": round(secs, 2)}
    line["gpu_launches"] = None
    return line


# ------------------------------------------------------------------------------ cfg 3
def active_updates(rd, pf, half_extent_m, n_fast, S_total, margin_m=8.0):
    """Updates whose range window can reach a scene of half-width half_extent_m centred at
    the origin (flat earth, nadir track along x): the nearest point of the scene to nadir
    must lie no farther in range than the window's far edge (plus margin_m for heights)."""
    half_window = rd.n_gates / 2.0 * rd.gate_width_m
    us = np.arange(S_total)
    t = us * n_fast / rd.prf_hz
    px = pf.p0[0] + pf.v[0] * t
    dx = np.maximum(np.abs(px) - half_extent_m, 0.0)
    H = pf.p0[2]
    excess = np.sqrt(H * H + dx * dx) - (pf.r_ref0 + pf.r_ref_rate * t)
    act = us[excess <= half_window + margin_m]
    return int(act.min()), int(act.max()) + 1


def run_cfg3(torch, rsim, args):
    c = sg.config(3)
    rd, fp = c["radar"], c["fast"]
    P_track = 257_143
    pf = sg.nadir_track(P_track)
    sides = sg.cfg3_sides(128, 3)
    n_real = int(os.environ.get("RSIM_CFG3_REALIZATIONS", len(sides)))
    sides = sides[:n_real]
    S_total = (P_track - 1) // fp.n_fast + 2
    u_lo, u_hi = active_updates(rd, pf, sides.max() / 2.0, fp.n_fast, S_total)
    t_gen = time.perf_counter()
    scats = []
    t_mid = P_track / (2.0 * rd.prf_hz)
    for r, L in enumerate(sides):
        d = sg.sea_surface(int(L), 1000 + r, backend="torch", device="cuda")
        d["t0"] = t_mid                   # each surface's state is given at the nadir crossing
        scats.append(rsim.Scatterers.from_arrays(d))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    pulse0 = u_lo * fp.n_fast
    n_pulses = (u_hi - 1 - u_lo) * fp.n_fast
    bfm = rsim.BatchedFastMode(rd, pf, scats, pulse0, n_pulses, fp.n_fast, fp.n_doppler,
                               fp.window, "split", update_block=64)
    u_mid = P_track // 2 // fp.n_fast
    tuning, tune_ms = bfm.autotune(reps=2, at_update=u_mid - bfm.block // 2)
    steps = max(1, min(args.steps, 3))

    def replay_ms():
        bfm.capture()
        bfm.replay()
        torch.cuda.synchronize()
        times = []
        t_begin = time.time()
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bfm.replay()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        _TIMED_WINDOWS.append((t_begin, time.time()))
        return statistics.median(times)

    # the other form of the autotuned plan (persistent <-> one CTA per work item), then the
    # autotuned plan itself (whose results the rest of the run reads)
    other = rsim.Tuning(tuning.sets_per_launch, tuning.samples_per_group,
                        0 if tuning.persistent else 4)
    bfm.tuning = other
    ms_other = replay_ms()
    bfm.tuning = tuning
    ms = replay_ms()
    N_tot = int(sum(s.n for s in scats))
    S = bfm.S
    mean_power = torch.zeros((n_pulses, rd.n_gates), dtype=torch.float64, device="cuda")
    for y in bfm.iq:
        mean_power += y.abs().to(torch.float64) ** 2
    mean_power /= len(bfm.iq)
    # oracle leg: the smallest realization over 8 updates around the nadir crossing
    r_min = int(np.argmin(sides))
    S_chk = 8
    T_gpu = rsim.doppler_accumulate(rd, pf, scats[r_min], u_mid - S_chk // 2, S_chk, fp.n_fast,
                                    fp.n_doppler, "split")
    sm = scats[r_min]
    host = {k: getattr(sm, k).cpu().numpy() for k in ("x", "y", "z", "vx", "vy", "vz", "nrcs")}
    host.update(origin=sm.origin, area=sm.area, t0=sm.t0)
    To, secs, cores = _cpu_leg(lambda orc: orc.doppler_spectra(
        rd, pf, host, u_mid - S_chk // 2, S_chk, fp.n_fast, fp.n_doppler))
    # the batched spectra of those updates are bit-identical to the single call above
    Tb = bfm.spectra[r_min][u_mid - S_chk // 2 - bfm.u0: u_mid + S_chk // 2 - bfm.u0]
    line = _base_line(c["name"], "batched fast-mode realization IQ pulses/s (split)",
                      "IQ pulses/s", round(n_real * n_pulses / (ms / 1e3), 1))
    line["config"].update({
        "realizations": n_real, "side_min": int(sides.min()), "side_max": int(sides.max()),
        "scatterers_total": N_tot, "track_pulses": P_track, "active_updates": [bfm.u0, bfm.u0 + S],
        "pulses_per_realization": n_pulses, "spectra_per_realization": S,
        "update_block": bfm.block, "tuning": {"sets_per_launch": tuning.sets_per_launch,
                                              "samples_per_group": tuning.samples_per_group,
                                              "persistent": tuning.persistent},
        "graph": "whole update loop (zeroing, batched spectrum launches, post-processing) "
                 "captured once, replayed"})
    line["ms_per_step"] = round(ms, 3)
    line["launch_forms"] = {
        ("persistent" if tuning.persistent else "cta_per_item") + "_autotuned_ms": round(ms, 3),
        ("cta_per_item" if tuning.persistent else "persistent") + "_same_plan_ms": round(ms_other, 3)}
    line["scatterer_updates_per_s_nominal"] = round(N_tot * S / (ms / 1e3), 1)
    line["note"] = ("nominal = every scatterer at every active update; blocks whose range window "
                    "cannot be reached are skipped, so the work done is less")
    line["autotune_ms_best_block"] = round(tune_ms, 3)
    line["surface_generation_s"] = round(t_gen, 2)
    line["mean_waveform_power"] = {"peak_gate": int(torch.argmax(mean_power.mean(0)).item()),
                                   "peak_value": float(mean_power.mean(0).max().item()),
                                   "total": float(mean_power.sum().item())}
    line["check_vs_oracle"] = {"realization": r_min, "side": int(sides[r_min]),
                               "updates": [u_mid - S_chk // 2, u_mid + S_chk // 2],
                               "rel_l2_spectra": _rl2(_np(T_gpu), To),
                               "batched_equals_single_call": bool(torch.equal(Tb, T_gpu))}
    line["cpu_baseline"] = {"value": round(S_chk * host["x"].size / secs, 1),
                            "unit": "scatterer-updates/s", "cores": cores, "kind": "oracle",
                            "sample": "realization %d (%d^2 scatterers), %d updates" % (
                                r_min, int(sides[r_min]), S_chk), "seconds": round(secs, 2)}
    return line


# ------------------------------------------------------------------------------ cfg 4
def run_cfg4(torch, rsim, args):
    c = sg.config(4)
    rd, pf, fp, P, L = c["radar"], c["platform"], c["fast"], c["n_pulses"], c["L"]
    scene = sg.sea_surface(L, c["seed"])
    G = rd.n_gates
    # target waveform power: |Y|^2 of an independent surface (seed 4243) scaled by Exp(1)
    # noise (seed 4242)
    tgt_scene = rsim.Scatterers.from_arrays(sg.sea_surface(L, 4243))
    _, Yt = rsim.simulate_fast(rd, pf, tgt_scene, P, fp.n_fast, fp.n_doppler, fp.window, "split")
    mean_p = (Yt.abs() ** 2).mean(0).to(torch.float64).cpu().numpy()
    Pstar = torch.from_numpy(sg.target_waveform(P, G, 4242, mean_p)).to("cuda")
    res = {}
    for prec in ("split", "fp64"):
        dev = rsim.Scatterers.from_arrays(scene)
        rdt = torch.float64 if prec == "fp64" else torch.float32
        z = dev.z.clone().requires_grad_(True)        # heights and NRCS stay float32
        s = dev.nrcs.clone().requires_grad_(True)
        tgt = Pstar.to(rdt)

        def fwd_bwd():
            Y = rsim.FastMode.apply(z, s, dev, rd, pf, 0, P, fp.n_fast, fp.n_doppler, fp.window,
                                    prec)
            loss = ((Y.abs() ** 2 - tgt) ** 2).sum()
            gz, gs = torch.autograd.grad(loss, (z, s))
            # detached: no autograd graph outlives the step.  A live graph would keep the
            # leaves' AccumulateGrad nodes, which remember the stream they were created on;
            # a later captured backward would then synchronise with that (legacy default)
            # stream, which invalidates the capture
            return loss.detach(), gz, gs

        def fwd():
            with torch.no_grad():
                return rsim.FastMode.apply(z, s, dev, rd, pf, 0, P, fp.n_fast, fp.n_doppler,
                                           fp.window, prec)

        reps = 10 if prec == "split" else 3
        # the step captured once in a CUDA graph (forward, loss, autograd backward) and
        # replayed, measured first; the eager step is bound by host-side autograd and launch
        # overhead
        graph_res = None
        try:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(3):
                    fwd_bwd()
            torch.cuda.current_stream().wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                g_out = fwd_bwd()
            t_g = _timed(torch, graph.replay, reps)
            graph_res = {"forward_backward_ms": round(t_g, 3), "out": g_out}
        except Exception as e:  # noqa: BLE001 -- reported, not fatal
            graph_res = {"unavailable": "%s: %s" % (type(e).__name__, str(e)[:120])}
            torch.cuda.synchronize()
        t_f = _timed(torch, fwd, reps)
        t_fb = _timed(torch, fwd_bwd, reps)
        loss, gz, gs = fwd_bwd()
        torch.cuda.synchronize()
        if "out" in graph_res:
            g_out = graph_res.pop("out")
            graph.replay()
            torch.cuda.synchronize()
            graph_res["gradients_equal_eager"] = bool(torch.equal(g_out[1], gz) and
                                                      torch.equal(g_out[2], gs))
        res[prec] = {"forward_ms": round(t_f, 3), "forward_backward_ms": round(t_fb, 3),
                     "loss": float(loss.item()), "gz": _np(gz).astype(np.float64),
                     "gs": _np(gs).astype(np.float64), "graph": graph_res}
    S = (P - 1) // fp.n_fast + 2
    Pst = _np(Pstar)

    def oracle_grad(orc):
        To = orc.doppler_spectra(rd, pf, scene, 0, S, fp.n_fast, fp.n_doppler)
        Yo = orc.synth(To, 0, fp.n_fast, 0, P, fp.window)
        # L = sum (|Y|^2 - P*)^2, dL/dY (convention dL/dRe + j dL/dIm) = 4 (|Y|^2 - P*) Y
        GY = 4.0 * (np.abs(Yo) ** 2 - Pst) * Yo
        GT = orc.synth_grad(GY, S, 0, fp.n_fast, fp.n_doppler, 0, fp.window)
        gz, gs = orc.fast_grad(rd, pf, scene, 0, fp.n_fast, GT)
        return gz, gs

    (gz_o, gs_o), secs, cores = _cpu_leg(oracle_grad)
    N = L * L
    g_split = res["split"].get("graph") or {}
    if "forward_backward_ms" in g_split:
        line = _base_line(c["name"], "adjoint forward+backward time (split; forward, loss and "
                          "autograd backward replayed as one CUDA graph)", "ms",
                          g_split["forward_backward_ms"], higher=False)
    else:
        line = _base_line(c["name"], "adjoint forward+backward time (split, eager)", "ms",
                          res["split"]["forward_backward_ms"], higher=False)
    line["config"].update({"scatterers": N, "pulses": P, "spectra": S, "gates": G,
                           "loss": "sum over pulses and gates of (|Y|^2 - P*)^2",
                           "target": "|Y|^2 profile of a seed-4243 surface x Exp(1) (seed 4242)"})
    for prec in ("split", "fp64"):
        r = res[prec]
        line[prec] = {"forward_ms": r["forward_ms"], "forward_backward_ms": r["forward_backward_ms"],
                      "backward_ms": round(r["forward_backward_ms"] - r["forward_ms"], 3),
                      "graph_replay": r.get("graph"),
                      "grad_rel_l2_vs_oracle": {"z": float(np.linalg.norm(r["gz"] - gz_o) / np.linalg.norm(gz_o)),
                                                "nrcs": float(np.linalg.norm(r["gs"] - gs_o) / np.linalg.norm(gs_o))}}
    line["cpu_baseline"] = {"value": round(secs * 1e3, 1), "unit": "ms", "cores": cores,
                            "kind": "oracle", "sample": "the whole forward + adjoint (%d scatterers, "
                            "%d spectra, %d pulses)" % (N, S, P), "seconds": round(secs, 2)}
    return line


# ------------------------------------------------------------------------ n_fast sweep
def run_nfast_sweep(torch, rsim, args):
    """Fast mode against regular mode on the 2048 x 2048 surface over 4096 pulses, for
    update intervals n_fast in {16 .. 256} and N_d = n_fast or 2 n_fast (the zero-padded
    variant, whose segments hold the offsets -n_fast..n_fast without wrapping): time,
    speed-up and the relative difference of the mean power waveform (mean over pulses of
    |Y|^2 per gate, the comparison of the paper's Fig. 4 and Fig. 6)."""
    c = sg.config(1)
    rd, pf, P, L = c["radar"], c["platform"], c["n_pulses"], c["L"]
    window = c["fast"].window
    dev = rsim.Scatterers.from_arrays(sg.sea_surface(L, c["seed"]))
    N, G = dev.n, rd.n_gates
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    Yr = torch.zeros((P, G), dtype=torch.complex64, device="cuda")
    wsr = torch.empty(rsim.workspace_size(P, G, 1), dtype=torch.uint8, device="cuda")

    def regular():
        Yr.zero_()
        rsim.direct_sum(rd, pf, dev, 0, P, "split", out=Yr, workspace=wsr)

    t_reg = _timed(torch, regular, 3, flush)
    regular()
    torch.cuda.synchronize()
    Yr64 = Yr.to(torch.complex128)
    wf_reg = (Yr64.abs() ** 2).mean(0)
    rows = []
    for nf in (16, 32, 64, 128, 256):
        for nd in (nf, 2 * nf):
            S = (P - 1) // nf + 2
            T = torch.zeros((S, G, nd), dtype=torch.complex64, device="cuda")
            Y = torch.empty((P, G), dtype=torch.complex64, device="cuda")
            ws = torch.empty(rsim.workspace_size(S, G, nd), dtype=torch.uint8, device="cuda")

            def fast():
                T.zero_()
                rsim.doppler_accumulate(rd, pf, dev, 0, S, nf, nd, "split", out=T, workspace=ws)
                rsim.synth_pulses(rd, T, 0, nf, 0, P, window, out=Y)

            t = _timed(torch, fast, 5, flush)
            fast()
            torch.cuda.synchronize()
            Y64 = Y.to(torch.complex128)
            wf = (Y64.abs() ** 2).mean(0)
            rows.append({
                "n_fast": nf, "n_doppler": nd, "spectra": S, "ms": round(t, 3),
                "speedup_vs_regular": round(t_reg / t, 2),
                "mean_power_waveform_rel_diff": float(torch.linalg.vector_norm(wf - wf_reg) /
                                                      torch.linalg.vector_norm(wf_reg)),
                "mean_power_ratio": float(wf.sum() / wf_reg.sum()),
                "iq_rel_l2_vs_regular": float(torch.linalg.vector_norm(Y64 - Yr64) /
                                              torch.linalg.vector_norm(Yr64)),
                "update_pulses_rel_l2": float(torch.linalg.vector_norm(Y64[::nf] - Yr64[::nf]) /
                                              torch.linalg.vector_norm(Yr64[::nf]))})
    line = _base_line("nfast_sweep_2048x2048_p4096", "fast vs regular mode over n_fast and N_d",
                      "x speed-up at n_fast=64", next(r["speedup_vs_regular"] for r in rows
                                                      if r["n_fast"] == 64 and r["n_doppler"] == 64))
    line["config"].update({"scatterers": N, "pulses": P, "gates": G, "window": window,
                           "precision": "split", "l2": "flushed before each timed call"})
    line["regular_ms"] = round(t_reg, 3)
    line["sweep"] = rows
    return line


# ------------------------------------------------------------------ antenna pattern table
def run_antenna_table(torch, rsim, args):
    """The 2048 x 2048 fast-mode pass with the two-way pattern tabulated on a u-v grid
    (129 x 129 nodes over |u|, |v| <= 0.05) instead of the analytic Gaussian: time of the
    summation and of the whole step against the Gaussian run, split vs FP64 error."""
    import dataclasses
    c = sg.config(1)
    rd0, pf, fp, P, L = c["radar"], c["platform"], c["fast"], c["n_pulses"], c["L"]
    rd = dataclasses.replace(rd0, antenna=sg.antenna_table(77))
    dev = rsim.Scatterers.from_arrays(sg.sea_surface(L, c["seed"]))
    N, G = dev.n, rd.n_gates
    S = (P - 1) // fp.n_fast + 2
    ws = torch.empty(rsim.workspace_size(S, G, fp.n_doppler), dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    res = {}
    for name, radar, prec in (("gaussian", rd0, "split"), ("table", rd, "split"),
                              ("table_fp64", rd, "fp64")):
        cdt = torch.complex128 if prec == "fp64" else torch.complex64
        T = torch.zeros((S, G, fp.n_doppler), dtype=cdt, device="cuda")

        def acc():
            T.zero_()
            rsim.doppler_accumulate(radar, pf, dev, 0, S, fp.n_fast, fp.n_doppler, prec, out=T,
                                    workspace=ws)

        t = _timed(torch, acc, 10 if prec == "split" else 2, flush)
        acc()
        torch.cuda.synchronize()
        res[name] = {"accumulate_ms": round(t, 3),
                     "scatterer_updates_per_s": round(N * S / (t / 1e3), 1), "T": _np(T)}
    line = _base_line("fast_2048x2048_p4096_antenna_table", "fast-mode scatterer pass with a "
                      "tabulated antenna pattern", "scatterer-updates/s",
                      res["table"]["scatterer_updates_per_s"])
    line["config"].update({"scatterers": N, "spectra": S, "table": "129 x 129 complex, |u|,|v| <= 0.05",
                           "l2": "flushed before each timed call"})
    for k in ("gaussian", "table", "table_fp64"):
        line[k] = {kk: v for kk, v in res[k].items() if kk != "T"}
    line["table_cost_vs_gaussian"] = round(res["table"]["accumulate_ms"] / res["gaussian"]["accumulate_ms"], 3)
    line["split_vs_fp64_rel_l2_with_table"] = _rl2(res["table"]["T"], res["table_fp64"]["T"])
    return line


# ------------------------------------------------------------------ delay-Doppler focusing
def run_delay_doppler(torch, rsim, args):
    """Delay-Doppler focusing (Section IV.C) of the 2048 x 2048 fast-mode IQ (4096 pulses,
    64 bursts of 64) and of the regular-mode IQ of the same surface: kernel time, and the
    normalised mean multi-looked waveform of fast mode against regular mode (the comparison
    of the paper's Fig. 9)."""
    c = sg.config(1)
    rd, pf, fp, P, L = c["radar"], c["platform"], c["fast"], c["n_pulses"], c["L"]
    dev = rsim.Scatterers.from_arrays(sg.sea_surface(L, c["seed"]))
    _, Yf = rsim.simulate_fast(rd, pf, dev, P, fp.n_fast, fp.n_doppler, fp.window, "split")
    Yr = rsim.direct_sum(rd, pf, dev, 0, P, "split")
    burst = 64

    def graph_ms(fn, reps=200):
        """Device time per call: the call captured once in a CUDA graph, replayed back to
        back (the eager call's host-side marshalling would otherwise be part of the time)."""
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_begin = time.time()
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        _TIMED_WINDOWS.append((t_begin, time.time()))
        return e0.elapsed_time(e1) / reps

    t = graph_ms(lambda: rsim.delay_doppler(rd, pf, Yf, 0, burst, focused=True))
    t_ml = graph_ms(lambda: rsim.delay_doppler(rd, pf, Yf, 0, burst))
    t_eager = _timed(torch, lambda: rsim.delay_doppler(rd, pf, Yf, 0, burst, focused=True), 50)
    mlf, _ = rsim.delay_doppler(rd, pf, Yf, 0, burst)
    mlr, _ = rsim.delay_doppler(rd, pf, Yr, 0, burst)
    wf = mlf.double().mean(0)
    wr = mlr.double().mean(0)
    nf, nr = wf / wf.max(), wr / wr.max()
    nb = P // burst
    bytes_moved = P * rd.n_gates * 8 * 2 + nb * rd.n_gates * 4
    line = _base_line("delay_doppler_fast_2048x2048_p4096", "delay-Doppler focusing time",
                      "ms", round(t, 4), higher=False)
    line["config"].update({"pulses": P, "burst": burst, "bursts": nb, "gates": rd.n_gates,
                           "outputs": "focused beams + multi-look",
                           "timing": "200 CUDA-graph replays of one call, back to back (IQ "
                                     "L2-resident)"})
    line["multilook_only_ms"] = round(t_ml, 4)
    line["eager_call_ms"] = round(t_eager, 4)
    import bench
    peak, basis = bench.measured_hbm_gbs()
    line["roofline"] = {"bound": "hbm", "bytes_per_launch": bytes_moved,
                        "achieved_gbs": round(bytes_moved / (t / 1e3) / 1e9, 1),
                        "peak_gbs": peak, "peak_basis": basis,
                        "frac": round(bytes_moved / (t / 1e3) / 1e9 / peak, 4),
                        "note": "one cluster of 8 CTAs per burst (%d CTAs, the burst exchanged "
                                "through distributed shared memory): latency-bound" % (8 * nb)}
    line["normalised_mean_waveform"] = {
        "fast": [round(float(v), 5) for v in nf], "regular": [round(float(v), 5) for v in nr],
        "rel_l2_fast_vs_regular": float(torch.linalg.vector_norm(nf - nr) / torch.linalg.vector_norm(nr)),
        "peak_gate_fast": int(torch.argmax(nf)), "peak_gate_regular": int(torch.argmax(nr))}
    return line


# ------------------------------------------------------------------ surface update
def run_surface_update(torch, rsim, args):
    """Fast mode with the surface regenerated at every update (Algorithm 1 in full) on the
    2048 x 2048 surface, 4096 pulses: time of one surface synthesis (two packed 2048 x 2048
    inverse transforms), of the whole step, and against the linear-kinematics step."""
    c = sg.config(1)
    rd, pf, fp, P, L = c["radar"], c["platform"], c["fast"], c["n_pulses"], c["L"]
    spec = sg.sea_spectrum(L, c["seed"])
    surf = rsim.EvolvingSurface(spec)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    t_surf = _timed(torch, lambda: surf.at(0.1234), 20, flush)
    # the syntheses as the update loop runs them: consecutive ones alternating between two
    # streams with their own workspaces and field sets, 64 per timed run
    n_loop = 64
    side = [torch.cuda.Stream(), torch.cuda.Stream()]
    wss = [None, surf.new_workspace()]
    loop_sets = surf.field_sets(2)

    def syntheses():
        cur = torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(cur)
        for sd in side:
            sd.wait_event(fork)
        for i in range(n_loop):
            surf.at(0.1234 + 0.0035 * i, stream=side[i % 2], fields=loop_sets[i % 2],
                    workspace=wss[i % 2])
        for sd in side:
            done = torch.cuda.Event()
            done.record(sd)
            cur.wait_event(done)

    t_surf_loop = _timed(torch, syntheses, 5, flush) / n_loop
    del loop_sets
    S = (P - 1) // fp.n_fast + 2
    ws = torch.empty(rsim.workspace_size(S, rd.n_gates, fp.n_doppler), dtype=torch.uint8,
                     device="cuda")

    def evolving():
        rsim.simulate_fast_evolving(rd, pf, surf, P, fp.n_fast, fp.n_doppler, fp.window, "split",
                                    workspace=ws)

    frozen = rsim.Scatterers.from_arrays(sg.sea_surface(L, c["seed"]))

    def linear():
        rsim.simulate_fast(rd, pf, frozen, P, fp.n_fast, fp.n_doppler, fp.window, "split",
                           workspace=ws)

    t_evo = _timed(torch, evolving, 5, flush)
    # the same loop with buffers allocated once, captured into a CUDA graph
    em = rsim.EvolvingFastMode(rd, pf, surf, P, fp.n_fast, fp.n_doppler, fp.window, "split")
    T_e, Y_e = [t.clone() for t in em.run()]
    em.capture()
    t_graph = _timed(torch, em.replay, 5, flush)
    graph_same = bool(torch.equal(em.spectra, T_e) and torch.equal(em.iq, Y_e))
    t_lin = _timed(torch, linear, 5, flush)
    # the per-update summation alone: one launch over a block of 16 updates, each with its
    # own synthesised state
    K = min(16, S)
    sets = surf.field_sets(K)
    states = []
    for i in range(K):
        t = i * fp.n_fast / rd.prf_hz
        surf.at(t, fields=sets[i])
        states.append(sets[i] + (t,))
    grid = surf.grid()
    t_states = _timed(torch, lambda: rsim.doppler_accumulate_states(
        rd, pf, grid, 0, states, fp.n_fast, fp.n_doppler, "split", workspace=ws), 10, flush)
    del sets, states
    # algorithmic bytes of one synthesis: read A (8 L^2) + omega (8 L^2), write/read the packed
    # transforms (2 x 2 x 8 L^2), write 4 fields (16 L^2)
    nbytes = 8 * L * L + 8 * L * L + 32 * L * L + 16 * L * L
    line = _base_line("fast_2048x2048_p4096_evolving_surface",
                      "fast-mode IQ pulses/s with the surface regenerated per update", "IQ pulses/s",
                      round(P / (t_graph / 1e3), 1))
    line["config"].update({"grid": L, "pulses": P, "updates": S, "window": fp.window,
                           "precision": "split", "l2": "flushed before each timed call"})
    line["surface_synthesis_ms"] = round(t_surf, 4)
    import bench
    peak, basis = bench.measured_hbm_gbs()
    line["surface_synthesis_roofline"] = {"bound": "hbm", "bytes": nbytes,
                                          "achieved_gbs": round(nbytes / (t_surf / 1e3) / 1e9, 1),
                                          "peak_gbs": peak, "peak_basis": basis,
                                          "frac": round(nbytes / (t_surf / 1e3) / 1e9 / peak, 4),
                                          "basis": "one synthesis after an L2 flush"}
    line["surface_synthesis_in_loop"] = {
        "ms_per_synthesis": round(t_surf_loop, 4),
        "achieved_gbs": round(nbytes / (t_surf_loop / 1e3) / 1e9, 1),
        "frac": round(nbytes / (t_surf_loop / 1e3) / 1e9 / peak, 4),
        "basis": "64 consecutive syntheses alternating between two streams (workspaces and "
                 "field sets), as the update loop runs them"}
    line["states_summation"] = {"updates_per_launch": K, "ms_per_launch": round(t_states, 4),
                                "ms_per_update": round(t_states / K, 4),
                                "hbm_bytes_per_update": 16 * L * L,
                                "achieved_gbs_state_reads": round(16 * L * L * K / (t_states / 1e3) / 1e9, 1)}
    line["step_ms"] = {"evolving_surface_graph": round(t_graph, 3),
                       "evolving_surface_eager": round(t_evo, 3),
                       "linear_kinematics": round(t_lin, 3)}
    line["graph_bit_identical_to_eager"] = graph_same
    return line


RUNS = {"0": run_cfg0, "2": run_cfg2, "3": run_cfg3, "4": run_cfg4, "nfast": run_nfast_sweep,
        "antenna": run_antenna_table, "dda": run_delay_doppler, "surface": run_surface_update}


def run(k: str, args):
    import torch
    import paper_2408_11472_gb300 as rsim
    from bench import ClockSampler
    torch.cuda.set_device(0)
    del _TIMED_WINDOWS[:]
    clocks = ClockSampler(0)
    clocks.start()
    line = RUNS[str(k)](torch, rsim, args)
    # SM clock and throttle reasons over the timed regions only (not the oracle's CPU legs)
    line["clocks"] = clocks.stop(windows=list(_TIMED_WINDOWS))
    line["clocks"]["timed_regions"] = len(_TIMED_WINDOWS)
    return line


# ------------------------------------------------------------------ ncu capture targets
def profile_target(kind: str, reps: int = 4):
    """Small, repeatable workloads for one-kernel ncu captures (no JSON line, no timing
    contract): `reps` untimed calls, then one timed call whose CUDA-event time is printed.
      surface  syntheses of the 2048 x 2048 evolving surface at successive times
               (surf_rows_kernel, surf_cols_kernel);
      antenna  the 2048 x 2048 fast-mode pass with the 129 x 129 tabulated pattern
               (accumulate_split_kernel<DOPPLER, ANT>).
    Device memory: about 0.4 GB (surface) or 1 GB (antenna)."""
    import dataclasses
    import torch
    import paper_2408_11472_gb300 as rsim
    torch.cuda.set_device(0)
    c = sg.config(1)
    rd0, pf, fp, P, L = c["radar"], c["platform"], c["fast"], c["n_pulses"], c["L"]
    if kind == "surface":
        surf = rsim.EvolvingSurface(sg.sea_spectrum(L, c["seed"]))

        def call(r):
            surf.at(0.01 * r)
    elif kind == "antenna":
        rd = dataclasses.replace(rd0, antenna=sg.antenna_table(77))
        dev = rsim.Scatterers.from_arrays(sg.sea_surface(L, c["seed"]))
        S = (P - 1) // fp.n_fast + 2
        ws = torch.empty(rsim.workspace_size(S, rd.n_gates, fp.n_doppler), dtype=torch.uint8,
                         device="cuda")
        T = torch.zeros((S, rd.n_gates, fp.n_doppler), dtype=torch.complex64, device="cuda")

        def call(r):
            T.zero_()
            rsim.doppler_accumulate(rd, pf, dev, 0, S, fp.n_fast, fp.n_doppler, "split", out=T,
                                    workspace=ws)
    else:
        raise ValueError("unknown profile target %r" % kind)
    for r in range(reps):
        call(r)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    call(reps)
    e1.record()
    torch.cuda.synchronize()
    print("%s: %.4f ms per call" % (kind, e0.elapsed_time(e1)), flush=True)
