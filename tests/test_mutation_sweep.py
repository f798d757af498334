"""Strength of the oracle's pins: a mutation sweep (opt-in; ``pytest tests -m mutation
--mutation``, about 5 s per mutant on 8 cores).

Each mutant is a plausible slip -- a flipped sign, a dropped factor, a shifted index, a
transposed operand -- planted in a scratch copy of the repository.  Paired mutants put the
same slip into both restatements of the method (the C oracle and its numpy brute force),
so that the two still agree and only the pins against what the paper and the mathematics
fix can catch it; the others go into the single restatements (the oracle's cancellation-
free differences, delay-Doppler focusing, surface update, adjoint, pattern derivatives).
The CPU test suite runs against every mutant, and each must fail at least one test.
Skipped unless ``--mutation`` is given, so the default CPU suite stays fast.
"""
import os
import shutil
import subprocess
import sys

import pytest

pytestmark = pytest.mark.mutation

SRC = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C = "oracle/rsim_oracle.c"
NP = "oracle/bruteforce.py"

MUTANTS = {
    "phase sign": [(C, "double phi = -2.0 * OR_PI * (psi - rint(psi));", "double phi = 2.0 * OR_PI * (psi - rint(psi));"),
                   (NP, "C = amp * np.exp(-2j * np.pi * frac)", "C = amp * np.exp(2j * np.pi * frac)")],
    "range factor (r_ref/R) once": [(C, "* (rref / R) * (rref / R);", "* (rref / R);"),
                                    (NP, "(r_ref / rng) ** 2", "(r_ref / rng)")],
    "antenna exponent halved": [(C, "exp(-2.0 * OR_LN2 * theta * theta / (tb * tb))", "exp(-1.0 * OR_LN2 * theta * theta / (tb * tb))"),
                                (NP, "** 2 / 2.0)", "** 2 / 4.0)")],
    "gate offset -1": [(C, "return dR / rd->gate_width_m + 0.5 * (double)rd->n_gates;", "return dR / rd->gate_width_m + 0.5 * (double)rd->n_gates - 1.0;"),
                       (NP, "radar.n_gates / 2.0)", "radar.n_gates / 2.0 - 1.0)")],
    "doppler sign": [(C, "double nu = -2.0 * dR21 / lambda;", "double nu = 2.0 * dR21 / lambda;"),
                     (NP, "np.angle(C2 * np.conj(C1))", "np.angle(C1 * np.conj(C2))")],
    "bin rounding floor": [(C, "return nu * (double)n_doppler + 0.5;", "return nu * (double)n_doppler;"),
                           (NP, "freq * n_doppler + 0.5", "freq * n_doppler")],
    "Eq.1 without sqrt": [(C, "case 0: return sqrt(1.0 - d);", "case 0: return 1.0 - d;"),
                          (NP, "w = np.sqrt(1.0 - dd)", "w = (1.0 - dd)")],
    "raised cosine as amplitude": [(C, "case 1: return cos(0.5 * OR_PI * d);", "case 1: return 0.5 * (1.0 + cos(OR_PI * d));"),
                                   (NP, "w = np.sqrt(0.5 * (1.0 + np.cos(np.pi * dd)))", "w = 0.5 * (1.0 + np.cos(np.pi * dd))")],
    "forward instead of inverse transform": [(C, "dft_rows(T, n_rows, n_doppler, +1, s);", "dft_rows(T, n_rows, n_doppler, -1, s);"),
                                             (NP, "seg = np.fft.ifft(T, axis=-1) * K", "seg = np.fft.fft(T, axis=-1)")],
    "segment origin +1": [(C, "int64_t m = pmod64(x - p_i, K);", "int64_t m = pmod64(x - p_i + 1, K);"),
                          (NP, "m = np.mod(x - p_i, K)", "m = np.mod(x - p_i + 1, K)")],
    "pulse pair two PRIs apart": [(C, "double t_n = (double)(p_i + 1) / rd->prf_hz;", "double t_n = (double)(p_i + 2) / rd->prf_hz;"),
                                  (C, "double t2 = (double)(pulse + 1) / rd->prf_hz;", "double t2 = (double)(pulse + 2) / rd->prf_hz;"),
                                  (C, "double dt = 1.0 / rd->prf_hz;", "double dt = 2.0 / rd->prf_hz;"),
                                  (NP, "(p + 1) / radar.prf_hz", "(p + 2) / radar.prf_hz")],
    "sigma A without sqrt": [(C, "sqrt((double)sc->nrcs[n] * sc->area)", "((double)sc->nrcs[n] * sc->area)"),
                             (NP, "np.sqrt(f[\"nrcs\"] * area)", "(f[\"nrcs\"] * area)")],
    "C_{i+1} rasterised": [(C, "neu_add(&pp[cell * 4 + 0], &pp[cell * 4 + 1], ci.re);", "neu_add(&pp[cell * 4 + 0], &pp[cell * 4 + 1], cn.re);"),
                           (C, "neu_add(&pp[cell * 4 + 2], &pp[cell * 4 + 3], ci.im);", "neu_add(&pp[cell * 4 + 2], &pp[cell * 4 + 3], cn.im);"),
                           (NP, "np.add.at(T[u], (g[ok], k[ok]), C1[ok])", "np.add.at(T[u], (g[ok], k[ok]), C2[ok])")],
    "state epoch ignored": [(C, "double ts = t - sc->t0;", "double ts = t;"),
                            (NP, "ts = t - float(scene.get(\"t0\", 0.0))", "ts = t")],
    "platform frozen": [(C, "double px = pf->p0[0] + pf->v[0] * t;", "double px = pf->p0[0];"),
                        (NP, "np.asarray(platform.v, dtype=np.float64) * t", "np.asarray(platform.v, dtype=np.float64) * 0.0")],
    "scatterer velocity sign": [(C, "(double)sc->vx[n] * ts;", "(double)sc->vx[n] * -ts;"),
                                (C, "(double)sc->vy[n] * ts;", "(double)sc->vy[n] * -ts;"),
                                (C, "(double)sc->vz[n] * ts;", "(double)sc->vz[n] * -ts;"),
                                (NP, "pos = np.stack([o[0] + f[\"x\"] + f[\"vx\"] * ts, o[1] + f[\"y\"] + f[\"vy\"] * ts,", "pos = np.stack([o[0] + f[\"x\"] - f[\"vx\"] * ts, o[1] + f[\"y\"] - f[\"vy\"] * ts,"),
                                (NP, "o[2] + f[\"z\"] + f[\"vz\"] * ts])", "o[2] + f[\"z\"] - f[\"vz\"] * ts])")],
    "platform moving backwards": [(C, "double px = pf->p0[0] + pf->v[0] * t;", "double px = pf->p0[0] - pf->v[0] * t;"),
                                  (NP, "np.asarray(platform.v, dtype=np.float64) * t", "np.asarray(platform.v, dtype=np.float64) * -t")],
    "off-nadir angle against R": [(C, "double theta = atan2(rho, dz);", "double theta = atan2(rho, R);"),
                                  (NP, "off_nadir = np.arctan2(horiz, d[2])", "off_nadir = np.arctan2(horiz, rng)")],
    # single restatements: the oracle's cancellation-free differences, delay-Doppler
    # focusing, surface update, adjoint
    "range change without its |e|^2 term": [(C, "double dR21 = (ex * (2.0 * c1->dx + ex) + ey * (2.0 * c1->dy + ey) + ez * (2.0 * c1->dz + ez))",
                                             "double dR21 = (ex * (2.0 * c1->dx) + ey * (2.0 * c1->dy) + ez * (2.0 * c1->dz))")],
    "range change from the platform's motion only": [(C, "double ex = (pf->v[0] - (double)sc->vx[n]) * dt;", "double ex = pf->v[0] * dt;"),
                                                     (C, "double ez = (pf->v[2] - (double)sc->vz[n]) * dt;", "double ez = pf->v[2] * dt;")],
    "pattern phase change sign": [(C, "nu -= atan2(gi, gr) / (2.0 * OR_PI);", "nu += atan2(gi, gr) / (2.0 * OR_PI);")],
    "gate excess with the height added": [(C, "double dzr = (pz - rref) - sz;", "double dzr = (pz - rref) + sz;")],
    "DD centroid sign": [("oracle/delay_doppler.py", "return -2.0 * float(platform.v[2])", "return 2.0 * float(platform.v[2])")],
    "DD correction sign": [("oracle/delay_doppler.py", "corr = np.exp(-2j * np.pi * nu_c * k)", "corr = np.exp(2j * np.pi * nu_c * k)")],
    "DD beam transform sign": [("oracle/delay_doppler.py", "dft = np.exp(-2j * np.pi * np.outer(nu_f, k))", "dft = np.exp(2j * np.pi * np.outer(nu_f, k))")],
    "DD beams not centred": [("oracle/delay_doppler.py", "    nu_f = (np.arange(burst) - burst // 2) / burst\n    dft", "    nu_f = np.arange(burst) / burst\n    dft")],
    "DD migration ramp sign": [("oracle/delay_doppler.py", "ramp = np.exp(2j * np.pi * np.outer(s, qs) / G)", "ramp = np.exp(-2j * np.pi * np.outer(s, qs) / G)")],
    "DD migration factor 2": [("oracle/delay_doppler.py", "return x * x / (2.0 * r0 * radar.gate_width_m)", "return x * x / (r0 * radar.gate_width_m)")],
    "DD multi-look sum": [("oracle/delay_doppler.py", "W[b] = (np.abs(Y[b]) ** 2).mean(axis=0)", "W[b] = (np.abs(Y[b]) ** 2).sum(axis=0)")],
    "surface time sign": [("oracle/surface.py", "At = A * np.exp(-1j * omega * t)", "At = A * np.exp(1j * omega * t)")],
    "surface v_z sign": [("oracle/surface.py", "\"vz\": field(-1j * omega)", "\"vz\": field(1j * omega)")],
    "surface dispersion": [("oracle/surface.py", "omega = np.sqrt(g * kmag)", "omega = np.sqrt(g) * kmag")],
    "surface v_x along k_y": [("oracle/surface.py", "\"vx\": field(omega * ux)", "\"vx\": field(omega * uy)")],
    "adjoint phase derivative sign": [(C, "double dphi = 4.0 * OR_PI * e->dz / (lambda * e->R);", "double dphi = -4.0 * OR_PI * e->dz / (lambda * e->R);")],
    "adjoint range-factor term": [(C, "double dlna = -4.0 * OR_LN2 * e->theta / (tb * tb) * (e->rho / R2) + 2.0 * e->dz / R2;", "double dlna = -4.0 * OR_LN2 * e->theta / (tb * tb) * (e->rho / R2);")],
    "adjoint beam term sign": [(C, "double dlna = -4.0 * OR_LN2 * e->theta / (tb * tb) * (e->rho / R2) + 2.0 * e->dz / R2;", "double dlna = 4.0 * OR_LN2 * e->theta / (tb * tb) * (e->rho / R2) + 2.0 * e->dz / R2;")],
    "adjoint nrcs factor": [(C, "if (sig > 0.0) gsig += (gt[0] * ci.re + gt[1] * ci.im) / (2.0 * sig);", "if (sig > 0.0) gsig += (gt[0] * ci.re + gt[1] * ci.im) / sig;")],
    "adjoint conj convention": [(C, "gz += gt[0] * dre + gt[1] * dim;                 /* Re(conj(G) dC/dz) */", "gz += gt[0] * dre - gt[1] * dim;")],
    "synth adjoint transform sign": [(C, "dft_rows(s, n_rows, n_doppler, -1, T);", "dft_rows(s, n_rows, n_doppler, +1, T);")],
    # tabulated antenna pattern (paired where both restatements implement it)
    "table transposed": [(C, "const double *g10 = g00 + 2;                         /* u + du */", "const double *g10 = g00 + (size_t)rd->ant_nu * 2;"),
                         (C, "const double *g01 = g00 + (size_t)rd->ant_nu * 2;    /* v + dv */", "const double *g01 = g00 + 2;"),
                         (NP, "top = tab[r, c] + fx * (tab[r, c + 1] - tab[r, c])", "top = tab[r, c] + fx * (tab[r + 1, c] - tab[r, c])"),
                         (NP, "bottom = tab[r + 1, c] + fx * (tab[r + 1, c + 1] - tab[r + 1, c])", "bottom = tab[r, c + 1] + fx * (tab[r + 1, c + 1] - tab[r, c + 1])")],
    "direction cosines flipped": [(C, "e->u = -dx / R;", "e->u = dx / R;"),
                                  (C, "e->v = -dy / R;", "e->v = dy / R;"),
                                  (NP, "pattern(radar.antenna, -d[0] / rng, -d[1] / rng)", "pattern(radar.antenna, d[0] / rng, d[1] / rng)")],
    "pattern phase conjugated": [(C, "e->re = base * (g[0] * e->cr - g[1] * e->ci);", "e->re = base * (g[0] * e->cr + g[1] * e->ci);"),
                                 (C, "e->im = base * (g[0] * e->ci + g[1] * e->cr);", "e->im = base * (g[0] * e->ci - g[1] * e->cr);"),
                                 (NP, "amp = np.sqrt(f[\"nrcs\"] * area) * gain * (r_ref / rng) ** 2", "amp = np.sqrt(f[\"nrcs\"] * area) * np.conj(gain) * (r_ref / rng) ** 2")],
    "pattern u-derivative scale": [(C, "gu[c] = ((1.0 - tv) * (g10[c] - g00[c]) + tv * (g11[c] - g01[c])) / rd->ant_du;", "gu[c] = ((1.0 - tv) * (g10[c] - g00[c]) + tv * (g11[c] - g01[c]));")],
    "pattern term of the adjoint sign": [(C, "double du = e->u * e->dz / R2, dv = e->v * e->dz / R2;", "double du = -e->u * e->dz / R2, dv = -e->v * e->dz / R2;")],
}



# what a scratch copy needs: the package (with its built library), the oracle, the input
# generator, the tests and the scripts they run
_ENTRIES = ("paper_2408_11472_gb300", "include", "oracle", "scenegen", "tests", "bench.py",
            "bench_configs.py", "__graft_entry__.py")


def _copy_repo(dst):
    if os.path.exists(dst):
        shutil.rmtree(dst)
    os.makedirs(dst)
    skip = shutil.ignore_patterns("__pycache__", ".pytest_cache", "librsim_oracle.so")
    for e in _ENTRIES:
        src = os.path.join(SRC, e)
        if os.path.isdir(src):
            shutil.copytree(src, os.path.join(dst, e), ignore=skip)
        else:
            shutil.copy2(src, os.path.join(dst, e))


def _run_cpu_suite(dst):
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "not gpu", "-q", "-x",
                        "-p", "no:cacheprovider", "--ignore=tests/test_scenegen.py"],
                       cwd=dst, capture_output=True, text=True, timeout=900)
    tail = [ln for ln in r.stdout.splitlines()
            if ln.startswith("FAILED") or "passed" in ln or "failed" in ln]
    return r.returncode, tail[-2:] if tail else [r.stdout[-300:]]


def test_unmutated_copy_passes(tmp_path):
    dst = str(tmp_path / "repo")
    _copy_repo(dst)
    rc, tail = _run_cpu_suite(dst)
    assert rc == 0, tail


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    dst = str(tmp_path / "repo")
    _copy_repo(dst)
    for f, old, new in MUTANTS[name]:
        p = os.path.join(dst, f)
        s = open(p).read()
        assert old in s, "mutant %r: %s no longer contains %r" % (name, f, old)
        open(p, "w").write(s.replace(old, new))
    rc, tail = _run_cpu_suite(dst)
    assert rc != 0, "mutant %r survived the CPU suite: %s" % (name, tail)
