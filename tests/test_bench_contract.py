"""The benchmark's JSON-line contract, checked on the host through its reference arm (the
FP64 oracle timed on the host cores) on a reduced scene: the keys and units of the line,
the reference arm's own cpu_baseline and e2e objects, and that only rank 0 prints under a
multi-process launch."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--L", "128",
                           "--steps", "2", "--warmup", "3", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _bench()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "IQ pulses/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["vs_baseline"] is None
    assert d["dtype"] == "f64" and "synthetic" in d["data"]
    # the step is one fast-mode pass: 4096 pulses from 65 spectra of 128 gates x 64 bins
    cfg = d["config"]
    assert cfg["workload"] == "fast_128x128_p4096"
    assert (cfg["scatterers"], cfg["pulses"], cfg["spectra"], cfg["gates"], cfg["doppler_bins"]) == \
        (128 * 128, 4096, 65, 128, 64)
    assert d["ms_per_step"] == pytest.approx(1e3 * cfg["pulses"] / d["value"], rel=1e-3)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["unit"] == d["unit"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _bench({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
