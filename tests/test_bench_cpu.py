"""bench.py on the CPU: the reference arm's JSON line (the oracle's fast route on
the host cores) carries every key of the benchmark contract, and the roofline
helpers compute what their cost model states (the survey's 1.9 kflop per pair +
13 kflop per atom at K = 6, N_a = 35, C_a = 209; the HBM sub-entries' bytes per
atom)."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["unit"] == "atom-steps/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "bcc_ta_8192_K6_P4_4body"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_survey_flop_model():
    b = _bench()
    p = synth.params_full()
    assert b.algorithmic_flops_per_atom(p, 25.74) == pytest.approx(1900.0 * 25.74 + 13000.0, rel=1e-12)
    assert b.algorithmic_flops_per_atom(p, 0.0) == pytest.approx(13000.0, rel=1e-12)
    # the kernel's own count merges duplicate Eq. 30a triples: lower than the survey's
    assert b.kernel_flops_per_atom(p, 25.74) < b.algorithmic_flops_per_atom(p, 25.74)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_hbm_subentries(precision):
    b = _bench()
    N, pairs = 8192, 25.0
    out = b.hbm_subentries(N, pairs, [0.01, 0.03, 0.005], precision)
    nb, fin = out["neighbor"], out["finalize"]
    assert nb["bytes_per_atom"] == 24.0 + 4.0 * pairs + 4.0
    assert fin["bytes_per_atom"] == (56.0 if precision == "mixed" else pairs * 36.0 + 24.0)
    for e, ms in ((nb, 0.01), (fin, 0.005)):
        assert e["bound"] == "hbm" and e["unit"] == "GB/s" and e["phase_ms"] == ms
        assert e["achieved"] == pytest.approx(e["bytes_per_atom"] * N / (ms / 1e3) / 1e9, rel=1e-12)
        assert e["frac"] == pytest.approx(e["achieved"] / e["peak"], rel=1e-12)
