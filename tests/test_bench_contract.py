"""bench.py's reference arm -- the oracle timed on the host cores -- run on
the CPU: its one JSON line carries the keys of the benchmark line, the same
metric and unit as the GPU arm, a cpu_baseline describing the run and an e2e
object without host-device bytes; fewer than 3 warm-up steps are refused."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          cwd=ROOT, timeout=900)


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_contract_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    bench = _bench_module()
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_fewer_than_three_warmup_steps_are_refused():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "2")
    assert r.returncode != 0
    assert "warmup" in r.stderr


def test_every_linearized_launch_has_a_roofline_model():
    """Every kernel launch of an L[g] application (lin_generic.cuh, and the
    fixes) is rated by bench.py's roofline model: a bandwidth-bound kernel
    with its compulsory bytes, or an arithmetic one with non-zero
    algorithmic flops.  A launch the model does not know would be reported
    with a fraction of 0."""
    import re
    bench = _bench_module()
    src = "".join(open(os.path.join(ROOT, "paper_2503_09580_gb300", "csrc", f)).read()
                  for f in ("lin_generic.cuh", "fixes.cu"))
    names = set(re.findall(r'LBO_LAUNCH\(p, "([a-z0-9_]+)"', src))
    names |= set(re.findall(r'launch_uhat\([^)]*"([a-z0-9_]+)"\)', src))
    names = {n for n in names if not n.startswith("cache_")}  # the Maxwellian cache: outside the timed application
    assert {"plane_inv_mh_fwd", "axis1_uhat_octant_inv", "uhat_octant", "mh_table", "conservation_fix"} <= names
    for n in sorted(names):
        if n in bench.HBM_KERNELS:
            assert bench.kernel_bytes_per_instance(n, 32, 8) > 0, n
        else:
            assert bench.kernel_flops_per_instance(n, 32) > 0, n
