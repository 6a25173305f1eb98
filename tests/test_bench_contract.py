"""The bench's reference arm on the host (no GPU): the oracle timed on a
bounded sample of the headline workload, printed as one JSON line with the
keys of the GPU arm; ranks other than 0 print nothing and exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _bench(["--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "elems/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2
    assert d["warmup"] == 3                            # fewer than 3 warm-up steps are raised to 3
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["ms_per_step"] > 0
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # value counts gathered + scattered tiler elements of the sampled frames
    frames = d["config"]["sample_frames"]
    units = frames * (1080 * 240 * 8 + 1080 * 720 + 135 * 720 * 8 + 405 * 720)
    assert abs(d["value"] * d["ms_per_step"] * 1e-3 - units) <= 1e-6 * units


def test_reference_arm_other_ranks_are_silent():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "3"], {"RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
