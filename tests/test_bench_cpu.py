"""CPU: the benchmark's reference arm (the FP64 oracle on the host cores, warm-up and timed
steps of one block each) prints the one JSON line of the benchmark contract; under a
multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--cpu-sample-walkers", "8", "--ref-seconds", "5", "--steps", "2", "--warmup", "3"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    return [ln for ln in out.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_the_contract_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "walker-moves/s" and d["unit"] == "walker-moves/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 3
    assert d["n_gpus"] == 1 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert "paper_scale_double_lorentz" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "of the 4096 walkers, 3 untimed + 2 timed blocks" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "walker-moves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the step time is that of the blocks actually run; the scaling to all walkers is separate
    assert d["ms_per_step"] > 0
    assert d["ms_per_step_scaled"]["value"] > d["ms_per_step"]


def test_reference_arm_prints_nothing_on_other_ranks():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []
