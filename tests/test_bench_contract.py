"""bench.py's host logic on the CPU.  The reference arm (the FP64 oracle timed on
the host cores) prints one line with the keys of the bench contract, and under a
multi-rank launch only rank 0 does work; the uneven batch splits into (n, q, K)
classes that cover every frame and into memory waves within the budget."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({}, "--impl", "reference", "--steps", "1", "--warmup", "3", "--ref-frames", "2")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["unit"] == "frames/s" and line["higher_is_better"] is True and line["value"] > 0
    assert abs(line["ms_per_step"] - 1e3 * 2 / line["value"]) <= 1e-6 * line["ms_per_step"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"]
    assert 1 <= cb["cores"] <= 2                       # two frames keep at most two threads busy
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"] and line["config"]["frames_per_step"] == 2


def test_reference_arm_other_ranks_exit_without_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--impl", "reference", "--steps", "1", "--warmup", "3",
             "--gpus", "2")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_uneven_batch_waves_respect_the_memory_budget():
    """Classes of the uneven batch are grouped into waves whose HBM message state
    fits the budget; fused classes hold no HBM state; every class runs once."""
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(5)
    parts = [{"id": i, "state": int(rng.integers(1, 50)) * 1000, "F": int(rng.integers(1, 20)),
              "fused": bool(rng.random() < 0.3)} for i in range(40)]
    budget = 200_000
    waves = bench._waves(parts, budget)
    ids = sorted(p["id"] for w in waves for p in w)
    assert ids == list(range(40))
    for w in waves:
        need = sum(0 if p["fused"] else p["state"] * p["F"] for p in w)
        assert need <= budget or len(w) == 1 or sum(not p["fused"] for p in w) == 1
    assert len(bench._waves(parts, 10 ** 12)) == 1


def test_uneven_classes_cover_every_frame():
    sys.path.insert(0, ROOT)
    import bench
    classes, snr = bench._uneven_classes(2000, seed=9)
    frames = sorted(f for idx in classes.values() for f in idx)
    assert frames == list(range(2000)) and snr.shape == (2000,)
    for (n, q, K) in classes:
        assert n in (128, 256, 512, 1024, 2048) and q in (16, 64) and 2 <= K <= 8
    assert ((8.0 <= snr) & (snr <= 16.0)).all()


def test_serving_steady_rate_counts_the_saturated_window_only():
    """The serving workload's steady throughput: completions after the first poll
    sweep, up to 90 % of all requests, over that window; the drain after it and
    the completions folded into the first sweep do not count."""
    sys.path.insert(0, ROOT)
    import bench
    # 1,000 requests: 200 done by the first sweep at t = 1 s, then 4,000 frames/s
    # until 900 are done (t = 1.175 s), then a slow drain of the last 100 over 1 s
    done = [1.0 + (i + 1) / 4000.0 for i in range(700)] + [1.175 + (i + 1) / 100.0 for i in range(100)]
    rate, win = bench.steady_rate(done, 1.0, 1000)
    assert abs(rate - 4000.0) < 1e-6 and win == [1.0, 1.175]
    # the whole run counted as frames over wall time would be far lower
    assert 1000 / max(done) < 0.25 * rate
    # most requests already done at the first sweep (no queue): no steady figure
    assert bench.steady_rate(done[:300], 1.0, 1000) is None
    # too few completions in the window
    assert bench.steady_rate([1.0 + i / 10.0 for i in range(60)], 1.0, 100) is None


def test_profile_commands_run_committed_files_with_valid_flags():
    """Every command a profile summary quotes runs a committed file (bench.py)
    with flags the benchmark still accepts."""
    import re
    import shlex
    sys.path.insert(0, ROOT)
    import bench
    parser = bench.make_parser()
    prof = os.path.join(ROOT, "profiles")
    seen = 0
    for name in sorted(os.listdir(prof)):
        text = open(os.path.join(prof, name)).read().replace("\\\n", " ")
        for m in re.finditer(r"python (\S+)((?: --?[\w-]+(?: [^\s-][^\s]*)?)*)", text):
            assert m.group(1) == "bench.py", (name, m.group(0))
            parser.parse_args(shlex.split(m.group(2)))
            seen += 1
        assert "_work" not in text, name
    assert seen >= 5
