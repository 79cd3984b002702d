"""bench.py's reference arm on the CPU: one JSON line with the keys the measurement contract names
(the oracle timed on the host cores on a bounded sample), and silence with exit status 0 on ranks
other than 0 of a multi-process launch; the sharding of the ragged batch's geometries over ranks."""
import json
import os
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d), KEYS - set(d)
    assert d["impl"] == "reference" and d["unit"] == "walker-evals/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_is_silent_on_other_ranks():
    r = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_ragged_geometries_are_sharded_once_and_balanced():
    """Longest-processing-time-first sharding of the 64 ragged geometries by N_e^3 W: every
    geometry on exactly one rank, and no rank above the mean load by more than the largest item
    (the greedy bound)."""
    sys.path.insert(0, str(ROOT))
    import bench
    from paper_2511_05222_gb300 import systems as S

    plan = S.ragged_batch_plan()
    cost = [sum(Z) ** 3 * W for Z, W in plan]
    for ws in (1, 2, 3, 4, 8):
        own = bench.shard_geometries(plan, ws)
        flat = sorted(g for o in own for g in o)
        assert flat == list(range(len(plan)))
        loads = [sum(cost[g] for g in o) for o in own]
        assert max(loads) <= sum(cost) / ws + max(cost)
