"""The benchmark's reference arm on the CPU: one JSON line with the keys the
benchmark contract names, and silence on ranks other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    env["SCCSD_ORACLE_SAMPLE"] = "small"   # the o=21 v=200 sample needs ~60 GB and minutes
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0"],
                          capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "o21_v200_J663"


def test_reference_arm_is_silent_on_other_ranks():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_ladder_flop_counts():
    """Executed (dense) and minimal (+/- packed) ladder flops per trial vector:
    at o=21 v=200 about 1.41e12 and 3.53e11; the packed count is the number of
    unique-pair multiply-adds of the symmetric and antisymmetric parts."""
    sys.path.insert(0, ROOT)
    import bench
    assert abs(bench.ladder_flops_dense(21, 200) / 1.4112e12 - 1.0) < 1e-3
    assert abs(bench.ladder_flops_packed(21, 200) / 3.53e11 - 1.0) < 2e-3
    o, v = 3, 4
    plus = sum(1 for i in range(o) for j in range(i, o) for a in range(v) for b in range(a, v)
               for c in range(v) for d in range(c, v))
    minus = sum(1 for i in range(o) for j in range(i + 1, o) for a in range(v)
                for b in range(a + 1, v) for c in range(v) for d in range(c + 1, v))
    assert bench.ladder_flops_packed(o, v) == 2.0 * (plus + minus)
    assert bench.ladder_flops_dense(o, v) == 2.0 * o * o * v ** 4


def test_ladder_call_flop_counts():
    """One 6-vector ladder call at o=21 v=200 J=663: the scope table's
    algorithmic count (symmetric build 1.06e12 plus 6 packed contractions of
    3.53e11) and the executed count of the kernels' padded tiles, which is
    larger but within 1.5x."""
    sys.path.insert(0, ROOT)
    import bench
    alg = bench.ladder_flops_algorithmic(21, 200, 663, 6)
    assert abs(alg / (1.0607e12 + 6 * 3.5298e11) - 1.0) < 2e-3
    exe = bench.ladder_flops_executed(21, 200, 663, 6, "bf16")
    assert alg < exe < 1.5 * alg
    assert bench.ladder_flops_executed(21, 200, 663, 6, "bf16x3") == 3 * exe
