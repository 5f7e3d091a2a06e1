"""The benchmark's reference arm (the FP64 oracle on the host cores) runs on the CPU and
prints one JSON line with the keys the benchmark contract asks for, on the same metric
and workload as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--settle", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"].startswith("snake env-steps/s")
    assert d["config"]["snakes_per_gpu"] == 16384 and d["config"]["nodes_per_gpu"] > 16384 * 20
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    # the GPU arm builds its config with the same function on the same batch: equal dicts,
    # the reference arm's sample stated under its own key
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    assert d["config"] == bench.workload_config(int(W.n_nodes(bench.eval_batch(1)).sum()), 1, 2)
    assert d["config"]["settle_steps"] == 2
    assert "sample" not in d["config"] and "snakes" in d["reference_sample"]


def test_cpu_baseline_reports_all_cores_and_one_core():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    w = W.learned(n=64, seed=4)
    r = bench.cpu_baseline(w, W.solver_settings(iters=bench.CAP, tol=bench.TOL), n_sample=4, budget_s=1.0,
                           settle=2)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1
    assert r["single_thread"]["cores"] == 1 and r["single_thread"]["value"] > 0
