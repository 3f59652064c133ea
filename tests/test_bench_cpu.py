"""The benchmark's contract on a machine without a GPU: the reference arm (the FP64 oracle timed on
the host cores, a bounded sample of the 128^3 workload) prints one JSON line with the keys the
driver reads, and the synthetic inputs are reproducible."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line_with_the_contract_keys():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-steps-per-iter", "1"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_workloads_are_reproducible():
    from paper_2609_30039_gb300 import workloads as W
    for make in (lambda: W.cpml_blocks(n=24, d=4, n_steps=10, block=4, region=(6, 18)),
                 lambda: W.random_state_scene(shape=(9, 8, 7)),
                 lambda: W.lorentz_batch(n_domains=3, sizes=(20, 24), d=4, n_steps=10)[2]):
        a, b = make(), make()
        for x, y in zip(a.inv_eps3(), b.inv_eps3()):
            assert np.array_equal(x, y)
        assert a.poles == b.poles
        if a.pole_mask is not None:
            assert np.array_equal(a.pole_mask, b.pole_mask)
        for s, t in zip(a.sources, b.sources):
            assert s.lo == t.lo and s.hi == t.hi and np.array_equal(s.wave, t.wave)


def test_gpus_n_without_torchrun_starts_n_ranks():
    """`bench.py --gpus 2` run directly (no WORLD_SIZE in the environment) re-launches itself under
    torch.distributed.run with two processes; in dry-run mode they join a gloo group and rank 0
    reports n_gpus = 2 and the max over both ranks."""
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR",
                                                            "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--dry-run", "--steps", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["max_rank_seen"] == 1.0
