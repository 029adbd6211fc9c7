"""Host logic of the benchmark (no GPU): workload labels and the structured-bank workload."""
import argparse
import importlib.util
import os

import numpy as np
import pytest

import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_workload_labels_name_the_truncation(bench):
    cfg = workload.config(2)
    assert bench.workload_label(cfg, 2, 3e-5) == \
        "cfg2: paper-shaped-fp32; n=2^20 fs=2048 f_low=20; 1 ref + 256 TaylorF2 nbrs; thr=3e-05 rel; W=2048"
    assert bench.workload_label(cfg, 2, 1e-3, "abs analytic real-kernel").endswith(
        "thr=0.001 abs analytic real-kernel; W=2048")


def test_structured_bank_workload(bench):
    """--bank N: the library's sets of a seeded bank become the batched workload's groups,
    every template exactly once (reference or neighbour), injections inside their groups."""
    from paper_2511_12894_gb300 import build
    build.build()
    args = argparse.Namespace(bank=3000, config=4, kernels=None)
    cfg = bench.load_workload(args)
    base = workload.config(4)
    assert cfg.index == 4 and cfg.n == base.n and cfg.fs == base.fs and cfg.name == "structured-bank-3000"
    bank = workload.synthetic_bank(3000, seed=2025)
    seen = sorted([(t.m1, t.m2) for r, nb in cfg.groups for t in (r,) + tuple(nb)])
    assert seen == sorted((t.m1, t.m2) for t in bank)
    assert len(cfg.injections) == 16
    for inj in cfg.injections:
        assert 0 <= inj.group < len(cfg.groups) and 0 <= inj.template_index < len(cfg.groups[inj.group][1])
        assert cfg.n // 64 <= inj.sample < cfg.n - cfg.n // 64
    # the default workloads are untouched
    assert bench.load_workload(argparse.Namespace(bank=0, config=2, kernels=None)) == workload.config(2)


def test_with_groups_skips_groups_without_dependents():
    base = workload.config(4, n_override=1 << 15, k_override=16)
    t = workload.Template(1.4, 1.3)
    groups = [(t, ()), base.groups[0], (t, ()), base.groups[1]]
    cfg = workload.with_groups(base, groups, "mixed")
    assert cfg.injections and all(inj.group in (1, 3) for inj in cfg.injections)
    assert workload.with_groups(base, [(t, ())], "empty").injections == ()


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the oracle on the host (no GPU) and prints one JSON line
    with the contract's keys; under torchrun only rank 0 prints, the other ranks exit 0 silently."""
    import json
    import subprocess
    import sys
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "1",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["metric"] == d["unit"] == "template*samples/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("cfg1")
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""
