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
