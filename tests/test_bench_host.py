"""bench.py's host-side parts, no GPU: the algorithmic-byte and FP64 work
models against hand counts, the clock-record summary, and the reference arm
(the oracle on the host cores), whose JSON line and rank handling follow
the same contract as the GPU arm's."""
import importlib.util
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_hand_count():
    """Two scenarios: (outer, inner P, inner Q) = (2, 3, 4) and (1, 2, 0) on a
    matrix pair with 9 and 6 rows (w = 4 bytes)."""
    b = _bench()
    info = dict(n_p=9, n_q=6, nnz_p=30, nnz_q=20, nnz_lp=25, nnz_lq=15)
    iters = np.array([[2, 3, 4], [1, 2, 0]], dtype=np.int32)
    n_bus, n_branch, w = 10, 14, 4
    # inner iterations: P 5 in all, Q 4 in all
    vec = 15 * w * (5 * 9 + 4 * 6)
    # mismatch passes: 2 outer + 1 per scenario -> 5 + 3
    mis = 32 * n_bus * (5 + 3)
    flows = 2 * (16 * n_bus + 8 * n_branch)
    mats = (5 * (30 + 2 * 25) + 4 * (20 + 2 * 15)) * (w + 4) / 2
    assert b.algorithmic_bytes(info, iters, w, n_bus, n_branch) == pytest.approx(
        vec + mis + flows + mats, rel=0, abs=1e-9)


def test_fp64_operations_hand_count():
    """A three-bus path slack - PV - PQ (two branches), one scenario of two
    outer iterations."""
    b = _bench()

    class G:
        bus_type = np.array([2, 1, 0])
        f = np.array([0, 1])
        t = np.array([1, 2])
        n_bus, n_branch = 3, 2

    # degrees 1, 2, 1; non-slack buses 1, 2 (adjacency 3), PQ bus 2 (adjacency 1)
    nP, nQ, AP, AQ = 2, 1, 3, 1
    per_outer = (4 * AP + 7 * nP + 2 * nQ) + (4 * AQ + 6 * nQ) + 12 * nP + 2 * nQ
    iters = np.array([[2, 1, 1]], dtype=np.int32)
    assert b.fp64_operations(G, iters) == 2 * per_outer + (nP + 16 * 2)


def test_clock_summary_reads_reasons():
    b = _bench()
    s = b.ClockSampler(0)
    s.rows = [["2070", "2070", "900.5", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["2055", "2070", "910.0", "0x0", "Not Active", "Not Active", "Not Active",
               "Not Active"],
              ["[N/A]"]]
    out = s.summary()
    assert out["sm_mhz"] == pytest.approx(2062.5)
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 3


def _run_reference(env_extra, tmp_path):
    env = dict(os.environ, **env_extra)
    env["OMP_NUM_THREADS"] = "1"
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--config", "grid120", "--steps", "2", "--warmup", "1", "--ref-sample", "8"]
    return subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True,
                          timeout=300)


def test_reference_arm_line(tmp_path):
    b = _bench()
    r = _run_reference({"RANK": "0", "WORLD_SIZE": "1"}, tmp_path)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == b.METRIC
    assert d["unit"] == "scenarios/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "scenarios/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("grid120")


def test_reference_arm_other_ranks_exit_quietly(tmp_path):
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, tmp_path)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_island_split_groups_bridge_outages():
    """Outage k is branch k: the bridges' rows and the others' are averaged
    apart (grid120's bridges from the host plan)."""
    b = _bench()
    from gridgen import config_grid
    from paper_1803_03290_gb300 import binding
    g = config_grid("grid120")
    br = binding.analyze(g)["bridge"].astype(bool)
    assert 0 < br.sum() < g.n_branch
    iters = np.zeros((g.n_branch, 3), dtype=np.int32)
    iters[br] = (3, 5, 7)
    iters[~br] = (2, 2, 1)
    out = b.island_split(g, iters)
    assert out["outages"] == int(br.sum())
    assert out["islanding"] == {"mean_outer": 3.0, "mean_inner_P": 5.0, "mean_inner_Q": 7.0}
    assert out["other"] == {"mean_outer": 2.0, "mean_inner_P": 2.0, "mean_inner_Q": 1.0}
