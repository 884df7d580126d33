"""Parity at the benchmark sizes, in the benchmark's launch configuration:
every outage of the 10,000-bus grid screened as bench.py screens it, with
sampled outputs checked against the oracle; and the 50,000-bus grid's angle
error on a seeded 500-scenario sample."""
import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import grid, oracle_base, oracle_n1, sample_outages
from oracle import screen

pytestmark = pytest.mark.gpu


def test_grid10k_all_outages_bench_configuration():
    g = grid("grid10k")
    c = gp.GPCG(g)                      # the benchmark's options (tol 1e-4, FP32 inner)
    c.base_solve()
    outages = np.arange(g.n_branch, dtype=np.int32)
    res = c.n1_screen(outages, outputs=("theta", "V", "status", "iters", "max_loading"))
    st = res["status"]
    assert (st == 0).sum() >= 0.99 * g.n_branch
    rng = np.random.default_rng(10)
    samp = np.unique(np.r_[rng.choice(g.n_branch, 48, replace=False),
                           sample_outages(g, 16, seed=10)])
    ref = oracle_n1("grid10k", outages[samp], tol=1e-4)
    # statuses agree; converged states meet the tolerance in the oracle's FP64 mismatch
    np.testing.assert_array_equal(st[samp], ref["status"])
    for k, s in enumerate(samp):
        if st[s] == 0:
            e = screen.scenario_mismatch(g, int(outages[s]), res["theta"][s], res["V"][s])
            assert e <= 1e-4 * (1 + 1e-9), (s, e)
    # island labels of the sample are exact
    lab = c.n1_screen(outages[samp], outputs=("label",))["label"]
    np.testing.assert_array_equal(lab, ref["label"])


def test_grid10k_refined_sample_angles():
    g = grid("grid10k")
    c = gp.GPCG(g, tol=1e-10, max_outer=100)
    c.base_solve()
    samp = sample_outages(g, 40, seed=11)
    res = c.n1_screen(samp, outputs=("theta", "V", "status", "flow"))
    ref = oracle_n1("grid10k", samp, tol=1e-10)
    np.testing.assert_array_equal(res["status"], ref["status"])
    ok = ref["status"] == 0
    assert np.abs(res["theta"][ok] - ref["theta"][ok]).max() <= 1e-6
    assert np.abs(res["V"][ok] - ref["V"][ok]).max() <= 1e-6


@pytest.mark.slow
def test_grid50k_angle_error_on_500_sample():
    g = grid("grid50k")
    c = gp.GPCG(g, tol=1e-10, max_outer=100)
    c.base_solve()
    samp = np.sort(np.random.default_rng(500).choice(g.n_branch, 500, replace=False)).astype(np.int32)
    res = c.n1_screen(samp, outputs=("theta", "V", "status"))
    ref = oracle_n1("grid50k", samp, tol=1e-10)
    np.testing.assert_array_equal(res["status"], ref["status"])
    ok = ref["status"] == 0
    err = np.abs(res["theta"][ok] - ref["theta"][ok]).max()
    assert err <= 1e-6, err
