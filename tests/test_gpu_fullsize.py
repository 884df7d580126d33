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
    """The 500-scenario seeded sample of grid50k, FP32 factors and scaled FP16
    factors, against the oracle's angles at a 1e-10 p.u. mismatch."""
    g = grid("grid50k")
    samp = np.sort(np.random.default_rng(500).choice(g.n_branch, 500, replace=False)).astype(np.int32)
    ref = oracle_n1("grid50k", samp, tol=1e-10)
    ok = ref["status"] == 0
    errs = {}
    for prec in (gp.BATCHED_FP32, gp.BATCHED_FP32_F16):
        c = gp.GPCG(g, precision=prec, tol=1e-10, max_outer=100)
        c.base_solve()
        res = c.n1_screen(samp, outputs=("theta", "V", "status"))
        c.close()
        np.testing.assert_array_equal(res["status"], ref["status"])
        errs[prec] = max(np.abs(res["theta"][ok] - ref["theta"][ok]).max(),
                         np.abs(res["V"][ok] - ref["V"][ok]).max())
    print(f"grid50k 500-sample max error vs oracle: FP32 factors {errs[gp.BATCHED_FP32]:.2e}, "
          f"FP16 factors {errs[gp.BATCHED_FP32_F16]:.2e}")
    assert max(errs.values()) <= 1e-6, errs
