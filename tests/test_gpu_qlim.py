"""Reactive limits of the PV generators through the CUDA path against the
CPU oracle: converged scenarios whose generators left their limits turn
those buses PQ at the limit (B'' extension rows), held ones whose |V| passed
the set point turn back PV, and both go on to the same state; a scenario
that needs more rows at once than it holds reports QLIM_OVERFLOW."""
import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import grid, oracle_base, oracle_n1
from oracle import screen

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-6
KX = gp.MAX_EXT_ROWS  # extension rows a scenario holds


def expected_status(ref, cap):
    """The status the GPU must report for each scenario: the oracle's, except
    that a scenario in which the oracle held more than `cap` buses at their
    limits at once (whether it then converged or not) overflows the rows a
    scenario holds."""
    return np.where(ref["n_held"] > cap, gp.SCEN_QLIM_OVERFLOW, ref["status"])


def _check(res, ref, cap):
    """Every scenario's status and island labels against the oracle; the
    states of the scenarios both solve agree."""
    st = ref["status"]
    np.testing.assert_array_equal(res["status"], expected_status(ref, cap))
    np.testing.assert_array_equal(res["label"], ref["label"])
    fit = (st == 0) & (ref["n_held"] <= cap)
    assert fit.sum() > 0.8 * st.size
    assert (fit & (ref["n_switched"] > 0)).sum() >= 5   # the limits are exercised
    assert (fit & (ref["n_returned"] > 0)).sum() >= 1   # and the way back to PV
    for k, tol in (("theta", ANGLE_TOL), ("V", ANGLE_TOL), ("flow", 10 * ANGLE_TOL),
                   ("max_loading", 10 * ANGLE_TOL)):
        np.testing.assert_allclose(res[k][fit], ref[k][fit], rtol=0, atol=tol)
    assert (ref["n_held"] > cap).any()          # the overflow is exercised


@pytest.mark.parametrize("precision", [gp.BATCHED_FP32, gp.BATCHED_FP64])
def test_q_limits_grid120_all_outages(precision):
    g = grid("grid120_qlim")
    c = gp.GPCG(g, precision=precision, tol=1e-10, max_outer=100, inner_rtol=1e-6,
                max_inner=2000)
    c.base_solve()
    outages = np.arange(g.n_branch, dtype=np.int32)
    res = c.n1_screen(outages)
    ref = oracle_n1("grid120_qlim", outages, processes=1)
    _check(res, ref, KX)
    c.close()


def test_q_limits_generator_outages():
    """A tripped generator's bus holds one of the rows; switches add more."""
    g = grid("grid120_qlim")
    c = gp.GPCG(g, tol=1e-10, max_outer=100)
    c.base_solve()
    buses = np.flatnonzero(g.bus_type == 1).astype(np.int32)
    res = c.n1_gen_screen(buses)
    th0, V0 = oracle_base("grid120_qlim")
    ref = screen.n1_screen(g, th0, V0, buses, tol=1e-10, max_outer=100, processes=1,
                           kind="generator")
    sw, st = ref["n_switched"], ref["status"]
    # with limits this tight many trips leave the others short of reactive
    # power and the iteration fails, in the oracle too: every status is
    # compared, failures included (the tripped bus holds one of the rows)
    np.testing.assert_array_equal(res["status"], expected_status(ref, KX - 1))
    assert (st != 0).sum() >= 1
    fit = (st == 0) & (ref["n_held"] <= KX - 1)
    assert fit.sum() >= 8 and (fit & (sw > 0)).sum() >= 1
    for k in ("theta", "V"):
        np.testing.assert_allclose(res[k][fit], ref[k][fit], rtol=0, atol=ANGLE_TOL)
    c.close()


def test_q_limits_sample_grid2k_screening_tolerance():
    """At the screening tolerance every converged state is within 1e-4 p.u.
    of the power balance (the oracle's FP64 mismatch with the switched
    buses found again) and keeps the other generators within their limits."""
    from oracle import powerflow as pf
    g = grid("grid2k_qlim")
    c = gp.GPCG(g)
    c.base_solve()
    outages = np.sort(np.random.default_rng(9).choice(g.n_branch, 200, replace=False)).astype(np.int32)
    res = c.n1_screen(outages, outputs=("theta", "V", "status"))
    ok = np.flatnonzero(res["status"] == 0)
    assert ok.size > 0.9 * outages.size
    pv = g.bus_type == 1
    for s in ok[:60]:
        on, label, isl, P, _ = screen.outage_setup(g, int(outages[s]))
        live = on & ~isl[g.f] & ~isl[g.t]
        yb = pf.ybus_entries(g.n_bus, g.f, g.t, g.r, g.x, g.b_sh, live, g.tap)
        th, V = res["theta"][s], res["V"][s]
        dP, dQ = pf.mismatch(yb, P, g.Q_sched, th, V)
        main = ~isl
        assert np.abs(dP[main & (g.bus_type != 2)]).max() <= 1e-4 * (1 + 1e-9)
        qg = -dQ                               # generator output at each PV bus
        held = main & pv & (np.abs(V - g.V_set) > 1e-9)   # turned PQ: at a limit
        free = main & pv & ~held
        assert np.all(qg[free] <= g.Q_max[free] + 1e-4) and np.all(qg[free] >= g.Q_min[free] - 1e-4)
        at_lim = np.minimum(np.abs(qg[held] - g.Q_max[held]), np.abs(qg[held] - g.Q_min[held]))
        assert np.all(at_lim <= 1e-4 * (1 + 1e-9))
        pq = main & (g.bus_type == 0)
        assert np.abs(dQ[pq]).max() <= 1e-4 * (1 + 1e-9)
    c.close()


def test_base_case_outside_limits_is_refused():
    g = grid("grid120_qlim").copy()
    pv = np.flatnonzero(g.bus_type == 1)
    g.Q_max = g.Q_max.copy()
    g.Q_max[pv[0]] = g.Q_min[pv[0]] + 1e-3     # far below what the base case needs
    c = gp.GPCG(g)
    with pytest.raises(gp.GPCGError) as e:
        c.base_solve()
    assert "reactive limits" in str(e.value)
    c.close()
