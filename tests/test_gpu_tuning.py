"""The autotuner's knobs -- tile width (scenarios a CTA solves together),
tiles per SM (scenarios in flight) and the dense tail of the substitutions'
level schedule -- against the oracle: every choice must give the oracle's
statuses and labels exactly and its states within the parity tolerance,
and the autotuner's choice must be reported and cached."""
import functools

import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import grid, oracle_n1, sample_outages
from oracle import adjoint

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-6


@functools.lru_cache(maxsize=None)
def _sample(name, k, seed):
    g = grid(name)
    A = sample_outages(g, k, seed=seed)
    return A, oracle_n1(name, A)


def _check(res, ref):
    np.testing.assert_array_equal(res["status"], ref["status"])
    np.testing.assert_array_equal(res["label"], ref["label"])
    ok = np.isin(ref["status"], [0, 3])
    assert ok.sum() >= 0.9 * ok.size
    for k, tol in (("theta", ANGLE_TOL), ("V", ANGLE_TOL), ("flow", 10 * ANGLE_TOL)):
        np.testing.assert_allclose(res[k][ok], ref[k][ok], rtol=0, atol=tol)


@pytest.mark.parametrize("tail", [-1, 64, 128, gp.MAX_TAIL_ROWS])
@pytest.mark.parametrize("tile,per_sm", [(2, 1), (2, 3), (8, 2)])
def test_every_knob_choice_matches_oracle(tail, tile, per_sm):
    """Each tail cap, tile width and tiles-per-SM count: the grid2k sample
    (islanding outages included) at a 1e-10 p.u. mismatch."""
    g = grid("grid2k")
    A, ref = _sample("grid2k", 64, 21)
    c = gp.GPCG(g, tol=1e-10, max_outer=100, tile=tile, ctas_per_sm=per_sm, tail_rows=tail)
    info = c.info()
    if tail < 0:
        assert info["tail_rows_p"] == 0 and info["tail_rows_q"] == 0
    else:
        assert 0 < info["tail_rows_p"] <= tail and 0 < info["tail_rows_q"] <= tail
    c.base_solve()
    res = c.n1_screen(A)
    info = c.info()
    assert info["tile"] == tile and info["ctas_per_sm"] == per_sm and info["tuned"] == 0
    _check(res, ref)
    c.close()


def test_tail_change_keeps_results_and_adjoint():
    """Rebuilding the tails through gpcg_set_options: the screen and the
    adjoint (whose copy of B' shares the tail's schedule) stay right."""
    g = grid("grid2k")
    A, ref = _sample("grid2k", 64, 21)
    c = gp.GPCG(g, tol=1e-10, max_outer=100, tile=2)
    c.base_solve()
    P, b = g.P_sched * 2.0, 1.0 / g.x
    L0, gP0, gb0 = c.n1_adjoint(A, P, b)
    for tail in (64, -1, gp.MAX_TAIL_ROWS):
        c.set_options(tol=1e-10, max_outer=100, tile=2, tail_rows=tail)
        rows = c.info()["tail_rows_p"]
        assert (rows == 0) if tail < 0 else (0 < rows <= tail)
        _check(c.n1_screen(A), ref)
        L, gP, gb = c.n1_adjoint(A, P, b)
        assert abs(L - L0) <= 1e-12 * abs(L0)
        np.testing.assert_allclose(gP, gP0, rtol=1e-9, atol=1e-12 * np.abs(gP0).max())
        np.testing.assert_allclose(gb, gb0, rtol=1e-9, atol=1e-12 * np.abs(gb0).max())
    Lo, _, _ = adjoint.loss_and_grad(g, A, P, b)
    assert abs(L0 - Lo) <= 1e-10 * abs(Lo)
    c.close()


def test_autotuner_choice_reported_and_cached():
    """A context with every knob left to the autotuner reports its choice;
    a second context on the same grid and scenario count takes it from the
    cache without probing, with the same results; a call whose scenario
    count is another power of two is tuned for it."""
    g = grid("grid2k")
    A, ref = _sample("grid2k", 64, 21)
    c1 = gp.GPCG(g, tol=1e-10, max_outer=100)
    c1.base_solve()
    r1 = c1.n1_screen(A)
    i1 = c1.info()
    assert i1["tuned"] in (1, 2)
    assert i1["tile"] in (2, 4, 8) and i1["ctas_per_sm"] >= 1
    assert i1["tail_rows_p"] in (0,) or 0 < i1["tail_rows_p"] <= gp.MAX_TAIL_ROWS
    _check(r1, ref)
    c2 = gp.GPCG(g, tol=1e-10, max_outer=100)
    c2.base_solve()
    r2 = c2.n1_screen(A)
    i2 = c2.info()
    assert i2["tuned"] == 2
    for k in ("tile", "ctas_per_sm", "tail_rows_p", "tail_rows_q"):
        assert i2[k] == i1[k]
    np.testing.assert_array_equal(r2["status"], r1["status"])
    ok = r1["status"] == 0
    np.testing.assert_allclose(r2["theta"][ok], r1["theta"][ok], rtol=0, atol=1e-12)
    # 8 outages: another power of two, tuned (or cached) for it
    r3 = c2.n1_screen(A[:8])
    assert c2.info()["tuned"] in (1, 2)
    np.testing.assert_array_equal(r3["status"], ref["status"][:8])
    c1.close()
    c2.close()


def test_autotuner_keeps_fixed_knobs():
    """Knobs fixed by the options are not tuned."""
    g = grid("grid2k")
    A, ref = _sample("grid2k", 64, 21)
    c = gp.GPCG(g, tol=1e-10, max_outer=100, tile=4, tail_rows=64)
    c.base_solve()
    _check(c.n1_screen(A), ref)
    info = c.info()
    assert info["tile"] == 4 and 0 < info["tail_rows_p"] <= 64
    assert info["tuned"] in (1, 2) and info["ctas_per_sm"] >= 1
    c.close()
