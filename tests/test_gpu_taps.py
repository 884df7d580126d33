"""Transformer turns ratios (Sec. II.B edge attribute) through the CUDA path,
against the CPU oracle on grids where 10-15 % of the branches are
transformers: the matrices as built, the SpMV with a transformer's outage
stamp, the base case and the N-1 screen (transformer outages included)."""
import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import grid, oracle_base, oracle_n1, sample_outages
from oracle import powerflow as pf, screen

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-6


def _dense(d):
    n = d["bus_of_row"].size
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(d["rowptr"][i], d["rowptr"][i + 1]):
            A[i, d["col"][k]] = d["val"][k]
    return A


def _oracle_matrix(g, which, on):
    keep = np.flatnonzero(g.bus_type != 2) if which == 0 else np.flatnonzero(g.bus_type == 0)
    A = (pf.bprime(g.n_bus, g.f, g.t, g.x, on, keep) if which == 0
         else pf.bdprime(g.n_bus, g.f, g.t, g.r, g.x, on, keep, g.tap)).toarray()
    return A, keep


@pytest.mark.parametrize("which", [0, 1])
def test_tapped_matrices(which):
    g = grid("grid120_xfmr")
    c = gp.GPCG(g)
    d = c.export_matrix(which)
    A, keep = _oracle_matrix(g, which, np.ones(g.n_branch, bool))
    pos = {b: k for k, b in enumerate(keep)}
    perm = np.array([pos[b] for b in d["bus_of_row"]])
    np.testing.assert_allclose(_dense(d), A[np.ix_(perm, perm)], rtol=0,
                               atol=1e-12 * np.abs(A).max())
    if which == 1:  # the turns ratios are in B'' and nowhere else
        A1, _ = _oracle_matrix(g.copy(), 1, np.ones(g.n_branch, bool))
        g0 = g.copy()
        g0.tap = None
        A0, _ = _oracle_matrix(g0, 1, np.ones(g.n_branch, bool))
        assert np.abs(A1 - A0).max() > 1e-3
    c.close()


@pytest.mark.parametrize("precision", [gp.BATCHED_FP64, gp.BATCHED_FP32])
def test_tapped_outage_stamp(precision):
    """B''_s x for every outage (transformers and lines), 8 FP32 ulps of the
    row scale for FP32 and FP64 rounding for FP64."""
    g = grid("grid120_xfmr")
    c = gp.GPCG(g)
    d = c.export_matrix(1)
    keep = np.flatnonzero(g.bus_type == 0)
    pos = {b: k for k, b in enumerate(keep)}
    perm = np.array([pos[b] for b in d["bus_of_row"]])
    outages = np.r_[np.arange(g.n_branch), -1].astype(np.int32)
    X = np.random.default_rng(7).standard_normal((outages.size, perm.size))
    Y = c.apply(1, 0, outages, X, precision)
    for s, l in enumerate(outages):
        on = np.ones(g.n_branch, bool)
        if l >= 0:
            on[l] = False
        A, _ = _oracle_matrix(g, 1, on)
        ref = A[np.ix_(perm, perm)] @ X[s]
        scale = np.abs(A).max() * np.abs(X[s]).max() * 8
        tol = 1e-13 * scale if precision == gp.BATCHED_FP64 else 2e-6 * scale
        np.testing.assert_allclose(Y[s], ref, rtol=0, atol=tol)
    c.close()


@pytest.mark.parametrize("name", ["grid120_xfmr", "grid2k_xfmr"])
def test_tapped_base_solve(name):
    c = gp.GPCG(grid(name))
    b = c.base_solve()
    th, V = oracle_base(name)
    np.testing.assert_allclose(b["theta"], th, atol=1e-8)
    np.testing.assert_allclose(b["V"], V, atol=1e-8)
    c.close()


def _compare(res, ref, n_out):
    np.testing.assert_array_equal(res["label"], ref["label"])
    np.testing.assert_array_equal(res["status"], ref["status"])
    ok = np.isin(ref["status"], [0, 3])
    assert ok.sum() > 0.9 * n_out
    for k, tol in (("theta", ANGLE_TOL), ("V", ANGLE_TOL), ("flow", 10 * ANGLE_TOL),
                   ("max_loading", 10 * ANGLE_TOL)):
        np.testing.assert_allclose(res[k][ok], ref[k][ok], rtol=0, atol=tol)


@pytest.mark.parametrize("precision,precond", [
    (gp.BATCHED_FP32, gp.PRECOND_EXACT), (gp.BATCHED_FP64, gp.PRECOND_EXACT),
    (gp.BATCHED_FP32, gp.PRECOND_IC0), (gp.BATCHED_FP64, gp.PRECOND_JACOBI),
    (gp.BATCHED_FP32_F16, gp.PRECOND_EXACT), (gp.PLAIN_FP64, gp.PRECOND_EXACT)])
def test_tapped_n1_grid120_all_outages(precision, precond):
    g = grid("grid120_xfmr")
    c = gp.GPCG(g, precision=precision, precond=precond, tol=1e-10, max_outer=100,
                inner_rtol=1e-6, max_inner=2000)
    c.base_solve()
    outages = np.arange(g.n_branch, dtype=np.int32)
    res = c.n1_screen(outages)
    ref = oracle_n1("grid120_xfmr", outages, processes=1)
    _compare(res, ref, outages.size)
    c.close()


def test_tapped_n1_grid2k_sample():
    """Refined to 1e-10 p.u. against the oracle on a sample with islanding and
    transformer outages; and at the 1e-4 screening tolerance every converged
    state's FP64 mismatch, evaluated by the oracle, is within it."""
    g = grid("grid2k_xfmr")
    xf = np.flatnonzero(g.tap != 1.0)
    outages = np.union1d(sample_outages(g, 64, seed=5), xf[:32]).astype(np.int32)
    c = gp.GPCG(g, tol=1e-10, max_outer=100)
    c.base_solve()
    res = c.n1_screen(outages)
    ref = oracle_n1("grid2k_xfmr", outages)
    _compare(res, ref, outages.size)
    c.close()
    c = gp.GPCG(g)
    c.base_solve()
    res = c.n1_screen(outages, outputs=("theta", "V", "status", "iters"))
    for s in np.flatnonzero(res["status"] == 0):
        e = screen.scenario_mismatch(g, int(outages[s]), res["theta"][s], res["V"][s])
        assert e <= 1e-4 * (1 + 1e-9)
    c.close()
