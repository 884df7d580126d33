"""Pins for the scenarios the oracle does not converge (test infrastructure).

The paper gives no stopping rule for an FDPF run that does not converge
(Sec. III.B; Sec. V reports convergence everywhere).  The oracle, like the
kernel, stops a warm-started run whose mismatch grows to 10x the smallest
value it reached and calls it DIVERGED.  These tests pin what that status
rests on, with a route independent of FDPF: a Newton-Raphson continuation
that takes the outaged branch's admittance from its base value to zero,
starting at the base case (so every point of the path is an exact AC
solution connected to the base state).

* On every outage of the benchmark grids that the oracle stops (the golden
  lists, written by make_n1_status.py from the oracle alone) the same FDPF
  without the growth rule does not converge either within 200 outer
  iterations: the rule shortens runs, it never cuts off a converging one.
* grid2k's outage: the continuation meets a fold before the branch is out
  (no AC solution continues the base state), and FDPF runs off to a
  mismatch above the absolute limit.
* grid10k's two outages: the continuation reaches the outage, at a state
  with a bus above 2 p.u. -- far outside the flat-voltage, small-angle
  region where B' and B'' stand in for the Jacobian, which is why FDPF
  (directly solved here, base-preconditioned CG on the GPU) does not get
  there from the base state.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve

from cases import GOLDEN
from gridgen import config_grid
from oracle import powerflow as pf
from oracle import screen


def golden_status(name):
    with open(os.path.join(GOLDEN, f"{name}_n1_status.json")) as fh:
        return json.load(fh)


def _ybus(g, scale_branch, scale):
    """Complex bus admittance with branch `scale_branch` scaled by `scale`
    (series admittance and charging), written out from the pi-model."""
    y = 1.0 / (g.r + 1j * g.x)
    bsh = g.b_sh.astype(complex)
    y[scale_branch] *= scale
    bsh[scale_branch] *= scale
    rows = np.r_[g.f, g.t, g.f, g.t]
    cols = np.r_[g.t, g.f, g.f, g.t]
    vals = np.r_[-y, -y, y + 0.5j * bsh, y + 0.5j * bsh]
    return sp.csr_matrix((vals, (rows, cols)), shape=(g.n_bus, g.n_bus))


def _newton(Y, P, Q, th, V, pvpq, pq, tol=1e-10, iters=25):
    """Newton-Raphson in polar coordinates on S = V conj(Y V):
    dS/dtheta = j diag(V) conj(diag(I) - Y diag(V)),
    dS/d|V|   = diag(V) conj(Y diag(V/|V|)) + conj(diag(I)) diag(V/|V|)."""
    th, V = th.copy(), V.copy()
    for _ in range(iters):
        Vc = V * np.exp(1j * th)
        I = Y @ Vc
        S = Vc * np.conj(I)
        F = np.r_[P[pvpq] - S.real[pvpq], Q[pq] - S.imag[pq]]
        if not np.isfinite(F).all():
            return th, V, False
        if np.abs(F).max() < tol:
            return th, V, True
        dV = sp.diags(Vc)
        dS_dth = 1j * dV @ np.conj(sp.diags(I) - Y @ dV)
        Vn = sp.diags(Vc / np.abs(Vc))
        dS_dVm = dV @ np.conj(Y @ Vn) + np.conj(sp.diags(I)) @ Vn
        J = sp.vstack([sp.hstack([dS_dth.real[pvpq][:, pvpq], dS_dVm.real[pvpq][:, pq]]),
                       sp.hstack([dS_dth.imag[pq][:, pvpq], dS_dVm.imag[pq][:, pq]])]).tocsc()
        dx = spsolve(J, F)
        th[pvpq] += dx[:pvpq.size]
        V[pq] += dx[pvpq.size:]
    return th, V, False


def outage_continuation(g, l, th0, V0):
    """Follow the AC solution from the base case while branch l's admittance
    goes from 1 to 0 times its value (adaptive steps).  Returns (mu reached,
    theta, V): mu = 1 when the outage itself is solved, else where the steps
    shrank below 1e-7 (a fold of the solution path)."""
    bt = g.bus_type
    pvpq = np.flatnonzero(bt != 2)
    pq = np.flatnonzero(bt == 0)
    th, V = th0.copy(), V0.copy()
    mu, h = 0.0, 0.05
    while mu < 1.0 and h >= 1e-7:
        m2 = min(1.0, mu + h)
        t2, v2, ok = _newton(_ybus(g, l, 1.0 - m2), g.P_sched, g.Q_sched, th, V, pvpq, pq)
        if ok:
            mu, th, V = m2, t2, v2
            h = min(0.05, 1.5 * h)
        else:
            h /= 2
    return mu, th, V


@pytest.mark.parametrize("name", ["grid2k", "grid10k"])
def test_stopped_runs_do_not_converge_without_the_growth_rule(name):
    d = golden_status(name)
    g = config_grid(name)
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-11, max_outer=200)
    assert st == pf.STATUS_OK
    assert d["not_converged"], "the golden list names the stopped runs"
    for l, status, outer in d["not_converged"]:
        assert status == pf.STATUS_DIVERGED
        on, _, isl, P, _ = screen.outage_setup(g, l)
        assert not isl.any()
        _, _, k, st2, err = pf.fdpf(g, on, ~isl, P, th0, V0, d["tol"], 200, growth_rule=False)
        assert st2 != pf.STATUS_OK and err > d["tol"], (l, st2, err)


def test_grid2k_stopped_run_has_no_solution_continuing_the_base_case():
    d = golden_status("grid2k")
    g = config_grid("grid2k")
    th0, V0, _, _, _ = pf.base_case(g, tol=1e-11, max_outer=200)
    for l, _, _ in d["not_converged"]:
        mu, _, _ = outage_continuation(g, l, th0, V0)
        assert mu < 1.0, l                       # a fold before the branch is out
        on, _, isl, P, _ = screen.outage_setup(g, l)
        _, _, _, st2, err = pf.fdpf(g, on, ~isl, P, th0, V0, d["tol"], 200, growth_rule=False)
        assert st2 == pf.STATUS_DIVERGED and err > pf.DIVERGE_LIMIT


def test_grid10k_stopped_runs_have_solutions_far_from_flat_voltages():
    d = golden_status("grid10k")
    g = config_grid("grid10k")
    th0, V0, _, _, _ = pf.base_case(g, tol=1e-11, max_outer=200)
    for l, _, _ in d["not_converged"]:
        mu, th, V = outage_continuation(g, l, th0, V0)
        assert mu == 1.0, l
        assert V.max() > 2.0, (l, V.max())
        # it is the post-outage solution: the oracle's FDPF stays there
        on, _, isl, P, _ = screen.outage_setup(g, l)
        _, _, k, st2, err = pf.fdpf(g, on, ~isl, P, th, V, 1e-9, 5)
        assert st2 == pf.STATUS_OK and k == 0, (l, st2, err)
