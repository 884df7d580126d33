"""Adjoint of a smooth overload penalty over all N-1 scenarios (DC model).

Test infrastructure (see the package docstring).

The paper's quick screen focuses on the P-theta equation (4) (Sec. IV.A);
the DC model below is that equation with |V| = 1: for scenario s (outage l),
with the islands removed and the islands' injection re-dispatched over the
main island's generators (Sec. IV.C, weights frozen),

    theta_s = B'_s^{-1} R_s P,        f_s = diag(b_s) A theta_s,
    L = sum_s sum_k softplus(|f_ks| / rating_k - 1)^2,

where b_k = 1/x_k is the branch susceptance (zero for the outaged branch and
for branches that touch an island), A the branch-bus incidence on the
main island's non-slack buses, B'_s = A^T diag(b_s) A, and R_s the linear
re-dispatch map.  With g_s = dL/df_s and lambda_s = B'_s^{-1} A^T diag(b_s) g_s
(one more solve with the symmetric B'_s):

    dL/dP   = sum_s R_s^T lambda_s
    dL/db_k = sum_s [ g_ks (A theta_s)_k - (A lambda_s)_k (A theta_s)_k ]

(the second term through d theta_s / d b_k = -B'_s^{-1} a_k a_k^T theta_s).

Pinned in the tests by central finite differences of the forward loss
(`loss_only`), which uses no derivative at all.
"""
from __future__ import annotations

import numpy as np

from .islands import components, island_mask
from .powerflow import DirectSolver, laplacian

PV, SLACK = 1, 2


def _softplus(u):
    return np.logaddexp(0.0, u)


def _sigmoid(u):
    return 0.5 * (1.0 + np.tanh(0.5 * u))


def scenario_setup(grid, l, b):
    """Per-scenario DC structures for outage l and susceptances b."""
    n, m = grid.n_bus, grid.n_branch
    on = np.ones(m, dtype=bool)
    on[l] = False
    label = components(n, grid.f, grid.t, on)
    isl = island_mask(label, grid.slack)
    live = on & ~isl[grid.f] & ~isl[grid.t]
    keep = np.flatnonzero(~isl & (grid.bus_type != SLACK))
    pos = -np.ones(n, dtype=np.int64)
    pos[keep] = np.arange(keep.size)
    part = (grid.bus_type == PV) & ~isl & (grid.P_gen > 0)
    w = np.zeros(n)
    if isl.any() and part.any():
        w[part] = grid.P_gen[part] / grid.P_gen[part].sum()
    bs = np.where(live, b, 0.0)
    B = laplacian(n, grid.f, grid.t, bs, live, keep)
    return dict(isl=isl, live=live, keep=keep, pos=pos, w=w, bs=bs,
                solver=DirectSolver(B))


def redispatch_map(P, S):
    """R_s P: island injection moved onto main-island generators (weights w)."""
    Pt = P.astype(np.float64).copy()
    if S["isl"].any():
        Pt = Pt + S["w"] * P[S["isl"]].sum()
        Pt[S["isl"]] = 0.0
    return Pt


def redispatch_map_T(lam_full, S):
    """R_s^T applied to a bus vector (zero at the slack and islands)."""
    out = lam_full.copy()
    if S["isl"].any():
        out[S["isl"]] = S["w"] @ lam_full
    return out


def _theta(grid, P, S):
    th = np.zeros(grid.n_bus)
    rhs = redispatch_map(P, S)[S["keep"]]
    th[S["keep"]] = S["solver"].solve(rhs)
    return th


def penalty(f, rating):
    u = np.abs(f) / rating - 1.0
    return _softplus(u) ** 2


def penalty_grad(f, rating):
    u = np.abs(f) / rating - 1.0
    return 2.0 * _softplus(u) * _sigmoid(u) * np.sign(f) / rating


def loss_only(grid, outages, P, b):
    """The forward loss (no derivatives)."""
    L = 0.0
    for l in outages:
        S = scenario_setup(grid, int(l), b)
        th = _theta(grid, P, S)
        f = S["bs"] * (th[grid.f] - th[grid.t])
        L += float(penalty(f, grid.rating)[S["live"]].sum())
    return L


def loss_and_grad(grid, outages, P, b):
    """(L, dL/dP, dL/db) by the adjoint formulas above."""
    n, m = grid.n_bus, grid.n_branch
    L = 0.0
    gP = np.zeros(n)
    gb = np.zeros(m)
    for l in outages:
        S = scenario_setup(grid, int(l), b)
        th = _theta(grid, P, S)
        At = th[grid.f] - th[grid.t]
        f = S["bs"] * At
        live = S["live"]
        L += float(penalty(f, grid.rating)[live].sum())
        g = np.where(live, penalty_grad(f, grid.rating), 0.0)
        # A^T diag(b_s) g on the main island's non-slack buses
        y = np.zeros(n)
        np.add.at(y, grid.f, S["bs"] * g)
        np.add.at(y, grid.t, -S["bs"] * g)
        lam = np.zeros(n)
        lam[S["keep"]] = S["solver"].solve(y[S["keep"]])
        gP += redispatch_map_T(lam, S)
        Al = lam[grid.f] - lam[grid.t]
        gb += np.where(live, g * At - Al * At, 0.0)
    return L, gP, gb
