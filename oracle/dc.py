"""N-1 quick screen of the P-theta (DC) model (test infrastructure).

The paper's quick screening looks at the P-theta equation (4) alone
(Sec. IV.A).  With |V| = 1 that equation is the DC power flow: for the
outage of branch l, with the islands removed and their injection
re-dispatched over the main island's generators (Sec. IV.C),

    B'_s theta_s = R_s P      (slack angle 0, islanded buses 0),
    f_s,k = (theta_s,i - theta_s,j) / x_k   on branches k = (i, j) in service
                                            between main-island buses, else 0,
    loading_s = max_k |f_s,k| / rating_k,
    n_overload_s = #{k : |f_s,k| / rating_k > 1}   (the overload screen, Sec. I).

B'_s is re-formed and factorised directly for every scenario (the same
"LUD" route as the AC oracle).  Pinned in the tests by closed forms: on a
radial grid every branch carries the net injection beyond it, and for a
non-bridge outage the post-outage flows equal the base flows corrected by
the line-outage distribution factors of the base matrix (Sherman-Morrison).
"""
from __future__ import annotations

import numpy as np

from . import adjoint as adj
from .islands import components

STATUS_OK, STATUS_ISLAND_NO_GEN = 0, 3
PV = 1


def dc_screen(grid, outages, P=None):
    """DC N-1 screen: theta [S][n], flow [S][m], max_loading [S], status [S],
    label [S][n] (component labels, minimum bus index), n_overload [S]."""
    n, m = grid.n_bus, grid.n_branch
    P = grid.P_sched if P is None else np.asarray(P, dtype=np.float64)
    b = 1.0 / grid.x
    S = len(outages)
    theta = np.zeros((S, n))
    flow = np.zeros((S, m))
    ml = np.zeros(S)
    nov = np.zeros(S, dtype=np.int32)
    status = np.zeros(S, dtype=np.int32)
    label = np.zeros((S, n), dtype=np.int32)
    for s, l in enumerate(outages):
        Ss = adj.scenario_setup(grid, int(l), b)
        th = adj._theta(grid, P, Ss)
        f = Ss["bs"] * (th[grid.f] - th[grid.t])
        theta[s] = th
        flow[s] = f
        ml[s] = float(np.max(np.abs(f) / grid.rating)) if m else 0.0
        nov[s] = int((np.abs(f) / grid.rating > 1.0).sum())
        main_gen = (grid.bus_type == PV) & ~Ss["isl"] & (grid.P_gen > 0)
        status[s] = STATUS_ISLAND_NO_GEN if Ss["isl"].any() and not main_gen.any() else STATUS_OK
        on = np.ones(m, dtype=bool)
        on[int(l)] = False
        label[s] = components(n, grid.f, grid.t, on)
    return dict(theta=theta, flow=flow, max_loading=ml, status=status, label=label,
                n_overload=nov)
