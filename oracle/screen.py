"""The N-1 screen (Sec. IV.A): one scenario per single-branch outage.

Test infrastructure (see the package docstring).

For outage l: remove branch l; find the islands (Sec. IV.C); re-dispatch the
islands' injection over the main island; run the FDPF on the main island
starting from the base-case state (warm start, Sec. III.B); compute branch
flows and the loading max(|P_ij|, |P_ji|)/rating of every branch.  Islanded
buses report theta = V = 0, their branches zero flow.

Generator outages (the loss of a single component, Sec. IV.A): the PV bus k
loses its generator, so it keeps its load (P_sched[k] - P_gen[k] and
Q_sched[k]) and no longer holds its voltage: it becomes a PQ bus.  The lost
generation is re-dispatched (``redispatch.redispatch_generator``); no branch
leaves service and nothing is islanded.
"""
from __future__ import annotations

import contextlib
import multiprocessing as mp
import os

import numpy as np

from .islands import components, island_mask
from .powerflow import (STATUS_ISLAND_NO_GEN, STATUS_OK, branch_flows,
                        fdpf, mismatch, ybus_entries)
from .redispatch import redispatch, redispatch_generator


_BLAS_THREADS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


@contextlib.contextmanager
def worker_pool(processes):
    """A pool of `processes` spawned workers whose linear algebra runs on one
    thread each (the dense factorisations of small matrices would otherwise
    start a BLAS thread per core in every worker)."""
    saved = {k: os.environ.get(k) for k in _BLAS_THREADS}
    for k in _BLAS_THREADS:
        os.environ[k] = "1"
    try:
        pool = mp.get_context("spawn").Pool(processes)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    with pool:
        yield pool


def outage_setup(grid, l):
    """(in_service, labels, islanded mask, re-dispatched P_sched, no_gen)."""
    on = np.ones(grid.n_branch, dtype=bool)
    if l >= 0:
        on[l] = False
    label = components(grid.n_bus, grid.f, grid.t, on)
    isl = island_mask(label, grid.slack)
    P, no_gen = redispatch(grid.bus_type, grid.P_sched, grid.P_gen, isl)
    return on, label, isl, P, no_gen


def solve_outage(grid, theta0, V0, l, tol, max_outer):
    on, label, isl, P, no_gen = outage_setup(grid, l)
    active = ~isl
    switched, returned, held = [], [], []
    theta, V, k, status, err = fdpf(grid, on, active, P, theta0, V0, tol, max_outer,
                                    switched=switched, returned=returned, held_count=held)
    live = on & active[grid.f] & active[grid.t]
    Pf, Pt = branch_flows(grid.f, grid.t, grid.r, grid.x, live, theta, V, grid.tap)
    loading = np.maximum(np.abs(Pf), np.abs(Pt)) / grid.rating
    if status == STATUS_OK and no_gen:
        status = STATUS_ISLAND_NO_GEN
    return dict(theta=theta, V=V, flow=Pf, flow_to=Pt, label=label, outer=k,
                status=status, max_loading=float(loading.max(initial=0.0)),
                n_overload=int((loading > 1.0).sum()), err=err,
                islanded=bool(isl.any()), n_switched=len(switched),
                n_returned=len(returned), n_held=max(held, default=0))


def scenario_mismatch(grid, l, theta, V):
    """Max |dP| (non-slack buses) and |dQ| (PQ buses) of the main island for
    outage ``l`` at the given state: an independent check of any solver's
    answer."""
    on, label, isl, P, _ = outage_setup(grid, l)
    active = ~isl
    live = on & active[grid.f] & active[grid.t]
    yb = ybus_entries(grid.n_bus, grid.f, grid.t, grid.r, grid.x, grid.b_sh, live, grid.tap)
    dP, dQ = mismatch(yb, P, grid.Q_sched, np.where(active, theta, 0.0),
                      np.where(active, V, 0.0))
    bt = grid.bus_type
    a = np.abs(dP[active & (bt != 2)]).max(initial=0.0)
    b = np.abs(dQ[active & (bt == 0)]).max(initial=0.0)
    return max(a, b)


def generator_setup(grid, k):
    """The grid after the generator of PV bus k trips, and the no-generator
    flag of its re-dispatch."""
    if grid.bus_type[k] != 1:
        raise ValueError(f"bus {k} is not a PV bus")
    P, no_gen = redispatch_generator(grid.bus_type, grid.P_sched, grid.P_gen, int(k))
    g = grid.copy()
    g.bus_type = grid.bus_type.copy()
    g.bus_type[k] = 0
    g.P_sched = P
    return g, no_gen


def solve_generator_outage(grid, theta0, V0, k, tol, max_outer):
    g, no_gen = generator_setup(grid, k)
    on = np.ones(g.n_branch, dtype=bool)
    active = np.ones(g.n_bus, dtype=bool)
    switched, returned, held = [], [], []
    theta, V, it, status, err = fdpf(g, on, active, g.P_sched, theta0, V0, tol, max_outer,
                                     switched=switched, returned=returned, held_count=held)
    Pf, Pt = branch_flows(g.f, g.t, g.r, g.x, on, theta, V, g.tap)
    loading = np.maximum(np.abs(Pf), np.abs(Pt)) / g.rating
    if status == STATUS_OK and no_gen:
        status = STATUS_ISLAND_NO_GEN
    return dict(theta=theta, V=V, flow=Pf, flow_to=Pt,
                label=np.zeros(g.n_bus, dtype=np.int32), outer=it, status=status,
                max_loading=float(loading.max(initial=0.0)),
                n_overload=int((loading > 1.0).sum()), err=err, islanded=False,
                n_switched=len(switched), n_returned=len(returned),
                n_held=max(held, default=0))


def generator_mismatch(grid, k, theta, V):
    """Max |dP| (non-slack buses) and |dQ| (PQ buses, the tripped one
    included) after the generator of bus k trips, at the given state."""
    g, _ = generator_setup(grid, k)
    on = np.ones(g.n_branch, dtype=bool)
    yb = ybus_entries(g.n_bus, g.f, g.t, g.r, g.x, g.b_sh, on, g.tap)
    dP, dQ = mismatch(yb, g.P_sched, g.Q_sched, theta, V)
    return max(np.abs(dP[g.bus_type != 2]).max(initial=0.0),
               np.abs(dQ[g.bus_type == 0]).max(initial=0.0))


def _worker(args):
    grid, theta0, V0, ls, tol, max_outer, kind = args
    solve = solve_outage if kind == "branch" else solve_generator_outage
    return [solve(grid, theta0, V0, int(l), tol, max_outer) for l in ls]


def n1_screen(grid, theta0, V0, outages, tol=1e-4, max_outer=50, processes=None,
              kind="branch"):
    """Solve every outage in ``outages`` (branch indices, or PV bus indices
    with kind="generator"); returns stacked result arrays."""
    outages = np.asarray(outages, dtype=np.int64)
    S = outages.shape[0]
    if processes is None:
        processes = len(os.sched_getaffinity(0))
    processes = max(1, min(processes, S))
    if processes == 1 or S < 8:
        res = _worker((grid, theta0, V0, outages, tol, max_outer, kind))
    else:
        chunks = np.array_split(outages, processes * 4)
        with worker_pool(processes) as pool:
            parts = pool.map(_worker, [(grid, theta0, V0, c, tol, max_outer, kind)
                                       for c in chunks if c.size])
        res = [r for p in parts for r in p]
    out = {}
    for key in ("theta", "V", "flow", "flow_to", "label"):
        out[key] = np.stack([r[key] for r in res]) if S else np.zeros((0, 0))
    for key, dt in (("outer", np.int32), ("status", np.int32),
                    ("max_loading", np.float64), ("n_overload", np.int32),
                    ("err", np.float64), ("islanded", bool), ("n_switched", np.int32),
                    ("n_returned", np.int32), ("n_held", np.int32)):
        out[key] = np.asarray([r[key] for r in res], dtype=dt)
    out["processes"] = processes
    return out
