"""Proportional re-dispatch of an island's injection (Sec. IV.C).

Test infrastructure (see the package docstring).

The paper states only that the power an island exported to (or imported
from) the main system is made up by the main system, shared proportionally
among its major generators or loads.  It gives no formula, so this function
is **parity unpinned**: it follows the reading below and is checked only
through the power-balance invariant (the main island's scheduled injection
after re-dispatch equals its value before the outage).

Reading: the island's net scheduled injection
    dP_isl = sum_{i in islands} P_sched[i]
is added to the main island's PV generators (slack excluded) with positive
scheduled generation, in proportion to that generation:
    P_sched[k] += dP_isl * P_gen[k] / sum_{k' main PV} P_gen[k'].
The sign is kept, so an exporting island raises the main generators and an
importing island lowers them.  If the main island has no such generator the
slack absorbs the difference and the scenario is flagged.

A generator outage (the loss of a single component other than a branch,
Sec. IV.A) is read the same way: the tripped PV bus loses its scheduled
generation P_gen[k], and that power is taken up by the other PV generators
with positive scheduled generation in proportion to it (slack excluded; the
slack absorbs it if there are none).  Also **parity unpinned** beyond the
balance invariant.
"""
from __future__ import annotations

import numpy as np

PV = 1


def redispatch(bus_type: np.ndarray, P_sched: np.ndarray, P_gen: np.ndarray,
               islanded: np.ndarray):
    """Return (P_sched after re-dispatch, no_generator_flag)."""
    P = P_sched.astype(np.float64).copy()
    if not islanded.any():
        return P, False
    dP = float(P_sched[islanded].sum())
    part = (bus_type == PV) & (~islanded) & (P_gen > 0.0)
    if not part.any():
        P[islanded] = 0.0
        return P, True
    w = P_gen[part] / P_gen[part].sum()
    P[part] += dP * w
    P[islanded] = 0.0
    return P, False


def redispatch_generator(bus_type: np.ndarray, P_sched: np.ndarray, P_gen: np.ndarray,
                         k: int):
    """Trip the generator of PV bus k: (P_sched after re-dispatch, no_generator_flag)."""
    P = P_sched.astype(np.float64).copy()
    lost = float(P_gen[k])
    P[k] -= lost
    part = (bus_type == PV) & (P_gen > 0.0)
    part[k] = False
    if not part.any():
        return P, True
    P[part] += lost * P_gen[part] / P_gen[part].sum()
    return P, False
