"""Small hand-built grids used by the tests (inputs only)."""
import json
import os

import numpy as np

from gridgen import Grid

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def grid_from_arrays(bus_type, P, Q, Pgen, Vset, f, t, r, x, b_sh, rating=None, tap=None,
                     Q_min=None, Q_max=None):
    m = len(f)
    return Grid(bus_type=np.asarray(bus_type, dtype=np.int8),
                P_sched=np.asarray(P, dtype=np.float64),
                Q_sched=np.asarray(Q, dtype=np.float64),
                P_gen=np.asarray(Pgen, dtype=np.float64),
                V_set=np.asarray(Vset, dtype=np.float64),
                f=np.asarray(f, dtype=np.int32), t=np.asarray(t, dtype=np.int32),
                r=np.asarray(r, dtype=np.float64), x=np.asarray(x, dtype=np.float64),
                b_sh=np.asarray(b_sh, dtype=np.float64),
                rating=np.ones(m) if rating is None else np.asarray(rating, dtype=np.float64),
                tap=None if tap is None else np.asarray(tap, dtype=np.float64),
                Q_min=None if Q_min is None else np.asarray(Q_min, dtype=np.float64),
                Q_max=None if Q_max is None else np.asarray(Q_max, dtype=np.float64))


def load_case(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        d = json.load(fh)
    return grid_from_arrays(d["bus_type"], d["P_sched"], d["Q_sched"], d["P_gen"],
                            d["V_set"], d["from"], d["to"], d["r"], d["x"], d["b_sh"],
                            d.get("rating"), d.get("tap"), d.get("Q_min"), d.get("Q_max")), d


def random_tree_grid(n, seed, lossless=True, all_pv=True):
    """Random tree, slack at bus 0, optional lossless / all-PV simplifications."""
    rng = np.random.default_rng(seed)
    parent = np.array([-1] + [int(rng.integers(0, i)) for i in range(1, n)])
    f = parent[1:]
    t = np.arange(1, n)
    x = rng.uniform(0.05, 0.3, n - 1)
    r = np.zeros(n - 1) if lossless else x / 10
    b_sh = np.zeros(n - 1) if lossless else rng.uniform(0, 0.05, n - 1)
    bt = np.full(n, 1 if all_pv else 0)
    bt[0] = 2
    if not all_pv:
        bt[rng.choice(np.arange(1, n), size=max(1, n // 5), replace=False)] = 1
    P = rng.uniform(-0.3, 0.1, n)
    P[0] = 0.0
    Q = -0.3 * np.abs(P)
    Vset = np.where(bt == 0, 1.0, rng.uniform(0.97, 1.05, n))
    Pgen = np.where(bt == 1, rng.uniform(0.1, 1.0, n), 0.0)
    return grid_from_arrays(bt, P, Q, Pgen, Vset, f, t, r, x, b_sh), parent
