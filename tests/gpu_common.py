"""Shared fixtures of the GPU parity tests (the CUDA path via the C ABI
against the CPU oracle on the same seeded inputs)."""
import functools

import numpy as np

from gridgen import CONFIGS, config_grid, make_grid
from oracle import powerflow as pf
from oracle import screen

# Grids of the named workloads with a share of their branches turned into
# transformers (off-nominal turns ratios U[0.95, 1.05] at the from end).
XFMR = {"grid120_xfmr": ("grid120", 0.15), "grid2k_xfmr": ("grid2k", 0.1)}


# Grids with reactive limits around their PV generators' base-case output:
# Q_max = Q_g + 0.05 + 0.1 |Q_g|, Q_min = Q_g - 0.05 - 0.1 |Q_g|, so the base
# case is within them and outages push some generators out.
QLIM = {"grid120_qlim": "grid120", "grid2k_qlim": "grid2k"}


def _with_q_limits(g):
    th, V, _, st, _ = pf.base_case(g, tol=1e-11, max_outer=200)
    assert st == pf.STATUS_OK
    yb = pf.ybus_entries(g.n_bus, g.f, g.t, g.r, g.x, g.b_sh, np.ones(g.n_branch, bool), g.tap)
    _, dQ = pf.mismatch(yb, g.P_sched, g.Q_sched, th, V)
    qg = -dQ
    g = g.copy()
    g.Q_max = qg + 0.05 + 0.1 * np.abs(qg)
    g.Q_min = qg - 0.05 - 0.1 * np.abs(qg)
    return g


@functools.lru_cache(maxsize=None)
def grid(name):
    if name in QLIM:
        g = _with_q_limits(config_grid(QLIM[name]))
        g.meta["config"] = name
        return g
    if name in XFMR:
        base, frac = XFMR[name]
        g = make_grid(gen_share=1.0, xfmr_frac=frac, **CONFIGS[base])
        g.meta["config"] = name
        return g
    return config_grid(name)


@functools.lru_cache(maxsize=None)
def oracle_base(name):
    g = grid(name)
    th, V, k, st, err = pf.base_case(g, tol=1e-11, max_outer=200)
    assert st == pf.STATUS_OK
    return th, V


def oracle_n1(name, outages, tol=1e-10, processes=None):
    g = grid(name)
    th0, V0 = oracle_base(name)
    return screen.n1_screen(g, th0, V0, outages, tol=tol, max_outer=100, processes=processes)


def sample_outages(g, k, seed=0, include_bridges=True):
    """A seeded sample of outages that always includes islanding ones."""
    from oracle import islands
    rng = np.random.default_rng(seed)
    picks = set(rng.choice(g.n_branch, size=min(k, g.n_branch), replace=False).tolist())
    if include_bridges:
        on = np.ones(g.n_branch, bool)
        found = 0
        for l in rng.permutation(g.n_branch):
            on[l] = False
            lab = islands.components(g.n_bus, g.f, g.t, on)
            on[l] = True
            if (lab != lab[g.slack]).any():
                picks.add(int(l))
                found += 1
                if found >= max(2, k // 8):
                    break
    return np.array(sorted(picks), dtype=np.int32)
