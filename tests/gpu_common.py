"""Shared fixtures of the GPU parity tests (the CUDA path via the C ABI
against the CPU oracle on the same seeded inputs)."""
import functools

import numpy as np

from gridgen import CONFIGS, config_grid, make_grid
from oracle import powerflow as pf
from oracle import screen

# Grids of the named workloads with a share of their branches turned into
# transformers (off-nominal turns ratios U[0.95, 1.05] at the from end).
XFMR = {"grid120_xfmr": ("grid120", 0.15), "grid2k_xfmr": ("grid2k", 0.1),
        "grid10k_xfmr": ("grid10k", 0.1)}


# Grids with reactive limits around their PV generators' base-case output:
# Q_max = Q_g + 0.05 + 0.1 |Q_g|, Q_min = Q_g - 0.05 - 0.1 |Q_g|, so the base
# case is within them and outages push some generators out.
QLIM = {"grid120_qlim": "grid120", "grid2k_qlim": "grid2k", "grid10k_qlim": "grid10k"}


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


# ---------------------------------------------------------------------------
# Every outage of a screen against the oracle, scenario by scenario.
def _every_outage_worker(args):
    """One chunk of scenarios: the oracle's own FDPF (status, labels), and
    the oracle's FP64 evaluation of the GPU's state (mismatch, overloads)."""
    g, th0, V0, idx, outages, paths, tol, max_outer = args
    th = np.load(paths["theta"], mmap_mode="r")
    V = np.load(paths["V"], mmap_mode="r")
    lab = np.load(paths["label"], mmap_mode="r")
    st = np.load(paths["status"], mmap_mode="r")
    from oracle import powerflow as opf
    rows = []
    for s in idx:
        l = int(outages[s])
        r = screen.solve_outage(g, th0, V0, l, tol, max_outer)
        lab_ok = bool(np.array_equal(r["label"], lab[s]))
        err = np.nan
        nov, ties = -1, 0
        if st[s] in (0, 3):
            ths, Vs = np.asarray(th[s]), np.asarray(V[s])
            err = screen.scenario_mismatch(g, l, ths, Vs)
            on, _, isl, _, _ = screen.outage_setup(g, l)
            live = on & ~isl[g.f] & ~isl[g.t]
            Pf, Pt = opf.branch_flows(g.f, g.t, g.r, g.x, live, np.where(isl, 0.0, ths),
                                      np.where(isl, 0.0, Vs), g.tap)
            ld = np.maximum(np.abs(Pf), np.abs(Pt)) / g.rating
            nov = int((ld > 1.0).sum())
            ties = int((np.abs(ld - 1.0) <= 1e-12).sum())
        rows.append((int(r["status"]), lab_ok, float(err), nov, ties, int(r["n_held"])))
    return idx, rows


def check_every_outage(g, th0, V0, outages, res, tol, tmpdir, max_outer=50, processes=None):
    """Run the oracle on every scenario of a GPU screen `res` (host outputs
    theta, V, label, status, n_overload of `outages`) in a pool of host
    processes.  Returns per scenario: the oracle's status, whether the island
    labels are identical, the oracle's FP64 mismatch of the GPU's state (NaN
    where the GPU did not converge), and the oracle's overload count at the
    GPU's state with the number of branches within 1e-12 of their rating,
    and the peak number of buses the oracle held at a reactive limit."""
    import os
    paths = {}
    for k in ("theta", "V", "label", "status"):
        paths[k] = os.path.join(str(tmpdir), f"{k}.npy")
        np.save(paths[k], res[k])
    S = len(outages)
    if processes is None:
        processes = len(os.sched_getaffinity(0))
    chunks = [c for c in np.array_split(np.arange(S), max(1, processes * 8)) if c.size]
    args = [(g, th0, V0, c, np.asarray(outages), paths, tol, max_outer) for c in chunks]
    st = np.empty(S, np.int32)
    lab_ok = np.empty(S, bool)
    err = np.empty(S)
    nov = np.empty(S, np.int32)
    ties = np.empty(S, np.int32)
    held = np.empty(S, np.int32)
    with screen.worker_pool(processes) as pool:
        for idx, rows in pool.imap_unordered(_every_outage_worker, args):
            for s, row in zip(idx, rows):
                st[s], lab_ok[s], err[s], nov[s], ties[s], held[s] = row
    return dict(status=st, label_ok=lab_ok, err=err, n_overload=nov, ties=ties, n_held=held)


def _every_dc_outage_worker(args):
    """One chunk of DC scenarios: the oracle's direct solves against each
    GPU run's angles and flows (max abs differences), its status, and its
    overload count with the branches within `tie` of their rating."""
    g, idx, outages, paths, tie = args
    from oracle import dc
    runs = {name: (np.load(p["theta"], mmap_mode="r"), np.load(p["flow"], mmap_mode="r"))
            for name, p in paths.items()}
    rows = []
    for s in idx:
        r = dc.dc_screen(g, outages[s:s + 1])
        ld = np.abs(r["flow"][0]) / g.rating
        diffs = {name: (float(np.abs(r["theta"][0] - th[s]).max()),
                        float(np.abs(r["flow"][0] - fl[s]).max()))
                 for name, (th, fl) in runs.items()}
        rows.append((int(r["status"][0]), int(r["n_overload"][0]),
                     int((np.abs(ld - 1.0) <= tie).sum()), diffs))
    return idx, rows


def check_every_dc_outage(g, outages, runs, tmpdir, tie=1e-6, processes=None):
    """The DC oracle on every scenario of GPU DC screens (`runs`: name ->
    host outputs theta, flow of `outages`) in a pool of host processes.
    Returns per scenario the oracle's status, overload count and number of
    near-ties, and for each run the max angle and flow differences."""
    import os
    paths = {}
    for name, res in runs.items():
        paths[name] = {}
        for k in ("theta", "flow"):
            paths[name][k] = os.path.join(str(tmpdir), f"dc_{name}_{k}.npy")
            np.save(paths[name][k], res[k])
    S = len(outages)
    if processes is None:
        processes = len(os.sched_getaffinity(0))
    chunks = [c for c in np.array_split(np.arange(S), max(1, processes * 8)) if c.size]
    args = [(g, c, np.asarray(outages), paths, tie) for c in chunks]
    out = {"status": np.empty(S, np.int32), "n_overload": np.empty(S, np.int32),
           "ties": np.empty(S, np.int32)}
    for name in runs:
        out[name] = {"dtheta": np.empty(S), "dflow": np.empty(S)}
    with screen.worker_pool(processes) as pool:
        for idx, rows in pool.imap_unordered(_every_dc_outage_worker, args):
            for s, (st, nov, ties, diffs) in zip(idx, rows):
                out["status"][s], out["n_overload"][s], out["ties"][s] = st, nov, ties
                for name, (dt, dfl) in diffs.items():
                    out[name]["dtheta"][s], out[name]["dflow"][s] = dt, dfl
    return out


def _every_generator_outage_worker(args):
    """One chunk of generator outages: the oracle's own FDPF (status, peak
    number of held buses) and its FP64 evaluation of the GPU's state."""
    g, th0, V0, idx, buses, paths, tol, max_outer = args
    th = np.load(paths["theta"], mmap_mode="r")
    V = np.load(paths["V"], mmap_mode="r")
    st = np.load(paths["status"], mmap_mode="r")
    rows = []
    for s in idx:
        k = int(buses[s])
        r = screen.solve_generator_outage(g, th0, V0, k, tol, max_outer)
        err = np.nan
        if st[s] in (0, 3):
            err = screen.generator_mismatch(g, k, np.asarray(th[s]), np.asarray(V[s]))
        rows.append((int(r["status"]), float(err), int(r["n_held"])))
    return idx, rows


def check_every_generator_outage(g, th0, V0, buses, res, tol, tmpdir, max_outer=50,
                                 processes=None):
    """The oracle on every generator outage of a GPU screen `res` (host
    outputs theta, V, status of the tripped PV `buses`) in a pool of host
    processes: per scenario the oracle's status, its FP64 mismatch of the
    GPU's state (NaN where the GPU did not converge) and the peak number of
    buses it held at a reactive limit."""
    import os
    paths = {}
    for k in ("theta", "V", "status"):
        paths[k] = os.path.join(str(tmpdir), f"gen_{k}.npy")
        np.save(paths[k], res[k])
    S = len(buses)
    if processes is None:
        processes = len(os.sched_getaffinity(0))
    chunks = [c for c in np.array_split(np.arange(S), max(1, processes * 8)) if c.size]
    args = [(g, th0, V0, c, np.asarray(buses), paths, tol, max_outer) for c in chunks]
    st = np.empty(S, np.int32)
    err = np.empty(S)
    held = np.empty(S, np.int32)
    with screen.worker_pool(processes) as pool:
        for idx, rows in pool.imap_unordered(_every_generator_outage_worker, args):
            for s, row in zip(idx, rows):
                st[s], err[s], held[s] = row
    return dict(status=st, err=err, n_held=held)


def with_tight_ratings(g, seed):
    """The grid with every branch rated at U[1.0, 1.5] times its base-case
    loading max(|P_ij|, |P_ji|) (plus 1e-3 p.u.), so that outages push flows
    above the ratings of their neighbours.  Ratings do not enter the power
    flow: only the overload screen sees them."""
    th, V, _, st, _ = pf.base_case(g, tol=1e-11, max_outer=200)
    assert st == pf.STATUS_OK
    Pf, Pt = pf.branch_flows(g.f, g.t, g.r, g.x, np.ones(g.n_branch, bool), th, V, g.tap)
    rng = np.random.default_rng(seed)
    g = g.copy()
    g.rating = np.maximum(np.abs(Pf), np.abs(Pt)) * rng.uniform(1.0, 1.5, g.n_branch) + 1e-3
    return g
