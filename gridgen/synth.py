"""Seeded synthetic grid generator.

The paper's test system (a 1,425-bus provincial grid, Sec. V) is not public,
so seeded synthetic grids with the shapes of the evaluated workloads stand in
for it.  A grid is a plain structure of arrays in the bus/branch form the
paper's graph model uses (Sec. II.B: buses are vertices with voltage, angle,
injection and type; branches are edges with impedance, charging and a flow
limit).

Recipe (every draw comes from one ``numpy.random.default_rng(seed)``):

* buses uniform in the unit square;
* a random spanning tree: minimum spanning tree of the 6-nearest-neighbour
  graph under i.i.d. U(0,1) edge weights (components of the k-NN graph, if
  any, are joined by their closest pair);
* chords: the shortest not-yet-present k-NN pairs are added until the
  requested branch count is reached (no parallel branches);
* optional radial spurs: a fraction of the buses hangs off random core buses
  in chains of one or two buses; each spur bus adds one branch;
* branch parameters x ~ U[0.01, 0.2], r = x/10, total charging
  b_sh ~ U[0, 0.05], rating ~ U[1, 3] (all per unit);
* every bus carries a load P_d ~ LogNormal(ln 0.5, 0.6) scaled by the loading
  factor, Q_d = 0.3 P_d;
* 20 % of the buses are PV generators; the PV bus nearest the centroid is
  the slack; PV generation is proportional to U[0.5, 1.5] draws, scaled so
  the PV buses together supply ``gen_share`` of the total load; the slack
  covers the rest and the losses;
* |V| set points 1.02 (PV) and 1.04 (slack); PQ buses start at 1.0.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components, minimum_spanning_tree
from scipy.spatial import cKDTree

PQ, PV, SLACK = 0, 1, 2


@dataclasses.dataclass
class Grid:
    """Bus/branch arrays, 0-based bus indices, per-unit quantities."""

    bus_type: np.ndarray  # int8 [n]   0=PQ 1=PV 2=slack
    P_sched: np.ndarray   # f64 [n]    net active injection (gen - load)
    Q_sched: np.ndarray   # f64 [n]    net reactive injection of PQ buses
    P_gen: np.ndarray     # f64 [n]    scheduled generation (re-dispatch weights)
    V_set: np.ndarray     # f64 [n]    |V| set point (PV/slack), start value (PQ)
    f: np.ndarray         # int32 [m]  from bus
    t: np.ndarray         # int32 [m]  to bus
    r: np.ndarray         # f64 [m]
    x: np.ndarray         # f64 [m]
    b_sh: np.ndarray      # f64 [m]    total line charging
    rating: np.ndarray    # f64 [m]
    tap: Optional[np.ndarray] = None  # f64 [m] off-nominal turns ratio at the from end
                                      # (transformers); None: every branch is a line
    Q_min: Optional[np.ndarray] = None  # f64 [n] reactive limits of the PV generators
    Q_max: Optional[np.ndarray] = None  # (None: no limits)
    xy: Optional[np.ndarray] = None  # f64 [n, 2] bus coordinates (plotting only)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_bus(self) -> int:
        return int(self.bus_type.shape[0])

    @property
    def n_branch(self) -> int:
        return int(self.f.shape[0])

    @property
    def slack(self) -> int:
        return int(np.flatnonzero(self.bus_type == SLACK)[0])

    def copy(self) -> "Grid":
        return dataclasses.replace(
            self, **{k.name: (getattr(self, k.name).copy()
                              if isinstance(getattr(self, k.name), np.ndarray)
                              else getattr(self, k.name))
                     for k in dataclasses.fields(self) if k.name != "meta"},
            meta=dict(self.meta))


def _spanning_tree(xy: np.ndarray, rng: np.random.Generator, k: int):
    n = xy.shape[0]
    tree = cKDTree(xy)
    kk = min(k + 1, n)
    dist, idx = tree.query(xy, k=kk)
    rows = np.repeat(np.arange(n), kk - 1)
    cols = idx[:, 1:].reshape(-1)
    d = dist[:, 1:].reshape(-1)
    a = np.minimum(rows, cols)
    b = np.maximum(rows, cols)
    key = a.astype(np.int64) * n + b
    key, first = np.unique(key, return_index=True)
    a, b, d = a[first], b[first], d[first]
    w = rng.uniform(0.0, 1.0, size=a.shape[0]) + 1e-12
    g = coo_matrix((w, (a, b)), shape=(n, n)).tocsr()
    # join k-NN components (rare) through their closest pair
    ncomp, lab = connected_components(g, directed=False)
    extra = []
    while ncomp > 1:
        c0 = np.flatnonzero(lab == lab[0])
        rest = np.flatnonzero(lab != lab[0])
        t_rest = cKDTree(xy[rest])
        dd, jj = t_rest.query(xy[c0], k=1)
        i0 = int(np.argmin(dd))
        u, v = int(c0[i0]), int(rest[jj[i0]])
        extra.append((min(u, v), max(u, v)))
        g = g + coo_matrix(([1e-12], ([min(u, v)], [max(u, v)])), shape=(n, n)).tocsr()
        ncomp, lab = connected_components(g, directed=False)
    mst = minimum_spanning_tree(g).tocoo()
    tf = np.minimum(mst.row, mst.col)
    tt = np.maximum(mst.row, mst.col)
    cand = (a, b, d)
    return tf.astype(np.int64), tt.astype(np.int64), cand


def make_grid(n_bus: int, n_branch: int, seed: int, spur_frac: float = 0.0,
              pv_frac: float = 0.2, load_scale: float = 1.0,
              gen_share: float = 1.0, knn: int = 6,
              local_gen: bool = True, v_pv: float = 1.02,
              v_slack: float = 1.04, xfmr_frac: float = 0.0) -> Grid:
    """Draw a connected synthetic grid with ``n_bus`` buses, ``n_branch`` branches.

    ``xfmr_frac`` > 0 makes that fraction of the branches transformers with
    an off-nominal turns ratio U[0.95, 1.05] at the from end; those draws come
    after every other one, so the rest of the grid is the same as without."""
    rng = np.random.default_rng(seed)
    n_spur = int(round(spur_frac * n_bus))
    n_core = n_bus - n_spur
    if n_core < 2:
        raise ValueError("need at least two core buses")
    xy = rng.uniform(0.0, 1.0, size=(n_core, 2))
    tf, tt, (ca, cb, cd) = _spanning_tree(xy, rng, knn)
    m_core = n_branch - n_spur
    if m_core < n_core - 1:
        raise ValueError("too few branches for a spanning tree")
    have = set((tf * n_core + tt).tolist())
    order = np.argsort(cd, kind="stable")
    ef, et = list(tf), list(tt)
    for o in order:
        if len(ef) >= m_core:
            break
        key = int(ca[o]) * n_core + int(cb[o])
        if key in have:
            continue
        have.add(key)
        ef.append(int(ca[o]))
        et.append(int(cb[o]))
    if len(ef) < m_core:
        raise ValueError("k-NN candidate pool too small for the branch count")
    # radial spurs: chains of length 1 or 2 hung off random core buses
    spur_xy = []
    nxt = n_core
    while nxt < n_bus:
        root = int(rng.integers(0, n_core))
        ln = int(rng.integers(1, 3))
        ln = min(ln, n_bus - nxt)
        prev = root
        for _ in range(ln):
            spur_xy.append(xy[root] + rng.normal(0.0, 0.002, size=2))
            ef.append(prev)
            et.append(nxt)
            prev = nxt
            nxt += 1
    if spur_xy:
        xy = np.vstack([xy, np.asarray(spur_xy)])
    f = np.asarray(ef, dtype=np.int32)
    t = np.asarray(et, dtype=np.int32)
    m = f.shape[0]
    # shuffle branch order so bridges and chords interleave
    perm = rng.permutation(m)
    f, t = f[perm], t[perm]
    flip = rng.uniform(size=m) < 0.5
    f, t = np.where(flip, t, f).astype(np.int32), np.where(flip, f, t).astype(np.int32)

    x = rng.uniform(0.01, 0.2, size=m)
    r = x / 10.0
    b_sh = rng.uniform(0.0, 0.05, size=m)
    rating = rng.uniform(1.0, 3.0, size=m)

    Pd = rng.lognormal(np.log(0.5), 0.6, size=n_bus) * load_scale
    Qd = 0.3 * Pd
    n_pv = max(1, int(round(pv_frac * n_bus)))
    pv = rng.choice(n_bus, size=n_pv, replace=False)
    bus_type = np.zeros(n_bus, dtype=np.int8)
    bus_type[pv] = PV
    centroid = xy.mean(axis=0)
    slack = int(pv[np.argmin(((xy[pv] - centroid) ** 2).sum(axis=1))])
    bus_type[slack] = SLACK
    gen_pv = np.flatnonzero(bus_type == PV)
    w = rng.uniform(0.5, 1.5, size=gen_pv.shape[0])
    if local_gen:
        # each load is served by its nearest generator (plane distance)
        _, near = cKDTree(xy[gen_pv]).query(xy, k=1)
        w = w * np.bincount(near, weights=Pd, minlength=gen_pv.shape[0])
    Pg = np.zeros(n_bus)
    Pg[gen_pv] = w / w.sum() * gen_share * Pd.sum()
    P_sched = Pg - Pd
    Q_sched = -Qd
    V_set = np.ones(n_bus)
    V_set[bus_type == PV] = v_pv
    V_set[slack] = v_slack
    tap = None
    if xfmr_frac > 0.0:
        tap = np.ones(m)
        k = rng.choice(m, size=max(1, int(round(xfmr_frac * m))), replace=False)
        tap[k] = rng.uniform(0.95, 1.05, size=k.shape[0])
    g = Grid(bus_type=bus_type, P_sched=P_sched, Q_sched=Q_sched, P_gen=Pg,
             V_set=V_set, f=f, t=t, r=r, x=x, b_sh=b_sh, rating=rating, tap=tap, xy=xy,
             meta=dict(n_bus=n_bus, n_branch=m, seed=seed, spur_frac=spur_frac,
                       load_scale=load_scale, gen_share=gen_share, xfmr_frac=xfmr_frac))
    return g


# Workload table.  ``load_scale`` is the loading factor lambda applied to
# every load; at the nominal loading (lambda = 1) the base case of grids with
# more than a few hundred buses has no power-flow solution, so lambda is the
# largest value from the ladder {1, .5, .3, .2, .1, .05, .03, .02, .01} for
# which the FP64 base case converges with every branch's angle difference
# below 0.4 rad (grid10k converges at 0.1 too, with differences up to 0.69
# rad; grid50k converges only at 0.01).
CONFIGS = {
    # 120-bus grid, all ~180 single-branch outages, plain FP64
    "grid120": dict(n_bus=120, n_branch=180, seed=1, spur_frac=0.0, load_scale=0.3),
    # 2,000-bus grid, ~2,700 outages (also the adjoint workload)
    "grid2k": dict(n_bus=2000, n_branch=2700, seed=2, spur_frac=0.0, load_scale=0.1),
    # 10,000-bus grid, ~13,500 outages, 5 % of buses on radial spurs
    "grid10k": dict(n_bus=10000, n_branch=13500, seed=3, spur_frac=0.05, load_scale=0.05),
    # 50,000-bus grid, ~70,000 outages; |V| set points of 1.0: with 1.02/1.04
    # the reactive circulation's losses exceed what a single slack can carry
    "grid50k": dict(n_bus=50000, n_branch=70000, seed=5, spur_frac=0.0, load_scale=0.01,
                    v_pv=1.0, v_slack=1.0),
}


def config_grid(name: str) -> Grid:
    """The synthetic grid of a named workload (see ``CONFIGS``)."""
    kw = dict(CONFIGS[name])
    g = make_grid(gen_share=1.0, **kw)
    g.meta["config"] = name
    return g
