"""Power mismatch, fast-decoupled matrices, branch flows and FDPF (FP64).

Test infrastructure (see the package docstring).

Network model (pi-model branch l = (i, j) from i to j): series admittance
y = 1/(r + jx) = g + j b_y with g = r/(r^2+x^2), b_y = -x/(r^2+x^2); half of
the total charging b_sh sits at each end.  A transformer branch carries an
off-nominal turns ratio tau (an edge attribute of the paper's graph model,
Sec. II.B): an ideal tau:1 transformer at the from end in series with the
pi-model, no phase shift.  Its from-end voltage reaches the pi-model as
V_i / tau, so with c = 1/tau (c = 1 for a line)
    Y_ii += c^2 (y + j b_sh/2),  Y_jj += y + j b_sh/2,  Y_ij = Y_ji = -c y.
G_ij and B_ij of eqs. (1)-(3) are the real and imaginary parts of Y.

Fast-decoupled matrices (eqs. (4)-(5); the paper names no variant, the XB
form is used): B' is the Laplacian of the in-service branches weighted by
1/x (turns ratios and charging left out); B'' is minus the imaginary part
of the bus admittance matrix of the series branches with their turns ratios,
charging left out: every branch adds w v v^T with w = x/(r^2+x^2) and
v = c e_i - e_j.  B' is restricted to the non-slack buses of the main island,
B'' to its PQ buses; both are sums of positive semi-definite branch terms
grounded at the removed buses, hence symmetric positive definite.

FDPF (eqs. (4)-(5), Sec. III.B): starting from a given state, repeat
  evaluate dP, dQ; stop when max|dP| (PV and PQ buses) and max|dQ| (PQ buses)
  are both <= tol; unless max|dP| is already <= tol, solve B' dtheta = dP/V,
  theta += dtheta and evaluate dQ again; unless max|dQ| is then <= tol,
  solve B'' dV = dQ/V, V += dV.  (A half-step whose own mismatch is within
  the tolerance is skipped, as in the fast-decoupled method the paper builds
  on; the outer count advances once per pass through the loop.)

Reactive limits of the PV generators (Q_min, Q_max per bus; the paper has
none, this is the usual enforcement): when the iteration has converged, the
generator output a PV bus needs, Q_g = Q(V) - Q_sched = -dQ, is compared
with its limits; every PV bus outside them becomes a PQ bus whose generator
is held at the violated limit (Q_sched += Q_max or Q_min), B'' gains its row,
and the iteration continues from the current state.  At the same check a
bus held at Q_max whose |V| has risen above its set point (or held at Q_min,
fallen below it) turns back PV at the set point: its generator can hold the
set point within its limits again.  The result converges with every PV bus
within its limits and every held bus on its side of the set point.
The paper gives no stopping rule for a diverging case; here a run is
declared diverged when the mismatch is not finite, exceeds DIVERGE_LIMIT, or
(for warm-started scenarios) has grown to DIVERGE_GROWTH times the smallest
value it reached (the iteration has left its basin of convergence).
Every solve here is direct (re-formed, fully factorised matrix), so the
result is the exact AC solution up to the tolerance.

Pins (tests): hand-solved two-bus case, the radial closed form (tree,
lossless, all-PV: flows fixed by Kirchhoff's current law, angles by arcsin),
Newton-Raphson on small cases, Sherman-Morrison/LODF for the first post-outage
P-theta solve, the power-balance and KCL invariants, the four-element
difference of Sec. IV.B.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
from scipy.sparse import coo_matrix, csc_matrix
from scipy.sparse.linalg import splu

PQ, PV, SLACK = 0, 1, 2
STATUS_OK, STATUS_MAXITER, STATUS_DIVERGED, STATUS_ISLAND_NO_GEN = 0, 1, 2, 3
DIVERGE_LIMIT = 1.0e4   # p.u.; a mismatch above this is taken as divergence
DIVERGE_GROWTH = 10.0   # or one this many times above the smallest seen so far
DENSE_MAX = 500          # direct solves use dense LU up to this size


def series_admittance(r: np.ndarray, x: np.ndarray):
    """(g, b_y) of y = 1/(r + jx)."""
    d = r * r + x * x
    return r / d, -x / d


def tap_factor(tap, m):
    """c = 1/tau per branch (1 for lines; ``tap`` None means no transformers)."""
    return np.ones(m) if tap is None else 1.0 / np.asarray(tap, dtype=np.float64)


def ybus_entries(n_bus, f, t, r, x, b_sh, in_service, tap=None):
    """Summed nonzeros (row, col, G, B) of the bus admittance matrix."""
    on = np.asarray(in_service, dtype=bool)
    c = tap_factor(tap, len(f))[on]
    f, t, r, x, b_sh = f[on], t[on], r[on], x[on], b_sh[on]
    g, b = series_admittance(r, x)
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([t, f, f, t])
    Gv = np.concatenate([-c * g, -c * g, c * c * g, g])
    Bv = np.concatenate([-c * b, -c * b, c * c * (b + 0.5 * b_sh), b + 0.5 * b_sh])
    # diagonal entries for every bus, so isolated buses still appear
    rows = np.concatenate([rows, np.arange(n_bus)])
    cols = np.concatenate([cols, np.arange(n_bus)])
    Gv = np.concatenate([Gv, np.zeros(n_bus)])
    Bv = np.concatenate([Bv, np.zeros(n_bus)])
    Gm = coo_matrix((Gv, (rows, cols)), shape=(n_bus, n_bus)).tocsr()
    Bm = coo_matrix((Bv, (rows, cols)), shape=(n_bus, n_bus)).tocsr()
    Gm.sum_duplicates()
    Bm.sum_duplicates()
    Gc, Bc = Gm.tocoo(), Bm.tocoo()
    return Gc.row, Gc.col, Gc.data, Bc.data


def mismatch(ybus, P_sched, Q_sched, theta, V):
    """dP_i and dQ_i of eq. (1) (and its reactive counterpart), all buses.

    dP_i = P_is - |V_i| sum_j |V_j| (G_ij cos th_ij + B_ij sin th_ij)
    dQ_i = Q_is - |V_i| sum_j |V_j| (G_ij sin th_ij - B_ij cos th_ij)
    with th_ij = th_i - th_j; the j = i term is the self term |V_i|^2 G_ii of
    eq. (2) (and -|V_i|^2 B_ii for Q).
    """
    row, col, Gv, Bv = ybus
    n = V.shape[0]
    th = theta[row] - theta[col]
    c, s = np.cos(th), np.sin(th)
    vv = V[row] * V[col]
    P = np.bincount(row, weights=vv * (Gv * c + Bv * s), minlength=n)
    Q = np.bincount(row, weights=vv * (Gv * s - Bv * c), minlength=n)
    return P_sched - P, Q_sched - Q


def laplacian(n_bus, f, t, w, in_service, keep):
    """Weighted Laplacian of the in-service branches, rows/cols ``keep``."""
    on = np.asarray(in_service, dtype=bool)
    f, t, w = f[on], t[on], w[on]
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([w, w, -w, -w])
    L = coo_matrix((vals, (rows, cols)), shape=(n_bus, n_bus)).tocsr()
    L.sum_duplicates()
    return L[keep][:, keep].tocsc()


def bprime(n_bus, f, t, x, in_service, keep):
    """B' (eq. (4)): branch weights 1/x."""
    return laplacian(n_bus, f, t, 1.0 / x, in_service, keep)


def bdprime(n_bus, f, t, r, x, in_service, keep, tap=None):
    """B'' (eq. (5)): branch terms w v v^T, w = x/(r^2+x^2), v = e_i/tau - e_j
    (charging excluded)."""
    on = np.asarray(in_service, dtype=bool)
    c = tap_factor(tap, len(f))[on]
    w = (x / (r * r + x * x))[on]
    f, t = f[on], t[on]
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([c * c * w, w, -c * w, -c * w])
    L = coo_matrix((vals, (rows, cols)), shape=(n_bus, n_bus)).tocsr()
    L.sum_duplicates()
    return L[keep][:, keep].tocsc()


class DirectSolver:
    """Full factorisation of one matrix, reused for every right-hand side."""

    def __init__(self, A):
        self.n = A.shape[0]
        if self.n == 0:
            self.kind = "empty"
        elif self.n <= DENSE_MAX:
            self.kind = "dense"
            self.lu = sla.lu_factor(A.toarray())
        else:
            self.kind = "sparse"
            self.lu = splu(csc_matrix(A))

    def solve(self, b):
        if self.kind == "empty":
            return b.copy()
        if self.kind == "dense":
            return sla.lu_solve(self.lu, b)
        return self.lu.solve(b)


def branch_flows(f, t, r, x, in_service, theta, V, tap=None):
    """Active power at both ends of every branch (zero when out of service).

    P_ij = c^2 V_i^2 g - c V_i V_j (g cos th_ij + b_y sin th_ij),
    P_ji = V_j^2 g - c V_i V_j (g cos th_ij - b_y sin th_ij),  c = 1/tau.
    """
    c = tap_factor(tap, len(f))
    g, b = series_admittance(r, x)
    th = theta[f] - theta[t]
    Vf, Vt = V[f], V[t]
    Pf = c * c * Vf * Vf * g - c * Vf * Vt * (g * np.cos(th) + b * np.sin(th))
    Pt = Vt * Vt * g - c * Vf * Vt * (g * np.cos(th) - b * np.sin(th))
    on = np.asarray(in_service, dtype=bool)
    return np.where(on, Pf, 0.0), np.where(on, Pt, 0.0)


def limit_violations(cand, dQ, Q_min, Q_max):
    """PV buses ``cand`` whose generator output Q(V) - Q_sched = -dQ is above
    Q_max (first array) or below Q_min (second)."""
    qg = -dQ[cand]
    return cand[qg > Q_max[cand]], cand[qg < Q_min[cand]]


def returns_to_pv(held, V, V_set):
    """Buses held at a reactive limit (``held``: bus -> +1 at Q_max, -1 at
    Q_min) whose generator can hold the set point again, in bus order: |V|
    above the set point at Q_max (less reactive output would do), below it at
    Q_min."""
    return sorted(b for b, side in held.items()
                  if (side > 0 and V[b] > V_set[b]) or (side < 0 and V[b] < V_set[b]))


def fdpf(grid, in_service, active, P_sched, theta0, V0, tol, max_outer, growth_rule=True,
         switched=None, returned=None, held_count=None):
    """Fast-decoupled power flow on the buses marked ``active``.

    ``active`` excludes islanded buses (they keep theta = V = 0).  Returns
    (theta, V, outer_iterations, status, final_max_mismatch).  With reactive
    limits on the grid, the buses switched to PQ are appended to the list
    ``switched`` (when given) in the order they switched, lowest index first
    within one switch; the buses that turned back PV to ``returned``; and
    after every switch the number of buses then held at a limit to
    ``held_count``.
    """
    n = grid.n_bus
    bt = grid.bus_type.copy()
    Q_min, Q_max = getattr(grid, "Q_min", None), getattr(grid, "Q_max", None)
    qlim = Q_min is not None and Q_max is not None
    pvpq = np.flatnonzero(active & (bt != SLACK))
    pq = np.flatnonzero(active & (bt == PQ))
    on = np.asarray(in_service, dtype=bool)
    # a branch touching an inactive bus is not part of the main network
    on = on & active[grid.f] & active[grid.t]
    tap = getattr(grid, "tap", None)
    ybus = ybus_entries(n, grid.f, grid.t, grid.r, grid.x, grid.b_sh, on, tap)
    solP = DirectSolver(bprime(n, grid.f, grid.t, grid.x, on, pvpq))
    solQ = DirectSolver(bdprime(n, grid.f, grid.t, grid.r, grid.x, on, pq, tap))
    theta = np.where(active, theta0, 0.0).astype(np.float64)
    V = np.where(active, V0, 0.0).astype(np.float64)
    Q_sched = grid.Q_sched.astype(np.float64).copy()
    held = {}  # bus -> +1 held at Q_max, -1 held at Q_min
    k = 0
    best = np.inf
    while True:
        dP, dQ = mismatch(ybus, P_sched, Q_sched, theta, V)
        err = max(np.abs(dP[pvpq]).max(initial=0.0), np.abs(dQ[pq]).max(initial=0.0))
        if (not np.isfinite(err) or err > DIVERGE_LIMIT
                or (growth_rule and err > DIVERGE_GROWTH * best)):
            return theta, V, k, STATUS_DIVERGED, err
        best = min(best, err)
        if err <= tol:
            if qlim:
                hi, lo = limit_violations(np.flatnonzero(active & (bt == PV)), dQ, Q_min, Q_max)
                back = returns_to_pv(held, V, grid.V_set)
                if hi.size or lo.size or back:
                    for b in back:
                        bt[b] = PV
                        Q_sched[b] = grid.Q_sched[b]
                        V[b] = grid.V_set[b]
                        del held[b]
                    Q_sched[hi] += Q_max[hi]
                    Q_sched[lo] += Q_min[lo]
                    held.update({int(b): 1 for b in hi})
                    held.update({int(b): -1 for b in lo})
                    sw = np.sort(np.concatenate([hi, lo]))
                    bt[sw] = PQ
                    if switched is not None:
                        switched.extend(int(b) for b in sw)
                    if returned is not None:
                        returned.extend(back)
                    if held_count is not None:
                        held_count.append(len(held))
                    pq = np.flatnonzero(active & (bt == PQ))
                    solQ = DirectSolver(bdprime(n, grid.f, grid.t, grid.r, grid.x, on, pq, tap))
                    best = np.inf  # the switch raises the mismatch on purpose
                    continue
            return theta, V, k, STATUS_OK, err
        if k >= max_outer:
            return theta, V, k, STATUS_MAXITER, err
        if np.abs(dP[pvpq]).max(initial=0.0) > tol:
            theta[pvpq] += solP.solve(dP[pvpq] / V[pvpq])
            dP, dQ = mismatch(ybus, P_sched, Q_sched, theta, V)
        if np.abs(dQ[pq]).max(initial=0.0) > tol:
            V[pq] += solQ.solve(dQ[pq] / V[pq])
        k += 1


def base_case(grid, tol=1e-10, max_outer=100):
    """FDPF of the intact grid from a flat start (theta = 0, |V| = V_set).
    A flat start may pass through large mismatches on its way, so the growth
    rule for divergence is not applied here (only the absolute limit)."""
    n = grid.n_bus
    on = np.ones(grid.n_branch, dtype=bool)
    active = np.ones(n, dtype=bool)
    return fdpf(grid, on, active, grid.P_sched.astype(np.float64), np.zeros(n),
                grid.V_set.astype(np.float64), tol, max_outer, growth_rule=False)
