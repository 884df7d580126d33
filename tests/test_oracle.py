"""Pins of the CPU oracle against closed forms, invariants, brute force and
an independent Newton-Raphson solve (no GPU needed)."""
import itertools

import numpy as np
import pytest

from cases import load_case, random_tree_grid, grid_from_arrays
from gridgen import config_grid
from oracle import factor, islands, powerflow as pf, redispatch, screen


# ---------------------------------------------------------------- closed forms
def test_two_bus_closed_form():
    g, d = load_case("two_bus.json")
    th, V, k, st, err = pf.base_case(g, tol=1e-13)
    assert st == pf.STATUS_OK
    exp = -np.arcsin(0.8 * 0.25 / (1.03 * 0.98))
    assert abs(th[1] - exp) < 1e-12
    assert V[0] == 1.03 and V[1] == 0.98


def radial_angles(g, parent, in_service=None):
    """Exact angles of a lossless tree whose non-slack buses are all PV:
    the flow into each subtree is minus its summed injection (KCL) and
    P_pc = V_p V_c sin(th_p - th_c)/x (eq. (1) with G = 0)."""
    n = g.n_bus
    children = [[] for _ in range(n)]
    edge_x = {}
    for e in range(g.n_branch):
        if in_service is not None and not in_service[e]:
            continue
        a, b = int(g.f[e]), int(g.t[e])
        edge_x[(a, b)] = edge_x[(b, a)] = g.x[e]
    # orient from the slack by BFS
    root = g.slack
    order, par = [root], {root: -1}
    adj = {i: [] for i in range(n)}
    for (a, b) in edge_x:
        adj[a].append(b)
    for u in order:
        for v in adj[u]:
            if v not in par:
                par[v] = u
                order.append(v)
    sub = g.P_sched.astype(float).copy()
    for u in reversed(order[1:]):
        sub[par[u]] += sub[u]
    th = np.zeros(n)
    V = g.V_set
    for u in order[1:]:
        p = par[u]
        F = -sub[u]  # power flowing from p into the subtree of u
        th[u] = th[p] - np.arcsin(F * edge_x[(p, u)] / (V[p] * V[u]))
    return th


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_radial_closed_form(seed):
    g, parent = random_tree_grid(40, seed)
    th, V, k, st, err = pf.base_case(g, tol=1e-13)
    assert st == pf.STATUS_OK
    np.testing.assert_allclose(th, radial_angles(g, parent), rtol=0, atol=1e-11)


@pytest.mark.parametrize("l", range(5))
def test_ring_outage_becomes_radial(l):
    g, _ = load_case("five_bus_ring.json")
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-13)
    assert st == pf.STATUS_OK
    r = screen.solve_outage(g, th0, V0, l, tol=1e-13, max_outer=100)
    on = np.ones(g.n_branch, bool)
    on[l] = False
    assert r["status"] == pf.STATUS_OK and not r["islanded"]
    np.testing.assert_allclose(r["theta"], radial_angles(g, None, on), atol=1e-11)
    assert r["flow"][l] == 0.0


# ------------------------------------------------------- independent Newton
def newton_solution(g, tol=1e-13):
    """Newton-Raphson on S = V conj(Y V) (complex form, finite-difference
    Jacobian): an independent route to the AC fixed point."""
    n = g.n_bus
    Y = np.zeros((n, n), complex)
    for e in range(g.n_branch):
        i, j = int(g.f[e]), int(g.t[e])
        y = 1.0 / (g.r[e] + 1j * g.x[e])
        # an ideal transformer a:1 at the from end: the pi-model sees V_i / a
        # and passes I / a back to bus i
        a = 1.0 if g.tap is None else float(g.tap[e])
        Y[i, j] -= y / a
        Y[j, i] -= y / a
        Y[i, i] += (y + 0.5j * g.b_sh[e]) / (a * a)
        Y[j, j] += y + 0.5j * g.b_sh[e]
    pvpq = np.flatnonzero(g.bus_type != 2)
    pq = np.flatnonzero(g.bus_type == 0)

    def F(z, th, V):
        th = th.copy()
        V = V.copy()
        th[pvpq] = z[:len(pvpq)]
        V[pq] = z[len(pvpq):]
        Vc = V * np.exp(1j * th)
        S = Vc * np.conj(Y @ Vc)
        return np.r_[g.P_sched[pvpq] - S.real[pvpq], g.Q_sched[pq] - S.imag[pq]]

    th = np.zeros(n)
    V = g.V_set.astype(float).copy()
    z = np.r_[th[pvpq], V[pq]]
    for _ in range(50):
        r = F(z, th, V)
        if np.abs(r).max() < tol:
            break
        J = np.zeros((len(z), len(z)))
        h = 1e-7
        for c in range(len(z)):
            dz = np.zeros(len(z))
            dz[c] = h
            J[:, c] = (F(z + dz, th, V) - F(z - dz, th, V)) / (2 * h)
        z = z - np.linalg.solve(J, r)
    th[pvpq] = z[:len(pvpq)]
    V[pq] = z[len(pvpq):]
    return th, V


def test_lossy_case_matches_newton():
    g, _ = load_case("five_bus_lossy.json")
    th, V, k, st, err = pf.base_case(g, tol=1e-12)
    assert st == pf.STATUS_OK and k > 2
    thn, Vn = newton_solution(g)
    np.testing.assert_allclose(th, thn, atol=1e-10)
    np.testing.assert_allclose(V, Vn, atol=1e-10)


def test_tree_with_pq_and_losses_matches_newton():
    g, _ = random_tree_grid(12, 7, lossless=False, all_pv=False)
    th, V, k, st, err = pf.base_case(g, tol=1e-12)
    assert st == pf.STATUS_OK
    thn, Vn = newton_solution(g)
    np.testing.assert_allclose(th, thn, atol=1e-9)
    np.testing.assert_allclose(V, Vn, atol=1e-9)


def test_mismatch_zero_only_at_solution():
    g, _ = load_case("five_bus_lossy.json")
    thn, Vn = newton_solution(g)
    yb = pf.ybus_entries(g.n_bus, g.f, g.t, g.r, g.x, g.b_sh, np.ones(g.n_branch, bool))
    dP, dQ = pf.mismatch(yb, g.P_sched, g.Q_sched, thn, Vn)
    assert np.abs(dP[1:]).max() < 1e-11 and np.abs(dQ[g.bus_type == 0]).max() < 1e-11
    thp = thn.copy()
    thp[3] += 1e-3
    dP2, _ = pf.mismatch(yb, g.P_sched, g.Q_sched, thp, Vn)
    assert np.abs(dP2[1:]).max() > 1e-3


# ------------------------------------- transformer turns ratios (Sec. II.B)
@pytest.mark.parametrize("flip", [False, True])
def test_two_bus_tap_closed_form(flip):
    """The tap's side does not matter for the angle: P = V_1 V_2 sin/(tau x)."""
    g, d = load_case("two_bus_tap.json")
    if flip:
        g.f, g.t = g.t.copy(), g.f.copy()
    th, V, k, st, err = pf.base_case(g, tol=1e-13)
    assert st == pf.STATUS_OK
    assert abs(th[1] + np.arcsin(0.8 * 0.25 * 1.05 / (1.03 * 0.98))) < 1e-12


def test_two_bus_tap_voltage_closed_form():
    """A PQ bus behind a tap: the quadratic of Q_2 = (V_2^2 - V_1 V_2/tau)/x,
    and with the tap on the PQ side V_2 scales by tau."""
    g, d = load_case("two_bus_tap_pq.json")
    th, V, k, st, err = pf.base_case(g, tol=1e-13)
    assert st == pf.STATUS_OK
    a, q, x, v1 = 0.97, -0.3, 0.2, 1.02
    assert abs(V[1] - (v1 / a + np.sqrt((v1 / a) ** 2 + 4 * q * x)) / 2) < 1e-12
    assert abs(th[1]) < 1e-13
    g.f, g.t = g.t.copy(), g.f.copy()
    th, V, k, st, err = pf.base_case(g, tol=1e-13)
    assert st == pf.STATUS_OK
    assert abs(V[1] - a * (v1 + np.sqrt(v1 * v1 + 4 * q * x)) / 2) < 1e-12


def _with_taps(g, seed, frac=0.5):
    rng = np.random.default_rng(seed)
    g = g.copy()
    g.tap = np.where(rng.uniform(size=g.n_branch) < frac,
                     rng.uniform(0.9, 1.1, g.n_branch), 1.0)
    return g


@pytest.mark.parametrize("seed", [0, 1])
def test_tapped_lossy_cases_match_newton(seed):
    g0, _ = load_case("five_bus_lossy.json")
    for g in (_with_taps(g0, seed), _with_taps(random_tree_grid(12, 7 + seed, lossless=False,
                                                                all_pv=False)[0], seed)):
        th, V, k, st, err = pf.base_case(g, tol=1e-12)
        assert st == pf.STATUS_OK
        thn, Vn = newton_solution(g)
        np.testing.assert_allclose(th, thn, atol=1e-9)
        np.testing.assert_allclose(V, Vn, atol=1e-9)


def test_unit_taps_change_nothing():
    g = config_grid("grid120")
    gt = g.copy()
    gt.tap = np.ones(g.n_branch)
    a = pf.base_case(g)
    b = pf.base_case(gt)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_tapped_bdprime_is_minus_imag_ybus():
    """With r = 0 and no charging, B'' is minus the imaginary part of the bus
    admittance matrix (turns ratios included) on the PQ buses."""
    g, _ = random_tree_grid(15, 4, lossless=True, all_pv=False)
    g = _with_taps(g, 9, frac=0.7)
    on = np.ones(g.n_branch, bool)
    keep = np.flatnonzero(g.bus_type == 0)
    row, col, Gv, Bv = pf.ybus_entries(g.n_bus, g.f, g.t, g.r, g.x, g.b_sh, on, g.tap)
    B = np.zeros((g.n_bus, g.n_bus))
    np.add.at(B, (row, col), Bv)
    Bpp = pf.bdprime(g.n_bus, g.f, g.t, g.r, g.x, on, keep, g.tap).toarray()
    np.testing.assert_allclose(Bpp, -B[np.ix_(keep, keep)], rtol=1e-14, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(Bpp) > 0)


def test_tapped_n1_kcl_and_power_balance():
    """Flows at both ends (branch_flows, taps included) against the
    mismatch's bus injections (ybus_entries): Kirchhoff's law per bus and
    the power balance, on every outage of a grid with 15 % transformers."""
    from gridgen import make_grid
    g = make_grid(120, 180, seed=1, load_scale=0.3, xfmr_frac=0.15)
    th0, V0, _, st, _ = pf.base_case(g)
    assert st == pf.STATUS_OK
    res = screen.n1_screen(g, th0, V0, np.arange(g.n_branch), tol=1e-10, processes=1)
    ok = 0
    for s in range(g.n_branch):
        if res["status"][s] != pf.STATUS_OK:
            continue
        on, label, isl, P, _ = screen.outage_setup(g, s)
        net = np.zeros(g.n_bus)
        np.add.at(net, g.f, res["flow"][s])
        np.add.at(net, g.t, res["flow_to"][s])
        nonslack = ~isl & (g.bus_type != 2)
        assert np.abs(net[nonslack] - P[nonslack]).max() < 1e-9
        losses = (res["flow"][s] + res["flow_to"][s]).sum()
        assert abs(P[nonslack].sum() + net[g.slack] - losses) < 1e-9
        ok += 1
    assert ok > 0.9 * g.n_branch


# ------------------------------------------- generator outages (Sec. IV.A)
def test_two_bus_generator_trip_closed_form():
    g, d = load_case("two_bus_gen_trip.json")
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-13)
    assert st == pf.STATUS_OK and V0[1] == 1.0
    r = screen.solve_generator_outage(g, th0, V0, 1, tol=1e-13, max_outer=100)
    # converged; the slack took the lost generation (no other generator)
    assert r["status"] == pf.STATUS_ISLAND_NO_GEN
    v1, x, pd, qd = 1.02, 0.2, 0.5, 0.2
    a = v1 * v1 - 2 * qd * x
    V2 = np.sqrt((a + np.sqrt(a * a - 4 * x * x * (pd * pd + qd * qd))) / 2)
    assert abs(r["V"][1] - V2) < 1e-12
    assert abs(r["theta"][1] + np.arcsin(pd * x / (v1 * V2))) < 1e-12
    assert abs(r["flow"][0] - pd) < 1e-12   # the line carries the load


@pytest.mark.parametrize("seed", [3, 8])
def test_generator_trip_matches_newton(seed):
    """The tripped bus as PQ with its load, the rest of the generation
    scaled up by hand: Newton on that grid reaches the same state."""
    g, _ = random_tree_grid(14, seed, lossless=False, all_pv=False)
    g.P_gen = np.where(g.bus_type == 1, np.abs(g.P_sched) + 0.2, 0.0)
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-12)
    assert st == pf.STATUS_OK
    pv = np.flatnonzero(g.bus_type == 1)
    for k in pv[:3]:
        r = screen.solve_generator_outage(g, th0, V0, int(k), tol=1e-12, max_outer=200)
        assert r["status"] in (pf.STATUS_OK, pf.STATUS_ISLAND_NO_GEN)
        h = g.copy()
        h.bus_type = g.bus_type.copy()
        h.bus_type[k] = 0
        others = [j for j in pv if j != k]
        h.P_sched = g.P_sched.copy()
        h.P_sched[k] -= g.P_gen[k]
        tot = sum(g.P_gen[j] for j in others)
        for j in others:
            h.P_sched[j] += g.P_gen[k] * g.P_gen[j] / tot
        thn, Vn = newton_solution(h)
        np.testing.assert_allclose(r["theta"], thn, atol=1e-9)
        np.testing.assert_allclose(r["V"], Vn, atol=1e-9)


def test_generator_outages_kcl_and_balance():
    g = config_grid("grid120")
    th0, V0, _, st, _ = pf.base_case(g)
    pv = np.flatnonzero(g.bus_type == 1)
    res = screen.n1_screen(g, th0, V0, pv, tol=1e-10, processes=1, kind="generator")
    assert np.all(res["status"] == pf.STATUS_OK)
    for s, k in enumerate(pv):
        h, no_gen = screen.generator_setup(g, int(k))
        assert not no_gen
        nonslack = g.bus_type != 2
        # the lost generation is taken up in full by the other generators
        assert abs(h.P_sched[nonslack].sum() - g.P_sched[nonslack].sum()) < 1e-12
        net = np.zeros(g.n_bus)
        np.add.at(net, g.f, res["flow"][s])
        np.add.at(net, g.t, res["flow_to"][s])
        assert np.abs(net[nonslack] - h.P_sched[nonslack]).max() < 1e-9
        # the tripped bus no longer holds its set point
        assert abs(res["V"][s][k] - g.V_set[k]) > 1e-6


# -------------------------------------------- reactive limits of PV buses
def test_two_bus_q_limit_closed_form():
    g, d = load_case("two_bus_qlim.json")
    sw = []
    th, V, k, st, err = pf.fdpf(g, np.ones(1, bool), np.ones(2, bool), g.P_sched,
                                np.zeros(2), g.V_set.astype(float), 1e-13, 100, False, sw)
    assert st == pf.STATUS_OK and sw == [1]
    v1, x, pc, qc = 1.0, 0.2, 0.3, -0.1        # P, Q consumed at bus 2 after the switch
    a = v1 * v1 - 2 * qc * x
    V2 = np.sqrt((a + np.sqrt(a * a - 4 * x * x * (pc * pc + qc * qc))) / 2)
    assert abs(V[1] - V2) < 1e-12
    assert abs(th[1] + np.arcsin(pc * x / (v1 * V2))) < 1e-12
    # without the limit the bus holds its set point
    g.Q_max = None
    th2, V2b, _, st2, _ = pf.base_case(g, tol=1e-13)
    assert st2 == pf.STATUS_OK and V2b[1] == 1.05


def test_q_limit_lower_bound_and_no_switch():
    """A limit that is never reached changes nothing; a lower limit above the
    needed output holds the generator at Q_min."""
    g, _ = load_case("two_bus_qlim.json")
    g.Q_max = np.array([0.0, 5.0])
    free = g.copy()
    free.Q_min = free.Q_max = None
    ref = pf.base_case(free, tol=1e-13)
    got = pf.base_case(g, tol=1e-13)
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    g.Q_min = np.array([0.0, 0.5])               # more than the ~0.37 the set point needs
    sw = []
    th, V, k, st, err = pf.fdpf(g, np.ones(1, bool), np.ones(2, bool), g.P_sched,
                                np.zeros(2), g.V_set.astype(float), 1e-13, 100, False, sw)
    assert st == pf.STATUS_OK and sw == [1] and V[1] > 1.05
    yb = pf.ybus_entries(2, g.f, g.t, g.r, g.x, g.b_sh, np.ones(1, bool))
    dP, dQ = pf.mismatch(yb, g.P_sched, g.Q_sched, th, V)
    assert abs(-dQ[1] - 0.5) < 1e-11             # the generator sits at Q_min


@pytest.mark.parametrize("seed", [2, 6])
def test_q_limits_match_newton_and_hold(seed):
    """On a lossy tree with tight limits: every PV bus left is within its
    limits at the result, every switched one is at a limit, and Newton on the
    grid with those buses turned PQ at their limits reaches the same state."""
    g, _ = random_tree_grid(14, seed, lossless=False, all_pv=False)
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-12)
    yb = pf.ybus_entries(g.n_bus, g.f, g.t, g.r, g.x, g.b_sh, np.ones(g.n_branch, bool))
    dP, dQ = pf.mismatch(yb, g.P_sched, g.Q_sched, th0, V0)
    pv = np.flatnonzero(g.bus_type == 1)
    qg = -dQ[pv]
    g.Q_min = np.full(g.n_bus, -10.0)
    g.Q_max = np.full(g.n_bus, 10.0)
    g.Q_max[pv] = qg - 0.02 - 0.05 * np.abs(qg)  # every generator a little short
    g.Q_min[pv] = qg - 1.0
    sw = []
    th, V, k, st, err = pf.fdpf(g, np.ones(g.n_branch, bool), np.ones(g.n_bus, bool),
                                g.P_sched, np.zeros(g.n_bus), g.V_set.astype(float), 1e-12,
                                200, False, sw)
    assert st == pf.STATUS_OK and len(sw) > 0
    dP, dQ = pf.mismatch(yb, g.P_sched, g.Q_sched, th, V)
    left = np.setdiff1d(pv, sw)
    assert np.all(-dQ[left] <= g.Q_max[left] + 1e-9) and np.all(-dQ[left] >= g.Q_min[left] - 1e-9)
    h = g.copy()
    h.bus_type = g.bus_type.copy()
    h.Q_sched = g.Q_sched.copy()
    for b in sw:
        h.bus_type[b] = 0
        h.Q_sched[b] += g.Q_max[b]             # all switched at Q_max here
    h.Q_min = h.Q_max = None
    thn, Vn = newton_solution(h)
    np.testing.assert_allclose(th, thn, atol=1e-9)
    np.testing.assert_allclose(V, Vn, atol=1e-9)


def limit_complementarity(name, kind="branch"):
    """Every N-1 scenario of a grid with reactive limits, in process (so that
    a rule replaced in this process is the one used).  At each converged
    state, for every PV generator of the main island (Q_g = Q(V) - Q_sched,
    the output it needs): one still at its set point is within [Q_min, Q_max];
    one off its set point is held at a limit, at Q_max only with |V| at or
    below the set point and at Q_min only at or above it.  These are the
    conditions under which no generator can switch either way.  Returns the
    oracle's screen result."""
    from gpu_common import grid, oracle_base
    g = grid(name)
    th0, V0 = oracle_base(name)
    units = (np.arange(g.n_branch) if kind == "branch"
             else np.flatnonzero(g.bus_type == 1)).astype(np.int32)
    res = screen.n1_screen(g, th0, V0, units, tol=1e-10, max_outer=100, processes=1,
                           kind="generator" if kind != "branch" else "branch")
    for s in np.flatnonzero(res["status"] == pf.STATUS_OK):
        if kind == "branch":
            on, _, isl, P, _ = screen.outage_setup(g, int(units[s]))
            h = g
        else:
            h, _ = screen.generator_setup(g, int(units[s]))
            on, isl, P = np.ones(g.n_branch, bool), np.zeros(g.n_bus, bool), h.P_sched
        live = on & ~isl[g.f] & ~isl[g.t]
        yb = pf.ybus_entries(g.n_bus, g.f, g.t, g.r, g.x, g.b_sh, live, g.tap)
        th, V = res["theta"][s], res["V"][s]
        _, dQ = pf.mismatch(yb, P, g.Q_sched, th, V)
        qg = -dQ
        for b in np.flatnonzero((h.bus_type == 1) & ~isl):
            if abs(V[b] - g.V_set[b]) <= 1e-9:
                assert g.Q_min[b] - 1e-8 <= qg[b] <= g.Q_max[b] + 1e-8, (s, b)
            elif abs(qg[b] - g.Q_max[b]) <= 1e-8:
                assert V[b] <= g.V_set[b] + 1e-12, (s, b, "held at Q_max above its set point")
            else:
                assert abs(qg[b] - g.Q_min[b]) <= 1e-8, (s, b, "off its set point, at no limit")
                assert V[b] >= g.V_set[b] - 1e-12, (s, b, "held at Q_min below its set point")
    return res


def test_limit_complementarity_every_outage_grid120():
    """Branch outages of grid120 with reactive limits: enough converge, some
    generator turns back PV on the way, and every converged state meets the
    switching conditions."""
    res = limit_complementarity("grid120_qlim")
    ok = res["status"] == pf.STATUS_OK
    assert ok.sum() >= 0.9 * ok.size
    assert (ok & (res["n_returned"] > 0)).sum() >= 1
    assert (ok & (res["n_switched"] > 0)).sum() >= 10


def test_limit_complementarity_generator_outages_grid120():
    res = limit_complementarity("grid120_qlim", kind="generator")
    assert (res["status"] == pf.STATUS_OK).sum() >= 8


# ----------------------------------------------- outage algebra (Sec. IV.B)
def test_sherman_morrison_first_solve():
    """B'_s = B' - b a a^T (a = e_i - e_j): the solve with the re-formed
    contingency matrix equals the rank-one update of the base solve."""
    g = config_grid("grid120")
    n = g.n_bus
    keep = np.flatnonzero(g.bus_type != 2)
    pos = -np.ones(n, int)
    pos[keep] = np.arange(keep.size)
    on = np.ones(g.n_branch, bool)
    B0 = pf.bprime(n, g.f, g.t, g.x, on, keep).toarray()
    rng = np.random.default_rng(3)
    c = rng.standard_normal(keep.size)
    base = np.linalg.solve(B0, c)
    lab0 = islands.components(n, g.f, g.t, on)
    tested = 0
    for l in range(g.n_branch):
        on_l = on.copy()
        on_l[l] = False
        if (islands.components(n, g.f, g.t, on_l) != lab0).any():
            continue  # bridge: B'_s singular on the full bus set
        a = np.zeros(keep.size)
        if pos[g.f[l]] >= 0:
            a[pos[g.f[l]]] = 1.0
        if pos[g.t[l]] >= 0:
            a[pos[g.t[l]]] = -1.0
        b = 1.0 / g.x[l]
        Ba = np.linalg.solve(B0, a)
        sm = base + b * (a @ base) / (1.0 - b * (a @ Ba)) * Ba
        Bs = pf.bprime(n, g.f, g.t, g.x, on_l, keep)
        got = pf.DirectSolver(Bs).solve(c)
        np.testing.assert_allclose(got, sm, rtol=1e-9, atol=1e-9 * np.abs(sm).max())
        tested += 1
    assert tested > 100


def test_bridge_iff_ptdf_one():
    """PTDF_ll = b_l a^T B'^{-1} a equals 1 exactly for bridges (the
    Sherman-Morrison denominator vanishes: the contingency matrix of Table I's
    'LU failure' cases is singular)."""
    g = config_grid("grid120")
    n = g.n_bus
    keep = np.flatnonzero(g.bus_type != 2)
    pos = -np.ones(n, int)
    pos[keep] = np.arange(keep.size)
    on = np.ones(g.n_branch, bool)
    B0 = pf.bprime(n, g.f, g.t, g.x, on, keep).toarray()
    Binv = np.linalg.inv(B0)
    n_bridge = 0
    for l in range(g.n_branch):
        a = np.zeros(keep.size)
        if pos[g.f[l]] >= 0:
            a[pos[g.f[l]]] = 1.0
        if pos[g.t[l]] >= 0:
            a[pos[g.t[l]]] = -1.0
        ptdf = a @ Binv @ a / g.x[l]
        on_l = on.copy()
        on_l[l] = False
        bridge = len(set(islands.components(n, g.f, g.t, on_l))) > 1
        n_bridge += bridge
        if bridge:
            assert abs(ptdf - 1.0) < 1e-9
        else:
            assert ptdf < 1.0 - 1e-6
    assert n_bridge > 0


def test_bridge_outage_schur_complement_is_main_island_bprime():
    """For a bridge outage, the base-case B' inverted and restricted to the
    main island equals the inverse of the post-outage B' of the main island
    (the island's Laplacian annihilates the all-ones vector, so the Schur
    complement of the island block removes exactly the bridge's diagonal
    term): the base-case factor is an exact preconditioner for the P-theta
    system of every islanding outage (Sec. IV.B eq. (6), Sec. IV.C)."""
    g = config_grid("grid120")
    n = g.n_bus
    keep = np.flatnonzero(g.bus_type != 2)
    pos = -np.ones(n, int)
    pos[keep] = np.arange(keep.size)
    on = np.ones(g.n_branch, bool)
    Binv = np.linalg.inv(pf.bprime(n, g.f, g.t, g.x, on, keep).toarray())
    checked = 0
    for l in range(g.n_branch):
        on_l, label, isl, _, _ = screen.outage_setup(g, l)
        if not isl.any():
            continue
        main = np.flatnonzero(~isl & (g.bus_type != 2))
        Bs = pf.bprime(n, g.f, g.t, g.x, on_l, main).toarray()
        sub = Binv[np.ix_(pos[main], pos[main])]
        np.testing.assert_allclose(sub @ Bs, np.eye(main.size), rtol=0, atol=1e-9)
        checked += 1
    assert checked > 0


def test_four_element_difference():
    """Sec. IV.B: an outage changes exactly A_ii, A_jj, A_ij, A_ji of B'
    (fewer when an endpoint is the slack; B'' only at PQ endpoints)."""
    g = config_grid("grid120")
    n = g.n_bus
    on = np.ones(g.n_branch, bool)
    keepP = np.flatnonzero(g.bus_type != 2)
    keepQ = np.flatnonzero(g.bus_type == 0)
    P0 = pf.bprime(n, g.f, g.t, g.x, on, keepP).toarray()
    Q0 = pf.bdprime(n, g.f, g.t, g.r, g.x, on, keepQ).toarray()
    for l in range(g.n_branch):
        on_l = on.copy()
        on_l[l] = False
        dP = pf.bprime(n, g.f, g.t, g.x, on_l, keepP).toarray() - P0
        dQ = pf.bdprime(n, g.f, g.t, g.r, g.x, on_l, keepQ).toarray() - Q0
        endsP = sum(int(g.bus_type[b] != 2) for b in (g.f[l], g.t[l]))
        endsQ = sum(int(g.bus_type[b] == 0) for b in (g.f[l], g.t[l]))
        assert np.count_nonzero(np.abs(dP) > 1e-12) == endsP ** 2
        assert np.count_nonzero(np.abs(dQ) > 1e-12) == endsQ ** 2


# ------------------------------------------------------- islands (Sec. IV.C)
def closure_labels(n, f, t, on):
    R = np.eye(n, dtype=bool)
    for e in range(len(f)):
        if on[e]:
            R[f[e], t[e]] = R[t[e], f[e]] = True
    for k in range(n):  # Warshall
        R = R | (R[:, [k]] & R[[k], :])
    return np.array([int(np.flatnonzero(R[i])[0]) for i in range(n)])


@pytest.mark.parametrize("seed", range(6))
def test_islands_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 11))
    # random connected graph: a tree plus a few chords
    f = [int(rng.integers(0, i)) for i in range(1, n)]
    t = list(range(1, n))
    for _ in range(int(rng.integers(0, n))):
        a, b = sorted(rng.choice(n, 2, replace=False))
        if (a, b) not in set(zip(f, t)) and (b, a) not in set(zip(f, t)):
            f.append(int(a))
            t.append(int(b))
    f, t = np.array(f), np.array(t)
    for l in range(len(f)):
        on = np.ones(len(f), bool)
        on[l] = False
        np.testing.assert_array_equal(islands.components(n, f, t, on),
                                      closure_labels(n, f, t, on))


# ---------------------------------------------- invariants on full N-1 runs
@pytest.fixture(scope="module")
def grid120_n1():
    g = config_grid("grid120")
    th0, V0, _, st, _ = pf.base_case(g)
    assert st == pf.STATUS_OK
    res = screen.n1_screen(g, th0, V0, np.arange(g.n_branch), tol=1e-10, processes=1)
    return g, res


def test_n1_kcl_and_power_balance(grid120_n1):
    g, res = grid120_n1
    n = g.n_bus
    ok = 0
    for s in range(g.n_branch):
        if res["status"][s] not in (pf.STATUS_OK, pf.STATUS_ISLAND_NO_GEN):
            continue
        on, label, isl, P, _ = screen.outage_setup(g, s)
        net = np.zeros(n)
        np.add.at(net, g.f, res["flow"][s])
        np.add.at(net, g.t, res["flow_to"][s])
        main = ~isl
        nonslack = main & (g.bus_type != 2)
        # KCL: the flows leaving a bus add up to its scheduled injection
        assert np.abs(net[nonslack] - P[nonslack]).max() < 1e-9
        # power balance: all injections = losses (sum of both-end flows)
        losses = (res["flow"][s] + res["flow_to"][s]).sum()
        slack_inj = net[g.slack]
        assert abs(P[nonslack].sum() + slack_inj - losses) < 1e-9
        assert np.all(res["theta"][s][isl] == 0) and np.all(res["V"][s][isl] == 0)
        ok += 1
    assert ok > 0.9 * g.n_branch


def test_n1_islanding_handled(grid120_n1):
    g, res = grid120_n1
    isl = res["islanded"]
    assert isl.any() and (~isl).any()
    # every islanding scenario is solved after re-dispatch (Table I claim)
    assert np.all(np.isin(res["status"][isl], [pf.STATUS_OK, pf.STATUS_ISLAND_NO_GEN]))


def test_redispatch_conserves_main_island_injection():
    g = config_grid("grid2k")
    on = np.ones(g.n_branch, bool)
    seen = 0
    for l in range(g.n_branch):
        on_l = on.copy()
        on_l[l] = False
        lab = islands.components(g.n_bus, g.f, g.t, on_l)
        isl = islands.island_mask(lab, g.slack)
        if not isl.any():
            continue
        P, no_gen = redispatch.redispatch(g.bus_type, g.P_sched, g.P_gen, isl)
        if not no_gen:
            assert abs(P[~isl].sum() - g.P_sched.sum()) < 1e-9
        assert np.all(P[isl] == 0)
        seen += 1
        if seen > 40:
            break
    assert seen > 0


@pytest.mark.parametrize("name", ["grid120", "grid2k", "grid10k", "grid50k"])
def test_base_case_converges(name):
    g = config_grid(name)
    th, V, k, st, err = pf.base_case(g)
    assert st == pf.STATUS_OK and err <= 1e-10


# -------------------------------------------- incomplete Cholesky (eq. (6))
def _lower_pattern(A):
    A = A.tocsr()
    return [sorted(int(c) for c in A.indices[A.indptr[i]:A.indptr[i + 1]] if c <= i)
            for i in range(A.shape[0])]


def test_ic0_reproduces_a_on_pattern():
    g = config_grid("grid120")
    keep = np.flatnonzero(g.bus_type != 2)
    A = pf.bprime(g.n_bus, g.f, g.t, g.x, np.ones(g.n_branch, bool), keep)
    pat = _lower_pattern(A)
    L = factor.ic_on_pattern(A, pat)
    Ld = factor.to_dense(L, A.shape[0])
    Ad = A.toarray()
    LLt = Ld @ Ld.T
    for i, row in enumerate(pat):
        for j in row:
            assert abs(LLt[i, j] - Ad[i, j]) < 1e-10 * abs(Ad[i, i])
    assert np.all(np.diag(Ld) > 0)


def test_ic0_exact_on_tree_and_full_pattern():
    g, _ = random_tree_grid(30, 4, lossless=False, all_pv=True)
    keep = np.flatnonzero(g.bus_type != 2)
    A = pf.bprime(g.n_bus, g.f, g.t, g.x, np.ones(g.n_branch, bool), keep)
    # leaves-first ordering of a tree: IC(0) drops no fill
    depth = np.zeros(g.n_bus, int)
    for e in range(g.n_branch):
        depth[g.t[e]] = depth[g.f[e]] + 1
    order = np.argsort(-depth[keep], kind="stable")
    Ao = A[order][:, order]
    L = factor.to_dense(factor.ic_on_pattern(Ao, _lower_pattern(Ao)), Ao.shape[0])
    np.testing.assert_allclose(L, np.linalg.cholesky(Ao.toarray()), atol=1e-12)
    # meshed matrix: IC on the full symbolic pattern is the exact factor
    m = config_grid("grid120")
    keep = np.flatnonzero(m.bus_type != 2)
    A = pf.bprime(m.n_bus, m.f, m.t, m.x, np.ones(m.n_branch, bool), keep)
    full = factor.symbolic_cholesky(A.shape[0], _lower_pattern(A))
    L = factor.to_dense(factor.ic_on_pattern(A, full), A.shape[0])
    Lc = np.linalg.cholesky(A.toarray())
    np.testing.assert_allclose(L, Lc, atol=1e-10)
    # and the symbolic pattern holds every nonzero of the dense factor
    mask = np.zeros_like(Lc, bool)
    for i, row in enumerate(full):
        mask[i, row] = True
    assert np.abs(Lc[~mask]).max() < 1e-12


def test_triangular_solves_invert():
    rng = np.random.default_rng(0)
    n = 25
    M = np.tril(rng.uniform(-1, 1, (n, n)) * (rng.uniform(size=(n, n)) < 0.3))
    M[np.diag_indices(n)] = rng.uniform(1, 2, n)
    L = {i: {j: M[i, j] for j in range(i + 1) if M[i, j] != 0} for i in range(n)}
    r = rng.standard_normal(n)
    np.testing.assert_allclose(factor.forward(L, r), np.linalg.solve(M, r), atol=1e-12)
    np.testing.assert_allclose(factor.backward(L, r), np.linalg.solve(M.T, r), atol=1e-12)
    z = factor.apply_preconditioner(L, r)
    np.testing.assert_allclose(M @ (M.T @ z), r, atol=1e-10)


# -------------------------------------------------- adjoint (DC, eq. (4))
def _adjoint_case():
    g = config_grid("grid120")
    b = 1.0 / g.x
    # scale the injections so that some flows exceed their ratings and the
    # penalty has curvature
    P = g.P_sched * 8.0
    outages = np.arange(0, g.n_branch, 3)
    return g, P, b, outages


def _fd5(fun, x, i, h):
    """Five-point central difference d fun / d x_i (error O(h^4))."""
    def at(d):
        y = x.copy()
        y[i] += d
        return fun(y)
    return (-at(2 * h) + 8 * at(h) - 8 * at(-h) + at(-2 * h)) / (12 * h)


def test_adjoint_matches_central_differences():
    from oracle import adjoint
    g, P, b, outages = _adjoint_case()
    L, gP, gb = adjoint.loss_and_grad(g, outages, P, b)
    assert L > 0
    rng = np.random.default_rng(0)
    nonslack = np.flatnonzero(g.bus_type != 2)
    # h = 1e-6 (the plain central difference) is limited by the rounding of the
    # summed loss, about eps |L| / h; the five-point rule at h = 1e-4 brings
    # the check to 1e-6 relative
    for i in rng.choice(nonslack, 8, replace=False):
        fd = _fd5(lambda y: adjoint.loss_only(g, outages, y, b), P, i, 1e-4)
        assert abs(fd - gP[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gP[i])
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += 1e-6
        Pm[i] -= 1e-6
        fd6 = (adjoint.loss_only(g, outages, Pp, b) - adjoint.loss_only(g, outages, Pm, b)) / 2e-6
        assert abs(fd6 - gP[i]) <= 1e-6 * max(1.0, abs(fd6)) + 64 * np.finfo(float).eps * L / 1e-6
    for k in rng.choice(g.n_branch, 8, replace=False):
        fd = _fd5(lambda y: adjoint.loss_only(g, outages, P, y), b, k, 1e-4 * b[k])
        assert abs(fd - gb[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, gb[k])
    # the slack's injection does not enter the DC model
    assert gP[g.slack] == 0.0


def test_adjoint_dc_angles_match_sherman_morrison():
    """theta_s of the adjoint's forward model is the DC solve of the
    re-formed contingency matrix: check it against the rank-one update of
    the base solve for a non-bridge outage."""
    from oracle import adjoint
    g, P, b, _ = _adjoint_case()
    n = g.n_bus
    keep = np.flatnonzero(g.bus_type != 2)
    B0 = pf.bprime(n, g.f, g.t, g.x, np.ones(g.n_branch, bool), keep).toarray()
    th0 = np.linalg.solve(B0, P[keep])
    for l in range(g.n_branch):
        S = adjoint.scenario_setup(g, l, b)
        if S["isl"].any():
            continue
        a = np.zeros(n)
        a[g.f[l]] += 1.0
        a[g.t[l]] -= 1.0
        a = a[keep]
        Ba = np.linalg.solve(B0, a)
        sm = th0 + b[l] * (a @ th0) / (1 - b[l] * (a @ Ba)) * Ba
        th = adjoint._theta(g, P, S)[keep]
        np.testing.assert_allclose(th, sm, rtol=1e-9, atol=1e-12)
        break


# ------------------------------------------------------- DC quick screen
def _subtree_flows(g, in_service):
    """DC flows of a radial network by KCL alone: a branch carries the summed
    injection of the part of the tree beyond it (independent of x)."""
    n = g.n_bus
    adj = {i: [] for i in range(n)}
    for e in range(g.n_branch):
        if in_service[e]:
            adj[int(g.f[e])].append((int(g.t[e]), e))
            adj[int(g.t[e])].append((int(g.f[e]), e))
    order, par, pedge = [g.slack], {g.slack: -1}, {}
    for u in order:
        for v, e in adj[u]:
            if v not in par:
                par[v], pedge[v] = u, e
                order.append(v)
    sub = g.P_sched.astype(float).copy()
    for u in reversed(order[1:]):
        sub[par[u]] += sub[u]
    f = np.zeros(g.n_branch)
    for v, e in pedge.items():
        # flow from parent to child = net injection absorbed beyond the child
        f[e] = -sub[v] if int(g.t[e]) == v else sub[v]
    return f


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dc_radial_flows_are_subtree_injections(seed):
    """A tree plus one chord; outaging the chord leaves the tree, whose DC
    flows follow from KCL without any solve."""
    from oracle import dc
    g0, parent = random_tree_grid(30, seed)
    rng = np.random.default_rng(seed + 10)
    a, b = 0, 0
    while a == b or parent[a] == b or parent[b] == a:
        a, b = (int(v) for v in rng.integers(0, 30, 2))
    g = grid_from_arrays(g0.bus_type, g0.P_sched, g0.Q_sched, g0.P_gen, g0.V_set,
                         np.r_[g0.f, a], np.r_[g0.t, b], np.r_[g0.r, 0.0],
                         np.r_[g0.x, 0.1], np.r_[g0.b_sh, 0.0])
    chord = g.n_branch - 1
    r = dc.dc_screen(g, [chord])
    on = np.ones(g.n_branch, bool)
    on[chord] = False
    np.testing.assert_allclose(r["flow"][0], _subtree_flows(g, on), rtol=0, atol=1e-12)
    assert r["flow"][0][chord] == 0.0 and r["status"][0] == 0


def test_dc_lodf_matches_reformed_solves():
    """Non-bridge outages: post-outage flows = base flows + LODF x the outaged
    branch's base flow, LODF_kl = b_k a_k^T B'^-1 a_l / (1 - b_l a_l^T B'^-1 a_l)
    from the base matrix only (Sherman-Morrison)."""
    from oracle import dc
    g = config_grid("grid120")
    n, m = g.n_bus, g.n_branch
    keep = np.flatnonzero(g.bus_type != 2)
    pos = -np.ones(n, int)
    pos[keep] = np.arange(keep.size)
    on = np.ones(m, bool)
    B0 = pf.bprime(n, g.f, g.t, g.x, on, keep).toarray()
    Binv = np.linalg.inv(B0)
    A = np.zeros((m, keep.size))
    for k in range(m):
        if pos[g.f[k]] >= 0:
            A[k, pos[g.f[k]]] = 1.0
        if pos[g.t[k]] >= 0:
            A[k, pos[g.t[k]]] = -1.0
    bvec = 1.0 / g.x
    f0 = bvec * (A @ (Binv @ g.P_sched[keep]))
    lab0 = islands.components(n, g.f, g.t, on)
    outs = []
    for l in range(m):
        on_l = on.copy()
        on_l[l] = False
        if (islands.components(n, g.f, g.t, on_l) == lab0).all():
            outs.append(l)
    r = dc.dc_screen(g, outs)
    for s, l in enumerate(outs):
        ptdf = bvec * (A @ (Binv @ A[l]))
        lodf = ptdf / (1.0 - ptdf[l])
        exp = f0 + lodf * f0[l]
        exp[l] = 0.0
        np.testing.assert_allclose(r["flow"][s], exp, rtol=0, atol=1e-9)
    assert len(outs) > 100


def test_dc_islanding_balance():
    """Bridge outages: dead branches carry nothing, and on the main island
    the flows balance the re-dispatched injections at every non-slack bus
    (the islands' net injection moved onto main-island PV generation)."""
    from oracle import dc
    g = config_grid("grid120")
    n, m = g.n_bus, g.n_branch
    on = np.ones(m, bool)
    lab0 = islands.components(n, g.f, g.t, on)
    bridges = []
    for l in range(m):
        on_l = on.copy()
        on_l[l] = False
        if (islands.components(n, g.f, g.t, on_l) != lab0).any():
            bridges.append(l)
    r = dc.dc_screen(g, bridges)
    for s, l in enumerate(bridges):
        isl = r["label"][s] != r["label"][s][g.slack]
        live = np.ones(m, bool)
        live[l] = False
        live &= ~isl[g.f] & ~isl[g.t]
        assert np.all(r["flow"][s][~live] == 0.0)
        assert np.all(r["theta"][s][isl] == 0.0)
        net = np.zeros(n)
        np.add.at(net, g.f, r["flow"][s])
        np.add.at(net, g.t, -r["flow"][s])
        main = ~isl & (g.bus_type != 2)
        # the re-dispatch itself is pinned by the hand-derived ring below
        Pt, _ = redispatch.redispatch(g.bus_type, g.P_sched, g.P_gen, isl)
        np.testing.assert_allclose(net[main], Pt[main], rtol=0, atol=1e-10)
    assert len(bridges) > 5


# ------------------------------------------------------------ re-dispatch
def ring_case():
    """The hand-derived re-dispatch fixture (tests/golden/redispatch_ring.json)."""
    import json
    import os
    from cases import GOLDEN
    with open(os.path.join(GOLDEN, "redispatch_ring.json")) as fh:
        d = json.load(fh)
    gd = d["grid"]
    g = grid_from_arrays(gd["bus_type"], gd["P_sched"], gd["Q_sched"], gd["P_gen"],
                         gd["V_set"], gd["from"], gd["to"], gd["r"], gd["x"], gd["b_sh"],
                         gd["rating"])
    return g, d


def test_redispatch_hand_derived_ring():
    """Sec. IV.C's proportional re-dispatch against values worked out by hand
    on a ring with a spur: an exporting island (its surplus shared 2:1 by the
    two main generators; a PV bus with no scheduled generation takes no
    share), an importing island (three generators share the deficit), a ring
    outage that moves nothing, and a generator trip.  An equal-shares or
    sign-flipped rule fails these; the balance invariant alone would not."""
    g, d = ring_case()
    n = g.n_bus
    for case in d["branch_outages"]:
        on, label, isl, P, no_gen = screen.outage_setup(g, case["outage"])
        assert np.flatnonzero(isl).tolist() == case["islanded"]
        np.testing.assert_allclose(P, case["P_after"], rtol=0, atol=1e-15)
        assert no_gen == case["no_gen"]
        P2, ng2 = redispatch.redispatch(g.bus_type, g.P_sched, g.P_gen, isl)
        np.testing.assert_allclose(P2, case["P_after"], rtol=0, atol=1e-15)
    for case in d["generator_outages"]:
        g2, no_gen = screen.generator_setup(g, case["bus"])
        np.testing.assert_allclose(g2.P_sched, case["P_after"], rtol=0, atol=1e-15)
        assert no_gen == case["no_gen"]
    c = d["no_generator_case"]
    on = np.ones(len(c["from"]), bool)
    on[c["outage"]] = False
    lab = islands.components(len(c["bus_type"]), np.array(c["from"]), np.array(c["to"]), on)
    isl = islands.island_mask(lab, 0)
    assert np.flatnonzero(isl).tolist() == c["islanded"]
    P, no_gen = redispatch.redispatch(np.array(c["bus_type"], np.int8),
                                      np.array(c["P_sched"]), np.array(c["P_gen"]), isl)
    np.testing.assert_allclose(P, c["P_after"], rtol=0, atol=1e-15)
    assert no_gen is True
    assert n == 7


def test_redispatch_ring_power_flow_balance():
    """The ring's N-1 solutions carry the hand-derived injections: at every
    main-island bus but the slack, the FP64 mismatch against P_after vanishes
    (so the FDPF used the re-dispatched schedule, not the original)."""
    g, d = ring_case()
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-12, max_outer=200)
    assert st == pf.STATUS_OK
    for case in d["branch_outages"]:
        r = screen.solve_outage(g, th0, V0, case["outage"], 1e-12, 100)
        assert r["status"] == pf.STATUS_OK
        on = np.ones(g.n_branch, bool)
        on[case["outage"]] = False
        isl = np.zeros(g.n_bus, bool)
        isl[case["islanded"]] = True
        live = on & ~isl[g.f] & ~isl[g.t]
        yb = pf.ybus_entries(g.n_bus, g.f, g.t, g.r, g.x, g.b_sh, live)
        dP, _ = pf.mismatch(yb, np.array(case["P_after"]), g.Q_sched, r["theta"], r["V"])
        main = ~isl & (g.bus_type != 2)
        assert np.abs(dP[main]).max() <= 1e-11
