"""The oracle's pins catch plausible mistakes: each test plants one in the
oracle (on the CPU, through monkeypatch) and checks that the pin meant for
it fails."""
import numpy as np
import pytest
from scipy.sparse import coo_matrix

import test_oracle as pins
from oracle import powerflow as pf
from oracle import screen


def _ybus_tap_on_wrong_end(n_bus, f, t, r, x, b_sh, in_service, tap=None):
    """The tap's c^2 put on the to end instead of the from end."""
    on = np.asarray(in_service, dtype=bool)
    c = pf.tap_factor(tap, len(f))[on]
    f, t, r, x, b_sh = f[on], t[on], r[on], x[on], b_sh[on]
    g, b = pf.series_admittance(r, x)
    rows = np.concatenate([f, t, f, t, np.arange(n_bus)])
    cols = np.concatenate([t, f, f, t, np.arange(n_bus)])
    z = np.zeros(n_bus)
    Gv = np.concatenate([-c * g, -c * g, g, c * c * g, z])
    Bv = np.concatenate([-c * b, -c * b, b + 0.5 * b_sh, c * c * (b + 0.5 * b_sh), z])
    Gm = coo_matrix((Gv, (rows, cols)), shape=(n_bus, n_bus)).tocsr()
    Bm = coo_matrix((Bv, (rows, cols)), shape=(n_bus, n_bus)).tocsr()
    Gm.sum_duplicates()
    Bm.sum_duplicates()
    Gc, Bc = Gm.tocoo(), Bm.tocoo()
    return Gc.row, Gc.col, Gc.data, Bc.data


def test_tap_on_wrong_end_is_caught(monkeypatch):
    monkeypatch.setattr(pf, "ybus_entries", _ybus_tap_on_wrong_end)
    with pytest.raises(AssertionError):
        pins.test_two_bus_tap_voltage_closed_form()


def test_flow_tap_applied_once_is_caught(monkeypatch):
    right = pf.branch_flows

    def flows_c_once(f, t, r, x, in_service, theta, V, tap=None):
        Pf, Pt = right(f, t, r, x, in_service, theta, V, tap)
        if tap is None:
            return Pf, Pt
        c = pf.tap_factor(tap, len(f))
        g, _ = pf.series_admittance(r, x)
        on = np.asarray(in_service, dtype=bool)
        # c V_i^2 g instead of c^2 V_i^2 g at the from end
        return np.where(on, Pf + (c - c * c) * V[f] ** 2 * g, 0.0), Pt

    monkeypatch.setattr(screen, "branch_flows", flows_c_once)
    with pytest.raises(AssertionError):
        pins.test_tapped_n1_kcl_and_power_balance()


def test_tripped_bus_left_pv_is_caught(monkeypatch):
    right = screen.generator_setup

    def keeps_voltage(grid, k):
        g, no_gen = right(grid, k)
        g.bus_type = grid.bus_type.copy()  # the bus still holds its set point
        return g, no_gen

    monkeypatch.setattr(screen, "generator_setup", keeps_voltage)
    with pytest.raises(AssertionError):
        pins.test_two_bus_generator_trip_closed_form()


def test_generation_not_removed_is_caught(monkeypatch):
    right = screen.redispatch_generator

    def keeps_generation(bus_type, P_sched, P_gen, k):
        P, no_gen = right(bus_type, P_sched, P_gen, k)
        P[k] += P_gen[k]                   # the tripped generator still injects
        return P, no_gen

    monkeypatch.setattr(screen, "redispatch_generator", keeps_generation)
    with pytest.raises(AssertionError):
        pins.test_two_bus_generator_trip_closed_form()


def test_limit_sign_flipped_is_caught(monkeypatch):
    def flipped(cand, dQ, Q_min, Q_max):
        qg = dQ[cand]                      # Q_sched - Q(V) taken for the output
        return cand[qg > Q_max[cand]], cand[qg < Q_min[cand]]

    monkeypatch.setattr(pf, "limit_violations", flipped)
    with pytest.raises(AssertionError):
        pins.test_two_bus_q_limit_closed_form()



def test_return_to_pv_side_flipped_is_caught(monkeypatch):
    """A held generator sent back to PV on the wrong side of its set point
    (at Q_max when |V| is below it)."""
    def flipped(held, V, V_set):
        return sorted(b for b, side in held.items()
                      if (side > 0 and V[b] < V_set[b]) or (side < 0 and V[b] > V_set[b]))

    monkeypatch.setattr(pf, "returns_to_pv", flipped)
    with pytest.raises(AssertionError):
        pins.test_limit_complementarity_every_outage_grid120()


def test_no_return_to_pv_is_caught(monkeypatch):
    """Held generators never sent back to PV (the earlier rule)."""
    monkeypatch.setattr(pf, "returns_to_pv", lambda held, V, V_set: [])
    with pytest.raises(AssertionError):
        pins.test_limit_complementarity_every_outage_grid120()


def test_equal_shares_redispatch_is_caught(monkeypatch):
    """The island's power split equally over the main generators instead of
    in proportion to their scheduled generation."""
    from oracle import redispatch

    def equal_shares(bus_type, P_sched, P_gen, islanded):
        P = P_sched.astype(np.float64).copy()
        if not islanded.any():
            return P, False
        part = (bus_type == 1) & (~islanded) & (P_gen > 0.0)
        if not part.any():
            P[islanded] = 0.0
            return P, True
        P[part] += float(P_sched[islanded].sum()) / part.sum()
        P[islanded] = 0.0
        return P, False

    monkeypatch.setattr(screen, "redispatch", equal_shares)
    monkeypatch.setattr(redispatch, "redispatch", equal_shares)
    with pytest.raises(AssertionError):
        pins.test_redispatch_hand_derived_ring()


def test_redispatch_sign_flipped_is_caught(monkeypatch):
    """The island's net injection subtracted from the main generators."""
    from oracle import redispatch

    def flipped(bus_type, P_sched, P_gen, islanded):
        P = P_sched.astype(np.float64).copy()
        if not islanded.any():
            return P, False
        part = (bus_type == 1) & (~islanded) & (P_gen > 0.0)
        P[part] -= float(P_sched[islanded].sum()) * P_gen[part] / P_gen[part].sum()
        P[islanded] = 0.0
        return P, False

    monkeypatch.setattr(screen, "redispatch", flipped)
    monkeypatch.setattr(redispatch, "redispatch", flipped)
    with pytest.raises(AssertionError):
        pins.test_redispatch_hand_derived_ring()


def test_bridge_left_in_service_is_caught(monkeypatch):
    """The island found, but the outaged bridge kept in the post-outage B':
    the main island's matrix keeps the bridge's diagonal term, and the
    Schur-complement pin fails."""
    right = screen.outage_setup

    def keeps_branch(grid, l):
        on, label, isl, P, no_gen = right(grid, l)
        on = on.copy()
        if l >= 0:
            on[l] = True
        return on, label, isl, P, no_gen

    monkeypatch.setattr(screen, "outage_setup", keeps_branch)
    with pytest.raises(AssertionError):
        pins.test_bridge_outage_schur_complement_is_main_island_bprime()
