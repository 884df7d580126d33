"""Generator outages (Sec. IV.A: the loss of a single component) through the
CUDA path (gpcg_n1_gen_screen) against the CPU oracle: the tripped PV bus
becomes PQ with its load, its generation is re-dispatched, and B'' gains the
bus's row."""
import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import grid, oracle_base
from oracle import screen

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-6


def oracle_gen(name, buses, tol=1e-10, processes=None):
    g = grid(name)
    th0, V0 = oracle_base(name)
    return screen.n1_screen(g, th0, V0, buses, tol=tol, max_outer=100, processes=processes,
                            kind="generator")


def _compare(res, ref, n_out):
    np.testing.assert_array_equal(res["status"], ref["status"])
    assert np.all(res["label"] == 0)
    ok = np.isin(ref["status"], [0, 3])
    assert ok.sum() > 0.9 * n_out
    for k, tol in (("theta", ANGLE_TOL), ("V", ANGLE_TOL), ("flow", 10 * ANGLE_TOL),
                   ("max_loading", 10 * ANGLE_TOL)):
        np.testing.assert_allclose(res[k][ok], ref[k][ok], rtol=0, atol=tol)


@pytest.mark.parametrize("name", ["grid120", "grid120_xfmr"])
@pytest.mark.parametrize("precision,precond", [
    (gp.BATCHED_FP32, gp.PRECOND_EXACT), (gp.BATCHED_FP64, gp.PRECOND_EXACT),
    (gp.BATCHED_FP32, gp.PRECOND_IC0), (gp.BATCHED_FP64, gp.PRECOND_JACOBI),
    (gp.PLAIN_FP64, gp.PRECOND_EXACT), (gp.BATCHED_FP32_F16, gp.PRECOND_EXACT)])
def test_gen_outages_grid120_all(name, precision, precond):
    g = grid(name)
    c = gp.GPCG(g, precision=precision, precond=precond, tol=1e-10, max_outer=100,
                inner_rtol=1e-6, max_inner=2000)
    c.base_solve()
    buses = np.flatnonzero(g.bus_type == 1).astype(np.int32)
    res = c.n1_gen_screen(buses)
    ref = oracle_gen(name, buses, processes=1)
    _compare(res, ref, buses.size)
    # the tripped bus no longer holds its set point
    moved = np.abs(res["V"][np.arange(buses.size), buses] - g.V_set[buses])
    assert np.all(moved[res["status"] == 0] > 1e-6)
    c.close()


@pytest.mark.parametrize("tile", [2, 8])
def test_gen_outages_grid2k_sample(tile):
    """Refined to 1e-10 p.u. against the oracle; at the 1e-4 screening
    tolerance every converged state's FP64 mismatch (the oracle's) is within
    it."""
    g = grid("grid2k")
    pv = np.flatnonzero(g.bus_type == 1)
    buses = np.sort(np.random.default_rng(11).choice(pv, 61, replace=False)).astype(np.int32)
    c = gp.GPCG(g, tol=1e-10, max_outer=100, tile=tile)
    c.base_solve()
    res = c.n1_gen_screen(buses)
    _compare(res, oracle_gen("grid2k", buses), buses.size)
    c.close()
    c = gp.GPCG(g, tile=tile)
    c.base_solve()
    res = c.n1_gen_screen(buses, outputs=("theta", "V", "status", "iters"))
    assert np.all(res["status"] == 0)
    for s, k in enumerate(buses):
        e = screen.generator_mismatch(g, int(k), res["theta"][s], res["V"][s])
        assert e <= 1e-4 * (1 + 1e-9)
    c.close()


def test_gen_outages_device_graph_replay():
    torch = pytest.importorskip("torch")
    g = grid("grid2k")
    buses = np.flatnonzero(g.bus_type == 1)[:100].astype(np.int32)
    c = gp.GPCG(g)
    c.base_solve()
    ref = c.n1_gen_screen(buses)
    dev = torch.device("cuda", 0)
    S, n, m = buses.size, g.n_bus, g.n_branch
    out = dict(theta=torch.empty(S, n, dtype=torch.float64, device=dev),
               V=torch.empty(S, n, dtype=torch.float64, device=dev),
               flow=torch.empty(S, m, dtype=torch.float64, device=dev),
               label=torch.empty(S, n, dtype=torch.int32, device=dev),
               iters=torch.empty(S, 3, dtype=torch.int32, device=dev),
               status=torch.empty(S, dtype=torch.int32, device=dev),
               max_loading=torch.empty(S, dtype=torch.float64, device=dev))
    for _ in range(2):  # capture, then replay
        c.n1_gen_screen_device(torch.from_numpy(buses).to(dev), out)
        torch.cuda.synchronize()
        for k in ("theta", "V", "flow", "label", "iters", "status", "max_loading"):
            assert np.array_equal(out[k].cpu().numpy(), ref[k]), k
    # a branch screen on the same context after generator screens is unchanged
    br = np.arange(40, dtype=np.int32)
    a = c.n1_screen(br)
    c.n1_gen_screen(buses[:7])
    b = c.n1_screen(br)
    for k in ("theta", "V", "status", "iters"):
        assert np.array_equal(a[k], b[k]), k
    c.close()


def test_gen_outage_rejects_non_pv_buses():
    g = grid("grid120")
    c = gp.GPCG(g)
    c.base_solve()
    for b in (int(np.flatnonzero(g.bus_type == 0)[0]), g.slack, -1, g.n_bus):
        with pytest.raises(gp.GPCGError) as e:
            c.n1_gen_screen(np.array([b], np.int32))
        assert e.value.status == 1
    r = c.n1_gen_screen(np.zeros(0, np.int32))
    assert r["theta"].shape == (0, g.n_bus)
    c.close()


def test_gen_outages_without_other_generators():
    """Only one PV generator carries P_gen: tripping it leaves nobody to take
    the re-dispatch (the slack absorbs it: ISLAND_NO_GEN); tripping a PV bus
    with P_gen = 0 re-dispatches nothing.  Against the oracle."""
    import paper_1803_03290_gb300 as gp
    from oracle import powerflow as pf
    g = grid("grid120").copy()
    pv = np.flatnonzero(g.bus_type == 1)
    g.P_gen = g.P_gen.copy()
    g.P_gen[pv[1:]] = 0.0          # bus pv[0] is the only generator with P_gen > 0
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-11, max_outer=200)
    assert st == pf.STATUS_OK
    buses = pv[:8].astype(np.int32)
    c = gp.GPCG(g, tol=1e-10, max_outer=100)
    c.base_solve()
    res = c.n1_gen_screen(buses)
    ref = screen.n1_screen(g, th0, V0, buses, tol=1e-10, max_outer=100, processes=1,
                           kind="generator")
    assert ref["status"][0] == pf.STATUS_ISLAND_NO_GEN
    _compare(res, ref, buses.size)
    c.close()
