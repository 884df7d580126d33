"""The DC (P-theta) N-1 quick screen, CUDA path against the oracle's direct
per-scenario solves (oracle.dc) on the same seeded grids."""
import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import check_every_dc_outage, grid, sample_outages, with_tight_ratings
from oracle import dc

pytestmark = pytest.mark.gpu


def _check(res, ref, th_tol, f_tol):
    np.testing.assert_array_equal(res["status"], ref["status"])
    np.testing.assert_allclose(res["theta"], ref["theta"], rtol=0, atol=th_tol)
    np.testing.assert_allclose(res["flow"], ref["flow"], rtol=0, atol=f_tol)
    np.testing.assert_allclose(res["max_loading"], ref["max_loading"], rtol=0, atol=f_tol)


# FP32 solves are refined once in FP64: error ~ (FP32 solve error)^2
@pytest.mark.parametrize("precision,th_tol,f_tol", [
    (gp.BATCHED_FP64, 1e-10, 1e-8), (gp.BATCHED_FP32, 1e-7, 1e-5),
    (gp.BATCHED_FP32_F16, 1e-7, 1e-5)])
def test_dc_grid120_all_outages(precision, th_tol, f_tol):
    g = grid("grid120")
    c = gp.GPCG(g, precision=precision)
    outages = np.arange(g.n_branch, dtype=np.int32)
    res = c.n1_dc_screen(outages)
    ref = dc.dc_screen(g, outages)
    _check(res, ref, th_tol, f_tol)
    assert (res["iters"] >= 1).all() and (res["iters"] <= 10).all()
    c.close()


@pytest.mark.parametrize("precision", [gp.BATCHED_FP64, gp.BATCHED_FP32])
def test_dc_grid120_overload_screen(precision):
    """Branches above their rating per DC scenario (count and bit mask)
    against the oracle's DC flows; branches within 1e-5 of their rating
    (the FP32 solves' flow tolerance) are left out."""
    g = with_tight_ratings(grid("grid120"), seed=13)
    c = gp.GPCG(g, precision=precision)
    outages = np.arange(g.n_branch, dtype=np.int32)
    res = c.n1_dc_screen(outages, outputs=("status", "n_overload", "overload", "flow"))
    c.close()
    ref = dc.dc_screen(g, outages)
    ld = np.abs(ref["flow"]) / g.rating
    tie = np.abs(ld - 1.0) <= 1e-5
    bits = gp.unpack_mask(res["overload"], g.n_branch)
    np.testing.assert_array_equal(bits & ~tie, (ld > 1.0) & ~tie)
    clear = ~tie.any(axis=1)
    np.testing.assert_array_equal(res["n_overload"][clear], ref["n_overload"][clear])
    np.testing.assert_array_equal(bits.sum(axis=1), res["n_overload"])
    assert (ref["n_overload"] > 0).sum() >= 20


def test_dc_grid2k_sample_with_injections():
    """A seeded sample (bridges included, ragged last tile) with caller
    injections: P scaled and perturbed, sum kept."""
    g = grid("grid2k")
    rng = np.random.default_rng(4)
    P = g.P_sched * rng.uniform(0.8, 1.2, g.n_bus)
    c = gp.GPCG(g, precision=gp.BATCHED_FP64)
    outages = sample_outages(g, 75, seed=6)
    res = c.n1_dc_screen(outages, P=P)
    ref = dc.dc_screen(g, outages, P=P)
    _check(res, ref, 1e-9, 1e-7)
    c.close()


def test_dc_device_mode_matches_host():
    torch = pytest.importorskip("torch")
    g = grid("grid2k")
    dev = torch.device("cuda", 0)
    c = gp.GPCG(g)
    outages = sample_outages(g, 40, seed=7)
    host = c.n1_dc_screen(outages)
    S = outages.size
    out = {"theta": torch.empty((S, g.n_bus), dtype=torch.float64, device=dev),
           "flow": torch.empty((S, g.n_branch), dtype=torch.float64, device=dev),
           "iters": torch.empty((S,), dtype=torch.int32, device=dev),
           "status": torch.empty((S,), dtype=torch.int32, device=dev),
           "max_loading": torch.empty((S,), dtype=torch.float64, device=dev)}
    c.n1_dc_screen_device(torch.from_numpy(outages).to(dev), out)
    torch.cuda.synchronize()
    for k in out:
        np.testing.assert_array_equal(out[k].cpu().numpy(), host[k])
    c.close()


def test_dc_rejects_bad_input():
    g = grid("grid120")
    c = gp.GPCG(g)
    with pytest.raises(gp.GPCGError):
        c.n1_dc_screen(np.array([0, g.n_branch], dtype=np.int32))
    assert c.n1_dc_screen(np.zeros(0, dtype=np.int32))["status"].size == 0
    c.set_options(precision=gp.PLAIN_FP64)
    with pytest.raises(gp.GPCGError):
        c.n1_dc_screen(np.array([0], dtype=np.int32))
    c.close()


def _with_tight_dc_ratings(g, seed):
    """Ratings U[1.0, 1.5] times each branch's DC base-case flow plus 1e-3
    p.u. (the DC flows of the intact grid, B' theta = P with the slack's
    angle 0), so that outages push the DC flows of their neighbours over."""
    import scipy.sparse as sps
    from scipy.sparse.linalg import spsolve
    n = g.n_bus
    w = 1.0 / g.x
    B = sps.csr_matrix((np.r_[w, w, -w, -w], (np.r_[g.f, g.t, g.f, g.t], np.r_[g.f, g.t, g.t, g.f])),
                       shape=(n, n))
    keep = np.flatnonzero(g.bus_type != 2)
    th = np.zeros(n)
    th[keep] = spsolve(B[keep][:, keep].tocsc(), g.P_sched[keep])
    f = w * (th[g.f] - th[g.t])
    g = g.copy()
    g.rating = np.abs(f) * np.random.default_rng(seed).uniform(1.0, 1.5, g.n_branch) + 1e-3
    return g


def test_dc_grid10k_every_outage(tmp_path):
    """Every one of grid10k's 13,500 outages through the DC quick screen,
    against the oracle's direct solves scenario by scenario (ratings set
    just above the DC base-case flows).  FP64 solves (1e-12 relative
    residual): statuses, angles within 1e-9 rad, flows within 1e-7 p.u.,
    overload counts exactly where no branch is within 1e-6 of its rating.
    FP32 solves refined once in FP64 (the benchmark's configuration):
    statuses, angles within the 1e-6 rad parity tolerance, and flows within
    what that bound allows, 2e-6 / x for a branch of reactance x."""
    g = _with_tight_dc_ratings(grid("grid10k"), seed=17)
    outages = np.arange(g.n_branch, dtype=np.int32)
    runs = {}
    for name, prec in (("fp64", gp.BATCHED_FP64), ("fp32", gp.BATCHED_FP32)):
        c = gp.GPCG(g, precision=prec)
        runs[name] = c.n1_dc_screen(outages, outputs=("theta", "flow", "status", "n_overload"))
        c.close()
    ref = check_every_dc_outage(g, outages, runs, tmp_path)
    for name in runs:
        np.testing.assert_array_equal(runs[name]["status"], ref["status"])
    assert ref["fp64"]["dtheta"].max() <= 1e-9, ref["fp64"]["dtheta"].max()
    assert ref["fp64"]["dflow"].max() <= 1e-7, ref["fp64"]["dflow"].max()
    clear = ref["ties"] == 0
    np.testing.assert_array_equal(runs["fp64"]["n_overload"][clear], ref["n_overload"][clear])
    assert clear.sum() >= 0.95 * outages.size
    assert (ref["n_overload"] > 0).sum() > 100
    assert ref["fp32"]["dtheta"].max() <= 1e-6, ref["fp32"]["dtheta"].max()
    assert ref["fp32"]["dflow"].max() <= 2e-6 / g.x.min(), ref["fp32"]["dflow"].max()
