"""Parity beyond the named workloads: seeded grids of other sizes, seeds,
spur shares and transformer shares, every outage screened through the CUDA
path and compared with the oracle scenario by scenario (statuses and island
labels exactly; angles and magnitudes within 1e-6 at a 1e-10 p.u.
mismatch)."""
import functools

import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gridgen import make_grid
from oracle import powerflow as pf
from oracle import screen

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-6

# (buses, branches, seed, spur share, transformer share, loading): the
# loading is the largest of the ladder at which each base case converges
GRIDS = {
    "g600": (600, 840, 11, 0.05, 0.0, 0.1),
    "g900x": (900, 1250, 12, 0.1, 0.1, 0.15),
    "g1500": (1500, 2100, 13, 0.0, 0.0, 0.1),
}


@functools.lru_cache(maxsize=None)
def _case(name):
    n, m, seed, spur, xf, lam = GRIDS[name]
    g = make_grid(n, m, seed, spur_frac=spur, load_scale=lam, xfmr_frac=xf)
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-11, max_outer=200)
    assert st == pf.STATUS_OK
    outages = np.arange(g.n_branch, dtype=np.int32)
    ref = screen.n1_screen(g, th0, V0, outages, tol=1e-10, max_outer=100)
    return g, outages, ref


@pytest.mark.parametrize("name,precision,precond", [
    ("g600", gp.BATCHED_FP32, gp.PRECOND_EXACT),
    ("g900x", gp.BATCHED_FP32, gp.PRECOND_EXACT),
    ("g1500", gp.BATCHED_FP32, gp.PRECOND_EXACT),
    ("g900x", gp.BATCHED_FP64, gp.PRECOND_IC0),
    ("g1500", gp.BATCHED_FP32_F16, gp.PRECOND_EXACT),
])
def test_every_outage_of_seeded_grids(name, precision, precond):
    g, outages, ref = _case(name)
    c = gp.GPCG(g, precision=precision, precond=precond, tol=1e-10, max_outer=100)
    c.base_solve()
    res = c.n1_screen(outages, outputs=("theta", "V", "flow", "label", "status",
                                        "max_loading", "n_overload"))
    c.close()
    np.testing.assert_array_equal(res["status"], ref["status"])
    np.testing.assert_array_equal(res["label"], ref["label"])
    ok = np.isin(ref["status"], [0, 3])
    assert ok.sum() >= 0.95 * ok.size
    assert ref["islanded"].sum() >= 10
    for k, tol in (("theta", ANGLE_TOL), ("V", ANGLE_TOL), ("flow", 10 * ANGLE_TOL),
                   ("max_loading", 10 * ANGLE_TOL)):
        np.testing.assert_allclose(res[k][ok], ref[k][ok], rtol=0, atol=tol)
    ld = np.maximum(np.abs(ref["flow"]), np.abs(ref["flow_to"])) / g.rating
    clear = ok & ~(np.abs(ld - 1.0) <= 1e-6).any(axis=1)   # no branch at its rating
    np.testing.assert_array_equal(res["n_overload"][clear], ref["n_overload"][clear])
