"""The GPU adjoint (gpcg_n1_adjoint) against the oracle's DC adjoint and
against finite differences of its own loss."""
import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import grid
from oracle import adjoint

pytestmark = pytest.mark.gpu


def _case(name, scale):
    g = grid(name)
    return g, g.P_sched * scale, 1.0 / g.x


@pytest.mark.parametrize("precond", [gp.PRECOND_EXACT, gp.PRECOND_IC0])
def test_adjoint_matches_oracle_grid120(precond):
    g, P, b = _case("grid120", 8.0)
    outages = np.arange(g.n_branch, dtype=np.int32)  # includes islanding outages
    c = gp.GPCG(g, precond=precond)
    L, gP, gb = c.n1_adjoint(outages, P, b)
    Lo, gPo, gbo = adjoint.loss_and_grad(g, outages, P, b)
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    np.testing.assert_allclose(gP, gPo, rtol=1e-8, atol=1e-10 * np.abs(gPo).max())
    np.testing.assert_allclose(gb, gbo, rtol=1e-8, atol=1e-10 * np.abs(gbo).max())
    # perturbed susceptances re-factorise the base case
    b2 = b * np.random.default_rng(1).uniform(0.8, 1.2, g.n_branch)
    L2, gP2, gb2 = c.n1_adjoint(outages, P, b2)
    Lo2, gPo2, gbo2 = adjoint.loss_and_grad(g, outages, P, b2)
    assert abs(L2 - Lo2) <= 1e-10 * abs(Lo2)
    np.testing.assert_allclose(gb2, gbo2, rtol=1e-8, atol=1e-10 * np.abs(gbo2).max())


def _fd5(fun, x, i, h):
    def at(d):
        y = x.copy()
        y[i] += d
        return fun(y)
    return (-at(2 * h) + 8 * at(h) - 8 * at(-h) + at(-2 * h)) / (12 * h)


def test_adjoint_matches_central_differences_grid120():
    """Central differences of the library's own loss (five-point rule).
    The penalty has a kink at zero flow, so steps stay small (1e-4)."""
    g, P, b = _case("grid120", 8.0)
    outages = np.arange(g.n_branch, dtype=np.int32)
    c = gp.GPCG(g)
    L, gP, gb = c.n1_adjoint(outages, P, b)
    rng = np.random.default_rng(2)
    nonslack = np.flatnonzero(g.bus_type != 2)
    for i in rng.choice(nonslack, 6, replace=False):
        fd = _fd5(lambda y: c.n1_adjoint(outages, y, b, grads=False)[0], P, i, 1e-4)
        assert abs(fd - gP[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gP[i])
    for k in rng.choice(g.n_branch, 6, replace=False):
        fd = _fd5(lambda y: c.n1_adjoint(outages, P, y, grads=False)[0], b, k, 1e-4 * b[k])
        assert abs(fd - gb[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, gb[k])


def test_adjoint_grid2k_all_outages_vs_oracle():
    """The adjoint workload: every outage of the 2,000-bus grid, against the
    oracle's adjoint; repeated calls are bitwise identical."""
    g, P, b = _case("grid2k", 1.0)
    outages = np.arange(g.n_branch, dtype=np.int32)
    c = gp.GPCG(g)
    L, gP, gb = c.n1_adjoint(outages, P, b)
    L_again, gP_again, gb_again = c.n1_adjoint(outages, P, b)
    assert L == L_again and np.array_equal(gP, gP_again) and np.array_equal(gb, gb_again)
    Lo, gPo, gbo = adjoint.loss_and_grad(g, outages, P, b)
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    np.testing.assert_allclose(gP, gPo, rtol=1e-7, atol=1e-9 * np.abs(gPo).max())
    np.testing.assert_allclose(gb, gbo, rtol=1e-7, atol=1e-9 * np.abs(gbo).max())


def test_adjoint_autograd_function():
    torch = pytest.importorskip("torch")
    g, P, b = _case("grid120", 8.0)
    c = gp.GPCG(g)
    dev = torch.device("cuda", 0)
    outages = torch.arange(g.n_branch, dtype=torch.int32, device=dev)
    Pt = torch.tensor(P, device=dev, requires_grad=True)
    bt = torch.tensor(b, device=dev, requires_grad=True)
    loss = gp.overload_loss(c, outages, Pt, bt)
    (3.0 * loss).backward()
    L, gP, gb = c.n1_adjoint(np.arange(g.n_branch), P, b)
    assert abs(loss.item() - L) <= 1e-12 * abs(L)
    np.testing.assert_allclose(Pt.grad.cpu().numpy(), 3.0 * gP, rtol=1e-12, atol=0)
    np.testing.assert_allclose(bt.grad.cpu().numpy(), 3.0 * gb, rtol=1e-12, atol=0)


def test_adjoint_edge_cases():
    g, P, b = _case("grid120", 1.0)
    c = gp.GPCG(g)
    L, gP, gb = c.n1_adjoint(np.zeros(0, np.int32), P, b)
    assert L == 0.0 and not gP.any() and not gb.any()
    with pytest.raises(gp.GPCGError):
        c.n1_adjoint(np.array([g.n_branch], np.int32), P, b)
    bad = b.copy()
    bad[0] = -1.0
    with pytest.raises(gp.GPCGError):
        c.n1_adjoint(np.array([0], np.int32), P, bad)
