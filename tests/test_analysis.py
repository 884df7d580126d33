"""Host-side structural analysis of the library (gpcg_analyze), no GPU:
orderings, factor patterns, level schedules, bridges."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix

from gridgen import config_grid
from oracle import factor, islands
from oracle import powerflow as pf
from paper_1803_03290_gb300 import binding

pytestmark = pytest.mark.filterwarnings("ignore")


def _permuted_lower_pattern(g, d, which):
    keep = np.flatnonzero(g.bus_type != 2) if which == 0 else np.flatnonzero(g.bus_type == 0)
    on = np.ones(g.n_branch, bool)
    A = (pf.bprime(g.n_bus, g.f, g.t, g.x, on, keep) if which == 0
         else pf.bdprime(g.n_bus, g.f, g.t, g.r, g.x, on, keep))
    pos = {b: k for k, b in enumerate(keep)}
    perm = np.array([pos[b] for b in d["bus_of_row"]])
    Ap = csr_matrix(A[perm][:, perm])
    return [sorted(int(c) for c in Ap.indices[Ap.indptr[i]:Ap.indptr[i + 1]] if c <= i)
            for i in range(Ap.shape[0])], keep


def _rows(d):
    return [sorted(d["lcol"][d["lrowptr"][i]:d["lrowptr"][i + 1]].tolist())
            for i in range(d["bus_of_row"].size)]


@pytest.mark.parametrize("name", ["grid120", "grid2k"])
@pytest.mark.parametrize("which", [0, 1])
def test_factor_patterns_and_levels(name, which):
    g = config_grid(name)
    ex = binding.analyze(g, binding.PRECOND_EXACT, which)
    ic = binding.analyze(g, binding.PRECOND_IC0, which)
    # rows cover exactly the matrix's buses
    lower, keep = _permuted_lower_pattern(g, ex, which)
    assert sorted(ex["bus_of_row"].tolist()) == sorted(keep.tolist())
    # exact: the complete symbolic Cholesky pattern of the permuted matrix
    assert _rows(ex) == factor.symbolic_cholesky(len(lower), lower)
    # IC(0): the lower triangle itself
    lower_ic, _ = _permuted_lower_pattern(g, ic, which)
    assert _rows(ic) == lower_ic
    for d in (ex, ic):
        lev = d["level"]
        assert np.all(np.diff(lev) >= 0)           # levels are contiguous row ranges
        for i, row in enumerate(_rows(d)):
            assert row[-1] == i
            for j in row[:-1]:
                assert lev[j] < lev[i]              # dependencies in lower levels
        assert d["info"]["levels"] == lev.max() + 1


def test_bridges_match_brute_force():
    g = config_grid("grid120")
    d = binding.analyze(g)
    for e in range(g.n_branch):
        on = np.ones(g.n_branch, bool)
        on[e] = False
        split = len(set(islands.components(g.n_bus, g.f, g.t, on))) > 1
        assert bool(d["bridge"][e]) == split
    assert d["info"]["n_bridges"] == int(d["bridge"].sum())


def test_internal_order_reduces_bandwidth():
    g = config_grid("grid2k")
    d = binding.analyze(g)
    order = d["bus_order"]
    assert sorted(order.tolist()) == list(range(g.n_bus))
    pos = np.empty(g.n_bus, int)
    pos[order] = np.arange(g.n_bus)
    before = np.abs(g.f - g.t).max()
    after = np.abs(pos[g.f] - pos[g.t]).max()
    assert after < before / 3


def test_analyze_rejects_bad_grids():
    g = config_grid("grid120")
    bad = g.copy()
    bad.t = bad.t.copy()
    bad.t[0] = 10_000
    with pytest.raises(binding.GPCGError) as e:
        binding.analyze(bad)
    assert e.value.status == 1
    # a disconnected grid: drop every branch of bus 7
    g2 = g.copy()
    keep = (g2.f != 7) & (g2.t != 7)
    for k in ("f", "t", "r", "x", "b_sh", "rating"):
        setattr(g2, k, getattr(g2, k)[keep])
    with pytest.raises(binding.GPCGError) as e:
        binding.analyze(g2)
    assert e.value.status == 4
