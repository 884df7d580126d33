"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: the FP64 paths agree with the oracle to rounding; solutions
driven to a 1e-10 p.u. mismatch agree in angle to well below the 1e-6 rad
bar; FP32 operators are held to a bound derived from FP32 rounding.
"""
import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import (check_every_outage, grid, oracle_base, oracle_n1, sample_outages,
                        with_tight_ratings)
from oracle import factor, powerflow as pf, screen

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-6      # rad, against the oracle at a 1e-10 p.u. mismatch
MISMATCH_TOL = 1e-4   # p.u., the screening tolerance


def make(name, **opt):
    c = gp.GPCG(grid(name), **opt)
    return c


# ------------------------------------------------------------ a1, a2
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("precond", [gp.PRECOND_EXACT, gp.PRECOND_IC0])
def test_matrix_and_factor(which, precond):
    g = grid("grid120")
    c = make("grid120", precond=precond)
    d = c.export_matrix(which)
    keep = np.flatnonzero(g.bus_type != 2) if which == 0 else np.flatnonzero(g.bus_type == 0)
    on = np.ones(g.n_branch, bool)
    A = (pf.bprime(g.n_bus, g.f, g.t, g.x, on, keep) if which == 0
         else pf.bdprime(g.n_bus, g.f, g.t, g.r, g.x, on, keep)).toarray()
    pos = {b: k for k, b in enumerate(keep)}
    perm = np.array([pos[b] for b in d["bus_of_row"]])
    Ap = A[np.ix_(perm, perm)]
    n = Ap.shape[0]
    Ag = np.zeros((n, n))
    for i in range(n):
        for k in range(d["rowptr"][i], d["rowptr"][i + 1]):
            Ag[i, d["col"][k]] = d["val"][k]
    np.testing.assert_allclose(Ag, Ap, rtol=0, atol=1e-12 * np.abs(Ap).max())
    # the factor: oracle incomplete Cholesky on the exported pattern
    rows = [sorted(d["lcol"][d["lrowptr"][i]:d["lrowptr"][i + 1]].tolist()) for i in range(n)]
    from scipy.sparse import csr_matrix
    Lo = factor.to_dense(factor.ic_on_pattern(csr_matrix(Ap), rows), n)
    Lg = np.zeros((n, n))
    for i in range(n):
        for k in range(d["lrowptr"][i], d["lrowptr"][i + 1]):
            Lg[i, d["lcol"][k]] = d["lval"][k]
    np.testing.assert_allclose(Lg, Lo, rtol=0, atol=1e-11 * np.abs(Lo).max())
    if precond == gp.PRECOND_EXACT:
        np.testing.assert_allclose(Lg, np.linalg.cholesky(Ap), atol=1e-10 * np.abs(Lo).max())
    # level schedule: every dependency sits in a lower level
    lev = d["level"]
    for i in range(n):
        for j in rows[i][:-1]:
            assert lev[j] < lev[i]


# ------------------------------------------------------------ a8.1 / a8.2
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("precision", [gp.BATCHED_FP64, gp.BATCHED_FP32])
def test_spmv_with_outage_stamp(which, precision):
    g = grid("grid120")
    c = make("grid120")
    d = c.export_matrix(which)
    keep = np.flatnonzero(g.bus_type != 2) if which == 0 else np.flatnonzero(g.bus_type == 0)
    pos = {b: k for k, b in enumerate(keep)}
    perm = np.array([pos[b] for b in d["bus_of_row"]])
    outages = np.r_[np.arange(g.n_branch), -1].astype(np.int32)  # 181: ragged tail of 32-tiles
    rng = np.random.default_rng(1)
    X = rng.standard_normal((outages.size, perm.size))
    Y = c.apply(which, 0, outages, X, precision)
    for s, l in enumerate(outages):
        on = np.ones(g.n_branch, bool)
        if l >= 0:
            on[l] = False
        A = (pf.bprime(g.n_bus, g.f, g.t, g.x, on, keep) if which == 0
             else pf.bdprime(g.n_bus, g.f, g.t, g.r, g.x, on, keep)).toarray()
        ref = A[np.ix_(perm, perm)] @ X[s]
        scale = np.abs(A).max() * np.abs(X[s]).max() * 8
        tol = 1e-13 * scale if precision == gp.BATCHED_FP64 else 2e-6 * scale
        np.testing.assert_allclose(Y[s], ref, rtol=0, atol=tol)


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("precond", [gp.PRECOND_EXACT, gp.PRECOND_IC0])
def test_preconditioner_apply(which, precond):
    c = make("grid2k", precond=precond)
    d = c.export_matrix(which)
    n = d["bus_of_row"].size
    L = {i: {int(d["lcol"][k]): float(d["lval"][k])
             for k in range(d["lrowptr"][i], d["lrowptr"][i + 1])} for i in range(n)}
    outages = np.arange(37, dtype=np.int32)  # 37 scenarios: two tiles, ragged
    rng = np.random.default_rng(2)
    X = rng.standard_normal((outages.size, n))
    Y64 = c.apply(which, 1, outages, X, gp.BATCHED_FP64)
    Y32 = c.apply(which, 1, outages, X, gp.BATCHED_FP32)
    for s in range(0, outages.size, 6):
        ref = factor.apply_preconditioner(L, X[s])
        np.testing.assert_allclose(Y64[s], ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    # FP32: the substitutions are backward stable; assess them by the
    # residual of the FP64 factor, || L L^T y - x || <= c eps ||L|| ||L^T y||
    import scipy.sparse as sp
    Ls = sp.csr_matrix((d["lval"], d["lcol"], d["lrowptr"]), shape=(n, n))
    for s in range(0, outages.size, 6):
        res = Ls @ (Ls.T @ Y32[s]) - X[s]
        bound = 64 * 6e-8 * (abs(Ls) @ (abs(Ls.T) @ np.abs(Y32[s]))).max()
        assert np.abs(res).max() <= bound


def test_preconditioner_apply_fp16_factor():
    """Scaled FP16 storage: L = Ls D with Ls rounded to FP16.  The GPU's
    substitutions with FP32 vectors are held to the FP32 backward-error bound
    of the FP16-rounded factor, rebuilt here from the exported FP64 factor."""
    import scipy.sparse as sp
    c = make("grid2k")
    d = c.export_matrix(0)
    n = d["bus_of_row"].size
    rows = np.repeat(np.arange(n), np.diff(d["lrowptr"]))
    diag = d["lval"][d["lrowptr"][1:] - 1]
    ls = (d["lval"] / diag[d["lcol"]]).astype(np.float16).astype(np.float64)
    L16 = sp.csr_matrix((ls * diag[d["lcol"]], d["lcol"], d["lrowptr"]), shape=(n, n))
    assert np.all(rows >= d["lcol"])
    outages = np.arange(33, dtype=np.int32)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((outages.size, n))
    Y = c.apply(0, 1, outages, X, gp.BATCHED_FP32_F16)
    for s in range(0, outages.size, 8):
        res = L16 @ (L16.T @ Y[s]) - X[s]
        bound = 64 * 6e-8 * (abs(L16) @ (abs(L16.T) @ np.abs(Y[s]))).max()
        assert np.abs(res).max() <= bound


# ------------------------------------------------------------ a3
@pytest.mark.parametrize("name", ["grid120", "grid2k"])
def test_base_solve(name):
    c = make(name)
    b = c.base_solve()
    th, V = oracle_base(name)
    np.testing.assert_allclose(b["theta"], th, atol=1e-8)
    np.testing.assert_allclose(b["V"], V, atol=1e-8)
    assert c.info()["base_outer"] > 0


# ------------------------------------------------------------ full N-1
def _compare(g, res, ref, outages, angle_tol):
    np.testing.assert_array_equal(res["label"], ref["label"])
    np.testing.assert_array_equal(res["status"], ref["status"])
    ok = np.isin(ref["status"], [0, 3])
    assert ok.sum() > 0.9 * len(outages)
    np.testing.assert_allclose(res["theta"][ok], ref["theta"][ok], rtol=0, atol=angle_tol)
    np.testing.assert_allclose(res["V"][ok], ref["V"][ok], rtol=0, atol=angle_tol)
    np.testing.assert_allclose(res["flow"][ok], ref["flow"][ok], rtol=0, atol=10 * angle_tol)
    np.testing.assert_allclose(res["max_loading"][ok], ref["max_loading"][ok], atol=10 * angle_tol)


@pytest.mark.parametrize("precision,precond", [
    (gp.BATCHED_FP64, gp.PRECOND_EXACT), (gp.BATCHED_FP32, gp.PRECOND_EXACT),
    (gp.BATCHED_FP64, gp.PRECOND_IC0), (gp.BATCHED_FP32, gp.PRECOND_IC0),
    (gp.BATCHED_FP64, gp.PRECOND_JACOBI), (gp.PLAIN_FP64, gp.PRECOND_EXACT),
    (gp.PLAIN_FP64, gp.PRECOND_IC0), (gp.PLAIN_FP64, gp.PRECOND_JACOBI),
    (gp.BATCHED_FP32_F16, gp.PRECOND_EXACT), (gp.BATCHED_FP32_F16, gp.PRECOND_IC0)])
def test_n1_grid120_all_outages(precision, precond):
    g = grid("grid120")
    c = make("grid120", precision=precision, precond=precond, tol=1e-10, max_outer=100,
             inner_rtol=1e-6, max_inner=2000)
    c.base_solve()
    outages = np.arange(g.n_branch, dtype=np.int32)
    res = c.n1_screen(outages)
    ref = oracle_n1("grid120", outages, processes=1)
    _compare(g, res, ref, outages, ANGLE_TOL)
    assert (res["iters"][:, 0] >= 1).all()


@pytest.mark.parametrize("precision", [gp.BATCHED_FP32, gp.BATCHED_FP64, gp.PLAIN_FP64])
def test_n1_grid120_overload_screen(precision):
    """The overload screen (Sec. I) of every grid120 outage: per scenario the
    branches whose loading max(|P_ij|, |P_ji|) / rating exceeds 1, as a count
    and a bit mask, against the oracle's flows at a 1e-10 p.u. mismatch
    (ratings set just above the base-case flows; branches within 1e-7 of
    their rating, where the two solutions may round either way, are left
    out of the comparison)."""
    g = with_tight_ratings(grid("grid120"), seed=12)
    th0, V0 = oracle_base("grid120")
    c = gp.GPCG(g, precision=precision, tol=1e-10, max_outer=100)
    c.base_solve()
    outages = np.arange(g.n_branch, dtype=np.int32)
    res = c.n1_screen(outages, outputs=("status", "n_overload", "overload", "max_loading"))
    c.close()
    ref = screen.n1_screen(g, th0, V0, outages, tol=1e-10, max_outer=100, processes=1)
    np.testing.assert_array_equal(res["status"], ref["status"])
    ok = np.isin(ref["status"], [0, 3])
    ld = np.maximum(np.abs(ref["flow"]), np.abs(ref["flow_to"])) / g.rating
    tie = np.abs(ld - 1.0) <= 1e-7
    bits = gp.unpack_mask(res["overload"], g.n_branch)
    np.testing.assert_array_equal(bits[ok] & ~tie[ok], (ld > 1.0)[ok] & ~tie[ok])
    clear = ok & ~tie.any(axis=1)
    np.testing.assert_array_equal(res["n_overload"][clear], ref["n_overload"][clear])
    np.testing.assert_array_equal(bits.sum(axis=1), res["n_overload"])
    assert (ref["n_overload"][ok] > 0).sum() >= 20


def test_plain_path_grid2k_sample():
    """The plain FP64 path -- one scenario at a time, its rows spread over
    every CTA of a cooperative launch with grid-wide barriers between the
    levels of the substitutions -- on a seeded grid2k sample (islanding
    outages included) at a 1e-10 p.u. mismatch: statuses and labels exact,
    angles and magnitudes within 1e-6 of the oracle's."""
    g = grid("grid2k")
    samp = sample_outages(g, 24, seed=14)
    c = make("grid2k", precision=gp.PLAIN_FP64, tol=1e-10, max_outer=100)
    c.base_solve()
    res = c.n1_screen(samp, outputs=("theta", "V", "status", "label", "iters", "flow",
                                     "max_loading", "n_overload"))
    c.close()
    ref = oracle_n1("grid2k", samp, tol=1e-10)
    np.testing.assert_array_equal(res["status"], ref["status"])
    np.testing.assert_array_equal(res["label"], ref["label"])
    ok = np.isin(ref["status"], [0, 3])
    assert ok.sum() >= 0.9 * samp.size and (res["label"] != 0).any()
    assert np.abs(res["theta"][ok] - ref["theta"][ok]).max() <= ANGLE_TOL
    assert np.abs(res["V"][ok] - ref["V"][ok]).max() <= ANGLE_TOL
    assert np.abs(res["flow"][ok] - ref["flow"][ok]).max() <= 10 * ANGLE_TOL
    np.testing.assert_array_equal(res["n_overload"][ok], ref["n_overload"][ok])
    assert (res["iters"][ok, 1] >= 1).all()


def test_plain_path_bounded_wait_gives_up_and_recovers():
    """Bounded device waits: the plain path's grid-wide barriers allowed a
    single poll give up (the CTAs of a launch never arrive within 64 ns of
    each other), so the call ends with GPCG_ERR_TIMEOUT instead of waiting;
    the same context then screens with the default limit and matches the
    oracle."""
    g = grid("grid120")
    samp = np.arange(0, g.n_branch, 9, dtype=np.int32)
    c = make("grid120", precision=gp.PLAIN_FP64, tol=1e-10, max_outer=100, wait_limit=1)
    c.base_solve()
    with pytest.raises(gp.GPCGError) as e:
        c.n1_screen(samp, outputs=("status",))
    assert e.value.status == 5 and "barrier" in str(e.value)
    c.set_options(wait_limit=0)
    res = c.n1_screen(samp, outputs=("theta", "status", "label"))
    c.close()
    ref = oracle_n1("grid120", samp, tol=1e-10)
    np.testing.assert_array_equal(res["status"], ref["status"])
    np.testing.assert_array_equal(res["label"], ref["label"])
    ok = ref["status"] == 0
    assert np.abs(res["theta"][ok] - ref["theta"][ok]).max() <= ANGLE_TOL


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_n1_tiles_ragged(tile):
    g = grid("grid120")
    c = make("grid120", tile=tile, tol=1e-10, max_outer=100)
    c.base_solve()
    outages = np.arange(g.n_branch - 1, -1, -3, dtype=np.int32)  # 60 scenarios, reversed
    res = c.n1_screen(outages)
    ref = oracle_n1("grid120", outages, processes=1)
    _compare(g, res, ref, outages, ANGLE_TOL)


def test_n1_grid2k_sample_refined():
    g = grid("grid2k")
    c = make("grid2k", tol=1e-10, max_outer=100)
    c.base_solve()
    outages = sample_outages(g, 96, seed=3)
    res = c.n1_screen(outages)
    ref = oracle_n1("grid2k", outages)
    _compare(g, res, ref, outages, ANGLE_TOL)


def test_n1_grid2k_every_outage(tmp_path):
    """Every grid2k outage at the screening tolerance, scenario by scenario
    against the oracle: statuses and island labels exact, every converged
    state's FP64 mismatch (evaluated by the oracle) at most 1e-4 p.u., and the
    overload count of each converged scenario equal to the oracle's at that
    state (ratings set just above the base-case flows)."""
    g = with_tight_ratings(grid("grid2k"), seed=21)
    th0, V0 = oracle_base("grid2k")
    c = gp.GPCG(g)
    c.base_solve()
    outages = np.arange(g.n_branch, dtype=np.int32)
    res = c.n1_screen(outages, outputs=("theta", "V", "status", "label", "n_overload",
                                        "overload"))
    c.close()
    ref = check_every_outage(g, th0, V0, outages, res, tol=MISMATCH_TOL, tmpdir=tmp_path)
    np.testing.assert_array_equal(res["status"], ref["status"])
    assert ref["label_ok"].all()
    conv = np.isin(res["status"], (gp.SCEN_OK, gp.SCEN_ISLAND_NO_GEN))
    assert conv.sum() > 0.9 * outages.size
    # (the oracle's polar and the kernel's rectangular FP64 evaluations of a
    # state differ by rounding, ~1e-13 here)
    assert np.nanmax(ref["err"][conv]) <= MISMATCH_TOL + 1e-11
    clear = conv & (ref["ties"] == 0)
    np.testing.assert_array_equal(res["n_overload"][clear], ref["n_overload"][clear])
    assert (res["n_overload"] > 0).sum() > 20
    bits = gp.unpack_mask(res["overload"], g.n_branch)
    np.testing.assert_array_equal(bits.sum(axis=1), res["n_overload"])


@pytest.mark.parametrize("name", ["grid2k", "grid10k"])
def test_bridge_outages_take_one_pcg_iteration_per_p_step(name):
    """With the exact base-case factor the P-theta system of an islanding
    (bridge) outage is preconditioned exactly on the main island: the Schur
    complement of the island's block of the base-case B' is the post-outage
    B' of the main island (the identity the oracle tests pin).  So every P
    solve of such a scenario stops after one PCG iteration, at most one per
    outer iteration, while the outages that island nothing take more."""
    from paper_1803_03290_gb300 import binding
    g = grid(name)
    c = gp.GPCG(g)
    c.base_solve()
    outages = np.arange(g.n_branch, dtype=np.int32)
    res = c.n1_screen(outages, outputs=("iters", "status"))
    c.close()
    br = binding.analyze(g)["bridge"].astype(bool)
    ok = res["status"] == gp.SCEN_OK
    it = res["iters"]
    sel, rest = br & ok, ~br & ok
    assert sel.sum() > 100 and rest.sum() > 100
    assert (it[sel, 1] <= it[sel, 0]).all()
    assert it[sel, 1].sum() >= 0.9 * it[sel, 0].sum()
    assert it[rest, 1].sum() > 1.3 * it[rest, 0].sum()


def test_edge_cases():
    g = grid("grid120")
    c = make("grid120")
    with pytest.raises(gp.GPCGError):
        c.n1_screen(np.array([0], np.int32))   # base case not solved yet
    c.base_solve()
    r = c.n1_screen(np.zeros(0, np.int32))
    assert r["theta"].shape == (0, g.n_bus)
    with pytest.raises(gp.GPCGError):
        c.n1_screen(np.array([g.n_branch], np.int32))
    with pytest.raises(gp.GPCGError):
        c.n1_screen(np.array([-1], np.int32))
    # duplicates give identical answers
    r = c.n1_screen(np.array([5, 5, 5], np.int32))
    assert np.array_equal(r["theta"][0], r["theta"][2])


def test_pinned_host_outputs_written_in_place():
    """Host-mode outputs in page-locked memory are written by the kernels in
    place; pageable ones go through device staging: both give the same
    results."""
    torch = pytest.importorskip("torch")
    g = grid("grid2k")
    c = make("grid2k")
    c.base_solve()
    outages = sample_outages(g, 40, seed=15)
    S, n, m = outages.size, g.n_bus, g.n_branch
    keys = ("theta", "V", "flow", "label", "iters", "status", "max_loading", "n_overload",
            "overload")
    pageable = c.n1_screen(outages, outputs=keys)
    shapes = {"theta": ((S, n), torch.float64), "V": ((S, n), torch.float64),
              "flow": ((S, m), torch.float64), "label": ((S, n), torch.int32),
              "iters": ((S, 3), torch.int32), "status": ((S,), torch.int32),
              "max_loading": ((S,), torch.float64), "n_overload": ((S,), torch.int32),
              "overload": ((S, gp.mask_words(m)), torch.int32)}
    pinned = {k: torch.full(shp, -3, dtype=dt, pin_memory=True) for k, (shp, dt) in shapes.items()}
    for _ in range(2):  # twice: the second call reuses the pinned buffers
        c.n1_screen(outages, out=pinned)
        for k in keys:
            got = pinned[k].numpy()
            want = pageable[k].view(np.int32) if k == "overload" else pageable[k]
            np.testing.assert_array_equal(got, want, err_msg=k)
    c.close()
