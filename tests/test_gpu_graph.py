"""Device-mode screens replayed from the captured CUDA graph, and the tile
autotuner: the results must be the oracle's whatever the replay state.

gpcg_n1_screen with device pointers captures the islanding and solve
launches once per (n_out, outputs, options) and replays them; the outage
list is copied in before each replay, so a replay with new outages must
screen the new outages.  gpcg_set_options drops the graph.
"""
import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import grid, oracle_n1, sample_outages

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-6


def _outputs(torch, S, n, m, dev):
    return {
        "theta": torch.full((S, n), np.nan, dtype=torch.float64, device=dev),
        "V": torch.full((S, n), np.nan, dtype=torch.float64, device=dev),
        "flow": torch.full((S, m), np.nan, dtype=torch.float64, device=dev),
        "label": torch.full((S, n), -7, dtype=torch.int32, device=dev),
        "iters": torch.full((S, 3), -7, dtype=torch.int32, device=dev),
        "status": torch.full((S,), -7, dtype=torch.int32, device=dev),
        "max_loading": torch.full((S,), np.nan, dtype=torch.float64, device=dev),
    }


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check_oracle(g, res, ref):
    np.testing.assert_array_equal(res["label"], ref["label"])
    np.testing.assert_array_equal(res["status"], ref["status"])
    ok = np.isin(ref["status"], [0, 3])
    np.testing.assert_allclose(res["theta"][ok], ref["theta"][ok], rtol=0, atol=ANGLE_TOL)
    np.testing.assert_allclose(res["V"][ok], ref["V"][ok], rtol=0, atol=ANGLE_TOL)
    np.testing.assert_allclose(res["flow"][ok], ref["flow"][ok], rtol=0, atol=10 * ANGLE_TOL)


def test_graph_replay_with_new_outages():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    g = grid("grid2k")
    c = gp.GPCG(g, tol=1e-10, max_outer=100, tile=0)
    c.base_solve()
    A = sample_outages(g, 96, seed=11)
    B = sample_outages(g, 96, seed=12)
    S = min(len(A), len(B))
    A, B = A[:S], B[:S]
    out = _outputs(torch, S, g.n_bus, g.n_branch, dev)
    dA = torch.from_numpy(A).to(dev)
    dB = torch.from_numpy(B).to(dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c.n1_screen_device(dA, out, stream=stream)       # captures
    stream.synchronize()
    assert c.info()["tile"] in (2, 4, 8)
    first = _host(out)
    _check_oracle(g, first, oracle_n1("grid2k", A))
    with torch.cuda.stream(stream):
        c.n1_screen_device(dB, out, stream=stream)       # replays, new outages
    stream.synchronize()
    _check_oracle(g, _host(out), oracle_n1("grid2k", B))
    with torch.cuda.stream(stream):
        c.n1_screen_device(dA, out, stream=stream)       # replays again
    stream.synchronize()
    again = _host(out)
    for k in ("status", "iters", "label"):
        np.testing.assert_array_equal(again[k], first[k])
    ok = first["status"] == 0
    np.testing.assert_allclose(again["theta"][ok], first["theta"][ok], rtol=0, atol=ANGLE_TOL)
    isl, sol = c.last_timings()
    assert isl > 0 and sol > 0
    c.close()


def test_set_options_drops_graph():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    g = grid("grid2k")
    c = gp.GPCG(g, tol=1e-10, max_outer=100)
    c.base_solve()
    A = sample_outages(g, 64, seed=5)
    S = len(A)
    dA = torch.from_numpy(A).to(dev)
    out = _outputs(torch, S, g.n_bus, g.n_branch, dev)
    c.n1_screen_device(dA, out)
    torch.cuda.synchronize()
    tight = _host(out)
    c.set_options(tol=1e-3, max_outer=3)                 # a looser screen
    c.n1_screen_device(dA, out)
    torch.cuda.synchronize()
    loose = _host(out)
    host = c.n1_screen(A)                                # same options, host mode
    for k in ("status", "iters", "label"):
        np.testing.assert_array_equal(loose[k], host[k])
    # the loose screen stopped earlier than the tight one
    assert loose["iters"][:, 0].sum() < tight["iters"][:, 0].sum()
    c.set_options(tol=1e-10, max_outer=100)
    c.n1_screen_device(dA, out)
    torch.cuda.synchronize()
    _check_oracle(g, _host(out), oracle_n1("grid2k", A))
    c.close()


def test_autotuner_keeps_choice_and_explicit_tile_wins():
    g = grid("grid2k")
    c = gp.GPCG(g, tile=0, tol=1e-10, max_outer=100)
    assert c.info()["tile"] == 0
    c.base_solve()
    A = sample_outages(g, 48, seed=9)
    r1 = c.n1_screen(A)
    t = c.info()["tile"]
    assert t in (2, 4, 8)
    r2 = c.n1_screen(A)
    assert c.info()["tile"] == t
    np.testing.assert_array_equal(r1["status"], r2["status"])
    c.set_options(tile=4)
    assert c.info()["tile"] == 4
    r4 = c.n1_screen(A)
    np.testing.assert_array_equal(r4["status"], r1["status"])
    ok = r1["status"] == 0
    np.testing.assert_allclose(r4["theta"][ok], r1["theta"][ok], rtol=0, atol=ANGLE_TOL)
    c.close()
