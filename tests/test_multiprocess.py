"""The multi-rank path on CPU: two gloo ranks shard the N-1 scenarios with no
collective on the data path and must reproduce a single-process run
(results bit-exact, adjoint gradient sums within FP64 reassociation)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    from gridgen import config_grid
    from oracle import adjoint, powerflow as pf, screen
    from paper_1803_03290_gb300 import shard

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    g = config_grid("grid120")
    th0, V0, _, _, _ = pf.base_case(g, tol=1e-11, max_outer=200)
    outages = np.arange(g.n_branch)
    mine = shard.shard_outages(outages, rank, world)
    res = screen.n1_screen(g, th0, V0, mine, tol=1e-10, processes=1)
    theta = shard.gather_rows(res["theta"], outages.size)
    status = shard.gather_rows(res["status"], outages.size)
    P, b = g.P_sched * 8.0, 1.0 / g.x
    L, gP, gb = adjoint.loss_and_grad(g, mine, P, b)
    Ltot = shard.sum_over_ranks(np.array([L]))[0]
    gPt = shard.sum_over_ranks(gP)
    gbt = shard.sum_over_ranks(gb)
    tmax = shard.max_over_ranks(float(rank + 1))
    if rank == 0:
        np.savez(os.path.join(outdir, "ranked.npz"), theta=theta, status=status, L=Ltot, gP=gPt,
                 gb=gbt, tmax=tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_one_process(tmp_path):
    import torch.multiprocessing as tmp
    from gridgen import config_grid
    from oracle import adjoint, powerflow as pf, screen

    port = _free_port()
    tmp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                        start_method="spawn")
    got = np.load(os.path.join(tmp_path, "ranked.npz"))
    g = config_grid("grid120")
    th0, V0, _, _, _ = pf.base_case(g, tol=1e-11, max_outer=200)
    ref = screen.n1_screen(g, th0, V0, np.arange(g.n_branch), tol=1e-10, processes=1)
    assert np.array_equal(got["theta"], ref["theta"])
    assert np.array_equal(got["status"], ref["status"])
    L, gP, gb = adjoint.loss_and_grad(g, np.arange(g.n_branch), g.P_sched * 8.0, 1.0 / g.x)
    assert abs(float(got["L"]) - L) <= 1e-12 * abs(L)
    np.testing.assert_allclose(got["gP"], gP, rtol=1e-12, atol=1e-12 * np.abs(gP).max())
    np.testing.assert_allclose(got["gb"], gb, rtol=1e-12, atol=1e-12 * np.abs(gb).max())
    assert float(got["tmax"]) == 2.0


def test_shard_bounds_cover_exactly():
    from paper_1803_03290_gb300.shard import shard_bounds
    for S in (0, 1, 7, 180, 13500):
        for world in (1, 2, 3, 8):
            spans = [shard_bounds(S, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == S
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
