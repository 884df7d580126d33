"""gpcg_n1_screen_noalloc, the screen for callers that cannot allocate GPU
memory while they run, against the regular gpcg_n1_screen.

The no-allocation entry point works in the library's fixed device array;
the regular one allocates its scratch.  Both run the same kernels, so on the
same context and outages they must agree (statuses, iteration counts and
island labels exactly; the FP64 state within the parity tests' angle
tolerance) -- and keep agreeing on a second call, which reuses the array.
This file is collected last so a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-6


def _device_outputs(torch, S, n, m, dev):
    return {
        "theta": torch.full((S, n), np.nan, dtype=torch.float64, device=dev),
        "V": torch.full((S, n), np.nan, dtype=torch.float64, device=dev),
        "flow": torch.full((S, m), np.nan, dtype=torch.float64, device=dev),
        "label": torch.full((S, n), -7, dtype=torch.int32, device=dev),
        "iters": torch.full((S, 3), -7, dtype=torch.int32, device=dev),
        "status": torch.full((S,), -7, dtype=torch.int32, device=dev),
        "max_loading": torch.full((S,), np.nan, dtype=torch.float64, device=dev),
        "n_overload": torch.full((S,), -7, dtype=torch.int32, device=dev),
        "overload": torch.full((S, (m + 31) // 32), 7, dtype=torch.int32, device=dev),
    }


def _compare(got, ref, exact_iters, call):
    """Statuses, labels and overload screens exactly (iteration counts too
    when both ran with the same tile width); the FP64 state within the
    parity tests' tolerances."""
    keys = ("status", "label", "n_overload", "overload") + (("iters",) if exact_iters else ())
    for k in keys:
        assert torch_equal(got[k], ref[k]), (call, k)
    ok = ref["status"] == 0
    assert ok.sum().item() > 0
    for k, tol in (("theta", ANGLE_TOL), ("V", ANGLE_TOL), ("flow", 10 * ANGLE_TOL),
                   ("max_loading", 10 * ANGLE_TOL)):
        d = (got[k][ok] - ref[k][ok]).abs().max().item()
        assert d <= tol, (call, k, d)


def torch_equal(a, b):
    return bool((a == b).all().item())


# (workload, precision): FP32 vectors and factors, the scaled FP16 factor,
# FP64, and a grid with reactive limits (the kernel with extension rows)
CASES = [("grid120", 1), ("grid2k", 1), ("grid120", 3), ("grid2k", 2), ("grid120_qlim", 1)]


@pytest.mark.parametrize("name,precision", CASES)
def test_noalloc_matches_regular_screen_twice(name, precision):
    torch = pytest.importorskip("torch")
    import paper_1803_03290_gb300 as gp
    from paper_1803_03290_gb300 import binding
    from gpu_common import grid

    dev = torch.device("cuda", 0)
    g = grid(name)
    c = gp.GPCG(g, precision=precision, tol=1e-10, max_outer=100)
    c.base_solve()
    S = g.n_branch if g.n_branch <= 200 else 300
    outages = torch.arange(S, dtype=torch.int32, device=dev) * (g.n_branch // S)
    ref = _device_outputs(torch, S, g.n_bus, g.n_branch, dev)
    c.n1_screen_device(outages, ref)
    torch.cuda.synchronize()
    lib = binding.load()
    assert hasattr(lib, "gpcg_n1_screen_noalloc")
    for call in range(2):
        got = _device_outputs(torch, S, g.n_bus, g.n_branch, dev)
        c.n1_screen_noalloc_device(outages, got)
        torch.cuda.synchronize()
        _compare(got, ref, True, call)
    c.close()


def test_noalloc_on_a_fresh_context():
    """The no-allocation screen as the context's first screen (no tile
    chosen yet: tiles of 2), then the regular screen: the same statuses,
    labels and overloads, and states within tolerance (iteration counts
    too when the autotuner kept tiles of 2 and the factors' dense tails:
    another tail rounds the inner solve differently)."""
    torch = pytest.importorskip("torch")
    import paper_1803_03290_gb300 as gp
    from gpu_common import grid

    dev = torch.device("cuda", 0)
    g = grid("grid2k")
    c = gp.GPCG(g, tol=1e-10, max_outer=100)
    c.base_solve()
    assert c.info()["tile"] == 0
    S = 256
    outages = torch.arange(S, dtype=torch.int32, device=dev) * (g.n_branch // S)
    got = [_device_outputs(torch, S, g.n_bus, g.n_branch, dev) for _ in range(2)]
    c.n1_screen_noalloc_device(outages, got[0])
    torch.cuda.synchronize()
    before = c.info()
    assert before["tile"] == 0
    ref = _device_outputs(torch, S, g.n_bus, g.n_branch, dev)
    c.n1_screen_device(outages, ref)
    c.n1_screen_noalloc_device(outages, got[1])
    torch.cuda.synchronize()
    after = c.info()
    same = after["tile"] == 2 and all(after[k] == before[k] for k in ("tail_rows_p", "tail_rows_q"))
    _compare(got[0], ref, same, 0)
    _compare(got[1], ref, True, 1)
    c.close()


def test_noalloc_rejects_bad_input():
    torch = pytest.importorskip("torch")
    import paper_1803_03290_gb300 as gp
    from gridgen import config_grid

    g = config_grid("grid120")
    c = gp.GPCG(g)
    c.base_solve()
    dev = torch.device("cuda", 0)
    bad = torch.tensor([0, g.n_branch], dtype=torch.int32, device=dev)
    out = _device_outputs(torch, 2, g.n_bus, g.n_branch, dev)
    with pytest.raises(gp.GPCGError) as e:
        c.n1_screen_noalloc_device(bad, out)
    assert e.value.status == 1
    c.set_options(precision=gp.PLAIN_FP64)
    with pytest.raises(gp.GPCGError):
        c.n1_screen_noalloc_device(bad[:1], out)
    c.close()
