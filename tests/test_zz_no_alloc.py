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
    }


@pytest.mark.parametrize("name", ["grid120", "grid2k"])
def test_noalloc_matches_regular_screen_twice(name):
    torch = pytest.importorskip("torch")
    import paper_1803_03290_gb300 as gp
    from paper_1803_03290_gb300 import binding
    from gridgen import config_grid

    dev = torch.device("cuda", 0)
    g = config_grid(name)
    c = gp.GPCG(g)
    c.base_solve()
    S = g.n_branch if name == "grid120" else 300
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
        for k in ("status", "iters", "label"):
            assert torch.equal(got[k], ref[k]), (call, k)
        ok = ref["status"] == 0
        for k in ("theta", "V"):
            d = (got[k][ok] - ref[k][ok]).abs().max().item()
            assert d <= ANGLE_TOL, (call, k, d)
        d = (got["flow"][ok] - ref["flow"][ok]).abs().max().item()
        assert d <= 10 * ANGLE_TOL, (call, "flow", d)
        d = (got["max_loading"][ok] - ref["max_loading"][ok]).abs().max().item()
        assert d <= 10 * ANGLE_TOL, (call, "max_loading", d)
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
