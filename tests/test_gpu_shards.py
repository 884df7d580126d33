"""Partition invariance of the N-1 screen: the outage list split into ragged
shards and screened shard by shard (what ranks do, run in sequence on one
GPU) gives the same results as one call, bit for bit -- a scenario's result
depends only on its own data, not on which tile or slot computes it."""
import numpy as np
import pytest

import paper_1803_03290_gb300 as gp
from gpu_common import grid
from paper_1803_03290_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,world", [("grid2k", 3), ("grid120", 4)])
def test_sharded_screen_is_bit_exact(name, world):
    """The tile width and the dense tail are fixed (they change the rounding
    of the inner solve, and the autotuner may choose them per scenario
    count); the tiles per SM stay with the autotuner, which may give the
    shards and the whole list different numbers of tiles in flight."""
    g = grid(name)
    c = gp.GPCG(g, tile=2, tail_rows=gp.MAX_TAIL_ROWS)
    c.base_solve()
    outages = np.random.default_rng(8).permutation(g.n_branch).astype(np.int32)[:301]
    outs = ("theta", "V", "flow", "label", "iters", "status", "max_loading")
    whole = c.n1_screen(outages, outputs=outs)
    parts = [c.n1_screen(shard.shard_outages(outages, r, world), outputs=outs)
             for r in range(world)]
    for k in outs:
        np.testing.assert_array_equal(np.concatenate([p[k] for p in parts]), whole[k], err_msg=k)
    c.close()


def test_sharded_dc_screen_is_bit_exact():
    g = grid("grid2k")
    c = gp.GPCG(g)
    outages = np.arange(g.n_branch, dtype=np.int32)[::7]
    whole = c.n1_dc_screen(outages)
    parts = [c.n1_dc_screen(shard.shard_outages(outages, r, 3)) for r in range(3)]
    for k in whole:
        np.testing.assert_array_equal(np.concatenate([p[k] for p in parts]), whole[k], err_msg=k)
    c.close()
