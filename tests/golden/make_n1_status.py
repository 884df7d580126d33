"""Write the oracle's N-1 statuses of the benchmark grids (test fixture).

For every single-branch outage of the named workloads, the oracle's FDPF
(direct solves, FP64) at the screening tolerance of 1e-4 p.u. from the
base-case state; the file keeps the counts and the outages that did not
converge.  Only ``oracle`` and ``gridgen`` are used.

    python tests/golden/make_n1_status.py grid2k grid10k
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from gridgen import config_grid  # noqa: E402
from oracle import powerflow as pf  # noqa: E402
from oracle import screen  # noqa: E402

TOL, MAX_OUTER = 1e-4, 50


def main(names):
    for name in names:
        g = config_grid(name)
        th0, V0, _, st, _ = pf.base_case(g, tol=1e-11, max_outer=200)
        assert st == pf.STATUS_OK
        outages = np.arange(g.n_branch)
        ref = screen.n1_screen(g, th0, V0, outages, tol=TOL, max_outer=MAX_OUTER)
        s = ref["status"]
        bad = np.flatnonzero((s != pf.STATUS_OK) & (s != pf.STATUS_ISLAND_NO_GEN))
        out = dict(workload=name, tol=TOL, max_outer=MAX_OUTER, n_outages=int(outages.size),
                   counts={str(k): int(v) for k, v in zip(*np.unique(s, return_counts=True))},
                   not_converged=[[int(l), int(s[l]), int(ref["outer"][l])] for l in bad],
                   generator="tests/golden/make_n1_status.py")
        with open(os.path.join(HERE, f"{name}_n1_status.json"), "w") as fh:
            json.dump(out, fh, indent=1)
            fh.write("\n")
        print(name, out["counts"], out["not_converged"])


if __name__ == "__main__":
    main(sys.argv[1:] or ["grid2k", "grid10k"])
