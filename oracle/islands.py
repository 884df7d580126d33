"""Islanding detection by graph traversal (Sec. IV.C).

Test infrastructure (see the package docstring).

An outage removes one edge from the bus/branch graph.  The connected
components of what remains are found by breadth-first search.  Each
component is labelled by the smallest bus index it contains, so labels are
canonical and can be compared exactly.  The main island is the component
that holds the slack bus; every other component is islanded.

Pinned by brute force on small graphs (all single-edge removals, components
from the transitive closure of the adjacency relation) in the tests.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def components(n_bus: int, f: np.ndarray, t: np.ndarray,
               in_service: np.ndarray) -> np.ndarray:
    """Component label (= min bus index of the component) of every bus."""
    adj = [[] for _ in range(n_bus)]
    for e in range(f.shape[0]):
        if in_service[e]:
            adj[int(f[e])].append(int(t[e]))
            adj[int(t[e])].append(int(f[e]))
    label = np.full(n_bus, -1, dtype=np.int32)
    # visiting buses in increasing index order makes the first bus reached
    # in every component its minimum index
    for s in range(n_bus):
        if label[s] >= 0:
            continue
        label[s] = s
        q = deque([s])
        while q:
            u = q.popleft()
            for v in adj[u]:
                if label[v] < 0:
                    label[v] = s
                    q.append(v)
    return label


def island_mask(label: np.ndarray, slack: int) -> np.ndarray:
    """True for buses outside the slack's component."""
    return label != label[slack]
