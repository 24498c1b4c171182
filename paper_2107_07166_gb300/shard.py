"""Sharding of a batch of independent systems across ranks.

Systems are independent, so a batch splits across ranks with no exchange on the data
path: every rank builds and evaluates its own systems.  The split is a greedy
longest-processing-time partition on the cost N log N of a system (the tree's depth times
its size), a fixed function of the sizes: every rank computes the same partition on its
own, with no communication.
"""
import numpy as np


def system_cost(sizes):
    """Cost model of one system: N log2 N (at least N)."""
    n = np.asarray(sizes, dtype=np.float64)
    return n * np.log2(np.maximum(n, 2.0))


def lpt_partition(sizes, n_parts: int):
    """Systems of sizes[] into n_parts groups: systems in decreasing cost (ties: lower
    index) each go to the group of least cost so far (ties: lower group).  Returns the
    groups' system indices, each increasing."""
    if n_parts < 1:
        raise ValueError("n_parts must be at least 1")
    cost = system_cost(sizes)
    order = sorted(range(len(cost)), key=lambda i: (-cost[i], i))
    load = [0.0] * n_parts
    parts = [[] for _ in range(n_parts)]
    for i in order:
        g = min(range(n_parts), key=lambda j: (load[j], j))
        parts[g].append(i)
        load[g] += cost[i]
    return [np.array(sorted(p), dtype=np.int64) for p in parts]
