"""One mesh on several GPUs by source partition.

u is linear in the sources: u(r_i) = sum over tets t of the potential of t's
charges (Eq. (2)).  So the source tets are split into R contiguous ranges of
their centroids' Morton order (compact pieces of the domain, balanced by tet
count); rank k builds a plan of its own tets over all nodes -- nodes its tets
do not reference still receive u -- evaluates u at every node, and one
all-reduce (sum) of u over the ranks gives the potential of the whole mesh.
Each rank's far field is the FMM of its own sources (its own octree), its near
field the analytic integrals of its own tets, so the only exchange is the
all-reduce of N_n x B values; the mass-lumped H (Sec. 4.1) then needs u on the
one-ring of a node, which every rank holds after the all-reduce.

This module holds the host logic (partition, reduction); the evaluation of a
shard is the library's demag_eval."""
from __future__ import annotations

import numpy as np


def morton_partition(nodes, tets, nshards):
    """Tet index arrays of `nshards` shards: the tets sorted by the Morton key
    (21 bits per axis in the bounding cube) of their centroid, cut into
    contiguous ranges of equal count (the last ones one shorter)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    if nshards < 1:
        raise ValueError("nshards must be >= 1")
    cen = nodes[tets].mean(axis=1)
    lo = nodes.min(axis=0)
    side = float((nodes.max(axis=0) - lo).max()) * (1.0 + 2.0 ** -20)
    q = np.minimum(((cen - lo) * (2.0 ** 21 / side)).astype(np.uint64), np.uint64(2 ** 21 - 1))
    key = np.zeros(len(tets), dtype=np.uint64)
    for b in range(21):
        for a in range(3):
            key |= ((q[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    order = np.argsort(key, kind="stable")
    return [np.sort(part) for part in np.array_split(order, nshards)]


def allreduce_u(u, group=None):
    """Sum of the ranks' partial potentials (torch.distributed, in place)."""
    import torch.distributed as dist

    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return u
