"""Partition of a batch of independent instances over ranks (one GPU per rank).

Instances of a batch share nothing (each is its own all-at-once system), so a multi-GPU batched
solve needs no collective on the data path: every rank solves the instances assigned to it, and
only the timing (a barrier and the slowest rank's time) crosses ranks.  The paper notes that its
preconditioner is parallelisable over processors (Sec. 1, after eq. def:matrix_P); between
independent instances the split is complete.

Assignment is greedy largest-first (longest processing time first): instances sorted by cost,
each given to the rank with the smallest load so far (ties to the lowest rank, then by instance
index, so every rank computes the same partition without communicating).  With cost c_i, total C
and P ranks, the largest load is at most C/P + max_i c_i.

Cost of an instance = space-time unknowns x estimated MINRES iterations.  The iteration estimate
is a per-scheme constant measured on the batch workload's instance mix; with the preconditioner of
Sec. 3.1.1 the count does not grow with n (Sec. 3.1.2), so the unknowns carry the size dependence.
"""
from __future__ import annotations

from typing import List, Sequence

# mean MINRES iterations to a true relative residual of 1e-8 (mixed precision, float32
# preconditioner in float64 refinement) per time scheme, measured on the 64-instance batch
# workload (one GB300): 80 at theta = 1/2 (36 instances), 57 at theta = 1 (28 instances)
EST_ITERATIONS = {0.5: 80.0, 1.0: 57.0}


def instance_cost(unknowns: int, theta: float = 1.0, est_iterations=None) -> float:
    est = EST_ITERATIONS if est_iterations is None else est_iterations
    return float(unknowns) * float(est.get(float(theta), 70.0))


def partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Instance indices per rank (each list ascending); every index appears exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    loads = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += float(costs[i])
    return [sorted(p) for p in parts]


def loads(costs: Sequence[float], parts: Sequence[Sequence[int]]) -> List[float]:
    return [sum(float(costs[i]) for i in p) for p in parts]


__all__ = ["EST_ITERATIONS", "instance_cost", "partition", "loads"]
