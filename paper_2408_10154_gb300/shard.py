"""Sharding of independent registration problems over ranks (one process
per GPU).  Loop edges are independent (Sec. 3.2 estimates every keyframe
transform in parallel; Eq. 7 fuses only the estimates of one edge), so a
rank owns whole edges, both directions included, and fuses them itself:
no data crosses ranks while registering.  The only exchange is the result
gather (12 + 1 floats per edge) after the batch.

Edges are balanced by their rendering work with the longest-processing-time
greedy rule; the work of one direction is the moving submap's size times
the pixels it is rendered at."""
from __future__ import annotations

import heapq

import numpy as np


def edge_cost(n_src: int, n_tgt: int, src_cams, tgt_cams) -> float:
    """Work of one loop edge in both directions: src is moved and rendered at
    the target keyframes, tgt at the source keyframes."""
    px = lambda cams: float(sum(int(c[4]) * int(c[5]) for c in cams))
    return float(n_src) * px(tgt_cams) + float(n_tgt) * px(src_cams)


def lpt_partition(costs, n_ranks: int):
    """Longest-processing-time greedy: edges in decreasing cost (ties by
    index), each to the currently least-loaded rank (ties by rank).  Returns
    one ascending index list per rank.  Deterministic, so every rank computes
    the same partition without communicating."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    costs = [float(c) for c in costs]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(n_ranks)]
    parts = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def gather_results(local: dict, n_total: int, width: int, device="cpu"):
    """Every rank contributes the rows it owns ({edge index: row of
    ``width`` numbers}); returns the full [n_total, width] float64 array on
    every rank.  One all-reduce of a zero-filled table: rows are owned by
    exactly one rank, so the sum is exact."""
    import torch
    import torch.distributed as dist
    t = torch.zeros((n_total, width), dtype=torch.float64, device=device)
    for i, row in local.items():
        t[int(i)] = torch.as_tensor(np.asarray(row, np.float64).reshape(width), device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t)
    return t.cpu().numpy()
