"""Edge sharding over ranks: LPT partition properties and the result gather
over two gloo ranks on CPU."""
import os
import socket

import numpy as np
import pytest

from paper_2408_10154_gb300 import shard


def test_lpt_covers_every_edge_once_and_is_balanced():
    rng = np.random.default_rng(7)
    costs = np.exp(rng.uniform(np.log(2e4), np.log(4e5), 32)) * rng.integers(4, 13, 32)
    for m in (1, 2, 3, 4, 8):
        parts = shard.lpt_partition(costs, m)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(32))
        loads = [costs[p].sum() for p in parts]
        # Graham's bound for LPT: max load <= (4/3 - 1/(3m)) OPT, and OPT >= mean load, OPT >= max cost
        opt_lb = max(costs.sum() / m, costs.max())
        assert max(loads) <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt_lb * (1 + 1e-12) or m == 1
        assert shard.lpt_partition(costs, m) == parts  # deterministic


def test_lpt_small_cases():
    assert shard.lpt_partition([], 2) == [[], []]
    assert shard.lpt_partition([5.0], 3) == [[0], [], []]
    # Graham's tight instance: LPT gives loads 7 / 5 where the optimum is 6 / 6,
    # exactly (4/3 - 1/(3m)) OPT for m = 2
    assert shard.lpt_partition([3, 3, 2, 2, 2], 2) == [[0, 2, 4], [1, 3]]
    with pytest.raises(ValueError):
        shard.lpt_partition([1.0], 0)


def test_edge_cost():
    cams = np.zeros((2, 18), np.float32)
    cams[:, 4], cams[:, 5] = 64, 48
    one = np.zeros((1, 18), np.float32)
    one[:, 4], one[:, 5] = 10, 10
    assert shard.edge_cost(100, 50, cams, one) == 100 * 100 + 50 * 2 * 64 * 48


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, costs, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        parts = shard.lpt_partition(costs, world)
        # stand-in for the rank's registrations: a row per owned edge
        local = {i: np.arange(13, dtype=np.float64) * (i + 1) + 0.25 for i in parts[rank]}
        full = shard.gather_results(local, len(costs), 13)
        q.put((rank, parts, full))
    finally:
        dist.destroy_process_group()


def test_gather_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    costs = [float(c) for c in np.random.default_rng(3).uniform(1, 10, 9)]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = np.stack([np.arange(13, dtype=np.float64) * (i + 1) + 0.25 for i in range(9)])
    parts0 = out[0][1]
    assert sorted(parts0[0] + parts0[1]) == list(range(9)) and parts0[0] and parts0[1]
    for _, parts, full in out:
        assert parts == parts0
        np.testing.assert_array_equal(full, want)
