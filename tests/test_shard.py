"""Sharding a batch of independent scenes across ranks: LPT planning, the gather of per-scene
results, the all-reduce of shared parameter gradients, and what the other ranks see when a
shard fails or a rank leaves.  CPU ranks on the gloo backend (world size 2); the per-scene
solve is a stand-in, since only the host-side plumbing is under test."""
import multiprocessing as mp
import queue
import socket

import numpy as np
import pytest

from paper_2603_16478_gb300.shard import plan_shards, scene_cost
from tests import _shard_workers as W


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run(world, costs, mode, timeout=60):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=W.body, args=(r, world, port, costs, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    expected = world - (1 if mode == "lost_rank" else 0)
    try:
        for _ in range(expected):
            r = q.get(timeout=timeout)
            out[r[0]] = r[1:]
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    return out, procs


def test_lpt_plan_covers_every_scene_once_and_balances():
    rng = np.random.default_rng(0)
    costs = list(rng.lognormal(0, 1, size=64))
    for world in (1, 2, 3, 8):
        shards = plan_shards(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(64))
        loads = [sum(costs[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(costs) + 1e-12
        assert shards == plan_shards(costs, world)  # deterministic
    # textbook LPT example: 5 jobs on 2 machines
    assert plan_shards([3, 3, 2, 2, 2], 2) == [[0, 2, 4], [1, 3]]
    assert scene_cost(1000, 50000, 100) > scene_cost(1000, 50000, 0)


def test_two_ranks_gather_every_scene_and_sum_the_shared_gradient():
    costs = [5.0, 1.0, 4.0, 2.0, 3.0, 7.0, 0.5]
    out, _ = _run(2, costs, "ok")
    assert set(out) == {0, 1}
    ref = {i: W.fake_scene_result(i)["per_scene"] for i in range(len(costs))}
    shared_ref = np.sum([W.fake_scene_result(i)["shared"] for i in range(len(costs))], axis=0)
    for r in (0, 1):
        status, res, shards, shared = out[r]
        assert status == "ok"
        assert {int(k): v for k, v in res.items()} == ref
        assert shards == plan_shards(costs, 2)
        assert np.allclose(shared, shared_ref)


def test_a_failed_shard_is_reported_to_every_rank():
    costs = [5.0, 1.0, 4.0, 2.0, 3.0]
    out, _ = _run(2, costs, "fail")
    lost = plan_shards(costs, 2)[1]
    for r in (0, 1):
        status, missing, _, _ = out[r]
        assert status == "lost" and missing == lost


def test_a_rank_that_leaves_makes_the_next_collective_fail_on_the_others():
    costs = [5.0, 1.0, 4.0, 2.0]
    out, procs = _run(2, costs, "lost_rank", timeout=90)
    status, err, _, _ = out[0]
    assert status == "collective_error", out[0]
    assert procs[1].exitcode == 3
