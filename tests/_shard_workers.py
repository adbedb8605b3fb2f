"""Rank bodies for the sharding tests (spawned CPU processes on the gloo backend)."""
import datetime
import os


def _init(rank, world, port, timeout_s=20):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=timeout_s))
    return dist


def fake_scene_result(i):
    """Stands in for one scene's adjoint: per-scene output and its share of a global gradient."""
    return {"per_scene": [float(i), float(i * i)], "shared": [1.0 * i, 2.0, -0.5 * i]}


def body(rank, world, port, costs, mode, q):
    import torch
    from paper_2603_16478_gb300.shard import ShardLost, allreduce_shared, run_sharded
    dist = _init(rank, world, port, timeout_s=10 if mode == "lost_rank" else 20)
    try:
        def run(items):
            if mode == "fail" and rank == 1:
                raise RuntimeError("NOT_CONVERGED in this rank's batch")
            return {i: fake_scene_result(i) for i in items}

        if mode == "lost_rank" and rank == 1:
            os._exit(3)  # leaves before the gather, between steps: nothing of it is in flight
        try:
            res, shards = run_sharded(costs, run)
        except ShardLost as e:
            q.put((rank, "lost", e.missing, None, None))
            return
        except Exception as e:  # the collective itself failed (a rank left)
            q.put((rank, "collective_error", type(e).__name__, None, None))
            return
        shared = torch.zeros(3, dtype=torch.float64)
        for i in shards[rank]:
            shared += torch.tensor(res[i]["shared"], dtype=torch.float64)
        allreduce_shared(shared)
        q.put((rank, "ok", {k: v["per_scene"] for k, v in res.items()}, shards, shared.tolist()))
    finally:
        if not (mode == "lost_rank"):
            dist.destroy_process_group()
