"""Host logic of the multi-GPU path on CPU: the systems of a batch split over
two gloo ranks (each computes the same assignment locally), and the timing
max over ranks."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

import sg_inputs as S

# loaded by path: the sharding logic is pure host code and needs no built library
_spec = importlib.util.spec_from_file_location(
    "sghsc_shard", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                "paper_1205_1864_gb300", "shard.py"))
shard = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(shard)


def _costs():
    return [shard.system_cost(c["ne"], c["M"], c["p"]) for c in S.draw_batch_configs(64, seed=1864)]


def test_assign_is_a_balanced_partition():
    costs = _costs()
    for world in (1, 2, 3, 4, 8):
        parts = shard.assign(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: no rank exceeds the lightest by more than the largest item
        assert max(loads) - min(loads) <= max(costs) + 1e-9
    assert shard.assign([], 2) == [[], []]
    with pytest.raises(ValueError):
        shard.assign(costs, 0)


def test_cost_grows_with_each_size():
    assert shard.system_cost(64, 4, 3) > shard.system_cost(32, 4, 3)
    assert shard.system_cost(64, 5, 3) > shard.system_cost(64, 4, 3)
    assert shard.system_cost(64, 4, 4) > shard.system_cost(64, 4, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.my_systems(_costs(), rank, world)
        got = [None] * world
        dist.all_gather_object(got, mine)
        tmax = shard.max_over_ranks(10.0 + rank)
        q.put((rank, got, tmax))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_disjoint_cover():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = len(_costs())
    for rank, got, tmax in res:
        assert tmax == 11.0
        assert got == shard.assign(_costs(), world)
        assert sorted(got[0] + got[1]) == list(range(n))
        assert not set(got[0]) & set(got[1])
