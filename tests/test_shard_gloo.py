"""Multi-rank path on the CPU: group sharding and the benchmark's max-over-ranks timing,
run as two gloo processes (world size 2, rendezvous on 127.0.0.1)."""
import os
import socket

import numpy as np
import pytest

from paper_2511_12894_gb300 import shard


def test_assign_covers_every_group_once_and_balances():
    rng = np.random.default_rng(0)
    costs = list(rng.uniform(1, 10, 37))
    for world in (1, 2, 3, 8):
        parts = shard.assign(costs, world)
        flat = sorted(g for p in parts for g in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[g] for g in p) for p in parts]
        # LPT bound: no rank exceeds the mean by more than the largest single cost
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9


def test_assign_edge_cases():
    assert shard.assign([], 2) == [[], []]
    assert shard.assign([5.0], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        shard.assign([1.0], 0)
    with pytest.raises(ValueError):
        shard.my_groups([1.0], 2, 2)


def test_group_cost_grows_with_kernel_length():
    n = 1 << 20
    assert shard.group_cost(n, [1000] * 10) < shard.group_cost(n, [40000] * 10)
    assert shard.group_cost(n, [1000] * 10) < shard.group_cost(n, [1000] * 20)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, costs, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.my_groups(costs, world, rank)
    # every rank works on its own groups; the elapsed time is reduced with MAX as in bench.py
    local_ms = torch.tensor([10.0 * (rank + 1) + sum(costs[g] for g in mine)], dtype=torch.float64)
    dist.all_reduce(local_ms, op=dist.ReduceOp.MAX)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    q.put((rank, mine, float(local_ms.item()), gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_overlap_and_reduce_max():
    import torch.multiprocessing as mp
    costs = [3.0, 1.0, 4.0, 1.5, 9.0, 2.6, 5.0]
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    mine = [r[1] for r in res]
    assert sorted(mine[0] + mine[1]) == list(range(len(costs)))
    assert not set(mine[0]) & set(mine[1])
    expect_max = max(10.0 * (r + 1) + sum(costs[g] for g in mine[r]) for r in range(world))
    assert all(abs(r[2] - expect_max) < 1e-9 for r in res)
    assert res[0][3] == res[1][3] == mine


def test_split_neighbours_covers_each_once():
    for k in (0, 1, 5, 16, 257):
        for world in (1, 2, 3, 8):
            runs = [shard.split_neighbours(k, world, r) for r in range(world)]
            flat = [j for run in runs for j in run]
            assert flat == list(range(k))
            assert max(len(r) for r in runs) - min(len(r) for r in runs) <= 1
    with pytest.raises(ValueError):
        shard.split_neighbours(4, 2, 2)


def test_global_rows_follow_group_order():
    sizes = [3, 0, 2, 4]
    assert shard.global_rows(sizes, [0, 1, 2, 3]) == list(range(9))
    assert shard.global_rows(sizes, [3, 0]) == [5, 6, 7, 8, 0, 1, 2]
    assert shard.global_rows(sizes, [1]) == []


def _synthetic_peaks(rows, nw):
    # per-row window peaks that identify their global row and window
    import torch
    r = torch.as_tensor(rows, dtype=torch.float32).reshape(-1, 1)
    w = torch.arange(nw, dtype=torch.float32).reshape(1, -1)
    P = 1000.0 * r + w
    A = (10000 * r + w).to(torch.int32)
    return P.reshape(len(rows), nw), A.reshape(len(rows), nw)


def _gather_worker(rank, world, port, sizes, costs, nw, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assign = shard.assign(costs, world)
    mine = assign[rank]
    # each rank's window peaks of its own references and neighbours, in its own order
    ref_rows = [list(a) for a in assign]
    nb_rows = [shard.global_rows(sizes, a) for a in assign]
    Pr, Ar = _synthetic_peaks(mine, nw)
    Pn, An = _synthetic_peaks(shard.global_rows(sizes, mine), nw)
    out = [shard.gather_rows(t, rows, total, rank, world, dist)
           for t, rows, total in ((Pr, ref_rows, len(sizes)), (Ar, ref_rows, len(sizes)),
                                  (Pn, nb_rows, sum(sizes)), (An, nb_rows, sum(sizes)))]
    q.put((rank, None if rank else [o.numpy() for o in out]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_window_peaks_in_row_order():
    """Sharded groups computed on two ranks and gathered to rank 0 give the single-process
    arrays: references in group order, then every group's neighbours in group order."""
    import torch.multiprocessing as mp
    sizes = [3, 5, 0, 2, 4, 1, 6]
    costs = [float(1 + k) for k in sizes]
    nw = 7
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, sizes, costs, nw, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res[1] is None
    Pr, Ar, Pn, An = res[0]
    eP, eA = _synthetic_peaks(list(range(len(sizes))), nw)
    assert np.array_equal(Pr, eP.numpy()) and np.array_equal(Ar, eA.numpy())
    eP, eA = _synthetic_peaks(list(range(sum(sizes))), nw)
    assert np.array_equal(Pn, eP.numpy()) and np.array_equal(An, eA.numpy())
    # the two ranks really held different groups
    a = shard.assign(costs, world)
    assert a[0] and a[1] and not set(a[0]) & set(a[1])
