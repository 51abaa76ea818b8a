"""The multi-rank host logic on the CPU.  A sweep of independent fits shards as whole
fits per rank, placed by greedy LPT: every rank computes the same placement without
communicating, together the ranks cover every fit once, and a step's time is the
slowest rank's (an all-reduce max), as `bench.py --workload 4` does on N GPUs.  The
two-rank case runs as two gloo processes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import gapgen  # noqa: E402
from paper_2207_03803_gb300.sharding import fit_cost, lpt_assign  # noqa: E402


def _sweep_costs():
    recs = gapgen.sweep_recipes()
    return [fit_cost(r.n_cfg + 3 * gapgen.count_shape(r)[0], r.n_sparse[0]) for r in recs]


def test_lpt_assignment_is_greedy_and_deterministic():
    # descending costs, each to the least-loaded rank (lower rank on ties)
    assert lpt_assign([5, 4, 3, 3, 2, 2, 2], 3) == [[0, 5], [1, 4, 6], [2, 3]]
    assert lpt_assign([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    assert lpt_assign([], 2) == [[], []]
    with pytest.raises(ValueError):
        lpt_assign([1.0], 0)
    costs = _sweep_costs()
    for n in (1, 2, 3, 8):
        parts = lpt_assign(costs, n)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # Graham's bound for LPT: at most 4/3 of the optimum, itself at least the mean load
        assert max(loads) <= 4.0 / 3.0 * max(sum(loads) / n, max(costs)) + 1e-9


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = _sweep_costs()
    mine = lpt_assign(costs, world)[rank]
    load = torch.tensor([sum(costs[i] for i in mine)], dtype=torch.float64)
    slowest = load.clone()
    dist.all_reduce(slowest, op=dist.ReduceOp.MAX)
    placed = [None] * world
    dist.all_gather_object(placed, mine)
    q.put((rank, mine, float(load), float(slowest), placed))
    dist.destroy_process_group()


def test_sweep_fits_shard_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, fits0, load0, max0, placed0), (_, fits1, load1, max1, placed1) = res
    assert sorted(fits0 + fits1) == list(range(64))
    assert placed0 == placed1 == [fits0, fits1]
    assert max0 == max1 == max(load0, load1)
