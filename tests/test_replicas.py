"""Host logic of the multi-GPU runs on CPU: the LPT split of an uneven batch and the
post-step reduction, with two gloo ranks standing in for two GPUs."""
import itertools
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2607_16906_b300 import replicas, synth


def _optimal_makespan(costs, world):
    best = float("inf")
    for assign in itertools.product(range(world), repeat=len(costs)):
        loads = [0.0] * world
        for c, r in zip(costs, assign):
            loads[r] += c
        best = min(best, max(loads))
    return best


@pytest.mark.parametrize("world", [2, 3])
def test_lpt_within_graham_bound_of_brute_force(world):
    """Graham's bound for LPT: makespan <= (4/3 - 1/(3N)) x the optimum (brute force over all
    assignments of 8 random jobs)."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        costs = list(rng.uniform(1.0, 10.0, 8))
        parts = replicas.lpt_partition(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(8))
        opt = _optimal_makespan(costs, world)
        assert replicas.makespan(costs, parts) <= (4.0 / 3.0 - 1.0 / (3 * world)) * opt + 1e-12


def test_lpt_special_cases():
    assert replicas.lpt_partition([], 2) == [[], []]
    assert replicas.lpt_partition([5.0], 3) == [[0], [], []]
    # equal costs: round-robin by index
    assert replicas.lpt_partition([1.0] * 4, 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        replicas.lpt_partition([1.0], 0)


def test_single_process_reduction_is_identity():
    assert replicas.reduce_step(12.5, 3) == (12.5, 3)


def _uneven_costs():
    probs = synth.uneven_problems(count=16)
    return [float(p.n) for p in probs]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, solved = replicas.reduce_step(100.0 + 10 * rank, 3 + rank)
        parts = replicas.lpt_partition(_uneven_costs(), world)
        mine = parts[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        replicas.barrier()
        out.put((rank, ms, solved, gathered, parts))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_split_and_reduce():
    """Two ranks: step time reduces to the max, solve counts to the sum; each rank computes the
    same LPT split of the 16-system uneven batch without communicating, the parts are disjoint and
    cover the batch."""
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
    costs = _uneven_costs()
    for rank, ms, solved, gathered, parts in res:
        assert ms == 110.0 and solved == 7
        assert gathered == parts
        assert sorted(i for g in gathered for i in g) == list(range(len(costs)))
    # the optimum of the two-way split by enumeration of all 2^16 subsets
    c = np.asarray(costs)
    masks = np.arange(1 << len(c))
    bits = (masks[:, None] >> np.arange(len(c))[None, :]) & 1
    side = bits @ c
    opt = np.max(np.stack([side, c.sum() - side]), axis=0).min()
    assert replicas.makespan(costs, res[0][4]) <= (4.0 / 3.0 - 1.0 / 6.0) * opt + 1e-9
