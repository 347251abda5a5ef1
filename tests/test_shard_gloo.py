"""Multi-rank path on the CPU: two gloo ranks split the 16 slices of the
12-qubit workload into disjoint blocks, sum their blocks with the FP64 oracle
and add the partial sums with one all-reduce; every rank must end with the
unsliced contraction. Also checks that the block dealing covers every slice
exactly once."""

import os
import socket

import numpy as np
import pytest

from paper_2205_00393_gb300.shard import rank_blocks, sharded_sum, step_range

torch = pytest.importorskip("torch")


def test_rank_blocks_cover_each_slice_once():
    for lo, hi, per_call, world in [(0, 16, 2, 2), (3, 40, 3, 4), (0, 5, 8, 3), (7, 7, 2, 2)]:
        seen = []
        for r in range(world):
            for a, b in rank_blocks(lo, hi, per_call, world, r):
                assert lo <= a < b <= hi and b - a <= per_call
                seen.extend(range(a, b))
        assert sorted(seen) == list(range(lo, hi))
    assert step_range(3, 2, 1, 2, 16) == (14, 16)
    assert step_range(4, 2, 0, 2, 16) == (0, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from tnc_inputs import circuit_to_network, grid_rqc
    from oracle import planner, tn
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = grid_rqc(3, 4, 8, 1)
        net = circuit_to_network(c)
        path = planner.greedy_path(net.indices, net.dims)
        tree = planner.Tree(net.indices, net.dims, net.open_ids, path)
        S = planner.find_slices(tree, 8, 7)

        def contract(a, b):
            return tn.contract(net, path, S, slices=range(a, b)) if b > a else np.zeros(1, np.complex128)
        total = sharded_sum(contract, 0, 1 << len(S), 3, world, rank)
        ref = tn.contract(net, path)
        q.put((rank, float(np.max(np.abs(total - ref))), float(np.max(np.abs(ref)))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_full_contraction():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=5) for _ in procs)
    for rank, diff, scale in res:
        assert diff <= 1e-12 * scale, (rank, diff, scale)
