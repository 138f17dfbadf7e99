"""The multi-process path of bench.py on CPU: two gloo ranks run independent
replicas (no data-path collective); the timing reduction takes the max over
ranks and the throughput the sum, as the benchmark reports them."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    t_max = bench.max_over_ranks(10.0 + rank, w)
    v_sum = bench.sum_over_ranks(100.0 * (rank + 1), w)
    bench.barrier(w)
    out[rank] = (t_max, v_sum)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_replica_reductions():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (11.0, 300.0)


def _oracle_leg(rank, world, port, out):
    """The reference arm under two ranks: rank 0 alone times the oracle."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import argparse
    import bench
    import ed_inputs as ei
    args = argparse.Namespace(gpus=world, steps=2, warmup=1)
    line = bench.run_reference(args, ei.workload("ring16"), budget_s=1.0)
    out[rank] = None if line is None else (line["impl"], line["unit"], line["value"] > 0,
                                           line["e2e"]["h2d_bytes_per_step"])
    import torch.distributed as dist
    dist.destroy_process_group()


def test_reference_arm_rank_zero_only():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_oracle_leg, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[1] is None
    assert res[0] == ("reference", "rows/s", True, 0)


def test_bench_roofline_op_count():
    """The algorithmic INT32 count the benchmark divides by the launch time:
    N=32 ring with reflection and spin inversion = 2 cosets x 32 rotations x
    (1 funnel shift + min + max) + 1 reversal + 1 final complement."""
    import bench
    assert bench.search_ops_per_term(32, 64, True, True, 32, 2, [0, 1]) == 2 * 32 * 3 + 1 + 1
    # generic search: 64 permutations x (36-op Benes + complement + 2 mins)
    assert bench.search_ops_per_term(32, 64, True, False, 1, 0, []) == 64 * 39
