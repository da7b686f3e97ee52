"""The benchmark's multi-rank host logic on CPU: two gloo ranks (world size 2), each with its
own independent replica of the workload (no data-path exchange; the only collectives are the
timing reductions): the whole-job time is the slowest rank's, the iteration count the sum."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # ragged per-rank numbers: the slower rank sets the job's time
        ms, iters = bench.reduce_over_ranks(dist, "cpu", [80.0, 95.5][rank], [200, 150][rank])
        geom, x_true, case = bench.workload(rank)
        digest = float(np.sum(x_true * np.arange(x_true.size).reshape(x_true.shape) % 7))
        out[rank] = (ms, iters, geom.n, geom.m, digest)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_iterations():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:     # no fork of a multi-threaded process
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in (0, 1):
        ms, iters, n, m, _ = res[r]
        assert ms == 95.5 and iters == 350.0       # the same whole-job numbers on every rank
        assert (n, m) == (512 * 512, 720 * 768)
    assert res[0][4] != res[1][4]                  # each rank solves its own problem


def test_one_process_needs_no_collective():
    import bench
    assert bench.reduce_over_ranks(None, "cpu", 12.5, 7) == (12.5, 7.0)


def test_reference_arm_other_ranks_do_no_work(capsys):
    """Under torchrun only rank 0 runs and prints the reference arm; the others exit at once."""
    import bench
    assert bench.bench_reference(None, 1, 2) is None
    assert capsys.readouterr().out == ""


def _slices_rank_main(rank, world, port, out):
    """Each gloo rank computes its own share of the 256-slice batch (no communication) and the
    ranks then gather the shares to check them against each other."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        cases = synth.batched_slices(256, seed=7)
        works = [bench.slice_work(c["geom"], 60) for c in cases]
        mine = bench.partition_slices(works, world)[rank]
        shares = [None] * world
        dist.all_gather_object(shares, (mine, sum(works[i] for i in mine)))
        out[rank] = (shares, works)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slice_batch_partition_over_gloo_ranks(world):
    """--workload slices: every slice is solved by exactly one rank, every rank computes the
    same partition, and the heaviest rank carries at most total / world + the largest slice."""
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_slices_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    shares0, works = res[0]
    for r in range(world):
        assert res[r][0] == shares0                # the same answer on every rank
    idx = sorted(i for part, _ in shares0 for i in part)
    assert idx == list(range(256))                 # each slice exactly once
    loads = [w for _, w in shares0]
    assert max(loads) <= sum(works) / world + max(works)
    assert max(loads) / (sum(works) / world) < 1.02    # and close to even on this batch


def test_partition_edge_cases():
    import bench
    assert bench.partition_slices([5, 3], 1) == [[0, 1]]
    assert bench.partition_slices([1, 1, 1], 4) == [[0], [1], [2], []]
    assert bench.partition_slices([], 2) == [[], []]
    assert bench.partition_slices([10, 1, 1, 8], 2) == [[0], [1, 2, 3]]


def test_rank_launch_is_checked_against_gpus():
    import bench
    assert bench.check_ranks(1, {}) is None
    assert bench.check_ranks(4, {"WORLD_SIZE": "4"}) is None
    assert "torch.distributed.run" in bench.check_ranks(8, {})
    assert "does not match" in bench.check_ranks(2, {"WORLD_SIZE": "4"})
    assert bench.check_ranks(0, {}) is not None
