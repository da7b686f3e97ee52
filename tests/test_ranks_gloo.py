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
