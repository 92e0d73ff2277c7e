"""The bench's N > 1 path on the host, without a GPU: two gloo ranks on CPU.

Every configuration fits one GPU, so N GPUs run N independent replicas (weak scaling, no
data-path collective): the ranks meet only at the barrier around the timed region and at the
max-over-ranks reduction of the timed milliseconds, and the whole-job value counts every rank's
keys over the slowest rank's time.  Each rank draws its own inputs; the reference arm runs on
rank 0 alone.
"""

import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        dist.barrier()
        q.put((rank, slowest, bench.whole_job_gkeys(1 << 20, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r for r, _, _ in got] == [0, 1]
    for _, slowest, value in got:
        assert slowest == 15.0                                 # the max over ranks, on every rank
        assert abs(value - 2 * (1 << 20) / 15e-3 / 1e9) < 1e-12  # both ranks' keys / slowest time


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert abs(bench.whole_job_gkeys(1 << 28, 1, 5.0) - (1 << 28) / 5e-3 / 1e9) < 1e-12


def test_each_rank_sorts_its_own_inputs():
    a0 = bench.make_inputs("uniform_i32_2p20", 0)
    a1 = bench.make_inputs("uniform_i32_2p20", 1)
    assert a0[0][0].shape == a1[0][0].shape and a0[0][0].dtype == a1[0][0].dtype
    assert not np.array_equal(a0[0][0], a1[0][0])


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        workload, steps, warmup, gpus = "uniform_i32_2p20", 1, 0, 2
    bench.run_reference(Args(), rank=1)
    assert capsys.readouterr().out == ""
