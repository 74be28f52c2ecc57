"""Host logic of bench.py's N > 1 launch (one process per GPU, independent
replicas, no data-path collective): the slowest rank's time is taken on every
rank, the whole-job rate sums the ranks' units over it, and the reference arm
runs on rank 0 only.  Two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 10.0 + 5.0 * rank                    # rank 1 is the slow one
        dist.barrier()
        ms_max = bench.max_over_ranks(my_ms, world, device="cpu")
        rate = bench.whole_job_rate(1000.0, world, ms_max / 1e3)
        out[rank] = (ms_max, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1]
    ms_max, rate = out[0]
    assert ms_max == 15.0
    assert rate == pytest.approx(2 * 1000.0 / 0.015)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = bench.parse.__globals__["argparse"].Namespace(workload="acoustics3d", steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
