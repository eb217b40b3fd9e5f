"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1).

Every rank runs its own walkers (weak scaling, no collective on the data
path); the job's time is the slowest rank's, and the reported value is the
walker-steps of all ranks per second of that time.  The reference arm runs on
rank 0 only.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_2408_14070_gb300 import inputs as I
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = [12.5, 20.0][rank]
    worst = bench.max_over_ranks(dist, local_ms, "cpu")
    rate = bench.whole_job_rate(1024, world, 200, worst / 1e3)
    sp = I.make_system(22, 2, bench.rank_seed(rank))
    x0 = I.make_chains(4, sp, bench.rank_seed(rank))
    dist.barrier()
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), worst=worst, rate=rate, x0=x0)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_shard_walkers(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0, r1 = (np.load(tmp_path / f"r{k}.npz") for k in range(2))
    assert float(r0["worst"]) == float(r1["worst"]) == 20.0
    assert float(r0["rate"]) == pytest.approx(1024 * 2 * 200 / 0.020)
    assert not np.array_equal(r0["x0"], r1["x0"])     # each rank its own walkers


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        steps, warmup, gpus = 2, 1, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
