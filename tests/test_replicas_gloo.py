"""The multi-GPU form of the benchmark is N replicas (one view per rank, no exchange
step on the data path): its host logic under two gloo ranks on the CPU."""
import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2507_20239_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 1.5 + rank                      # rank 1 is the slower one
        slow = replicas.slowest(ms)
        rate = replicas.job_rate(1, replicas.world(), slow)
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"slowest": slow, "rate": rate, "world": replicas.world()}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time_and_the_whole_job_rate(tmp_path):
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        with open(tmp_path / f"r{r}.json") as f:
            assert json.load(f) == {"slowest": 2.5, "rate": 800.0, "world": 2}


def test_one_rank_without_a_process_group():
    assert replicas.world() == 1
    assert replicas.slowest(3.25) == 3.25
    assert replicas.job_rate(4, 1, 2.0) == 2000.0
    with pytest.raises(ValueError):
        replicas.job_rate(1, 1, 0.0)


def test_each_rank_renders_its_own_view_of_the_same_scene():
    import bench
    s0, s1 = bench.make_scene(2_000, 0), bench.make_scene(2_000, 1)
    p0, p1 = s0.params(), s1.params()
    for k in p0:
        assert np.array_equal(p0[k], p1[k]), k
    c0, c1 = s0.cameras[0], s1.cameras[0]
    assert (c0.width, c0.height) == (c1.width, c1.height)
    assert not np.allclose(np.asarray(c0.R), np.asarray(c1.R))
