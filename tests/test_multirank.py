"""Host logic of the N > 1 benchmark path, on CPU ranks over gloo.

With several GPUs every rank builds its own replica scene (independent units,
no data exchange), and the job's time is the slowest rank's. These tests run
two gloo ranks on the CPU and check the pieces bench.py uses for that: the
max-over-ranks reduction, the whole-job throughput, and that the replica scenes
of different ranks are different, seeded, reproducible inputs.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    from paper_1503_06029_gb300 import inputs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench._dist()
    assert (w, r, local) == (world, rank, rank)
    seconds = 0.5 + rank  # rank 1 is the slow one
    slowest = bench.max_over_ranks(seconds, dist, "cpu")
    value = bench.job_value(world, 1000, slowest)
    sc = inputs.planes_3d(n=256, ell=16, seed=2 + rank)
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([slowest, value, float(sc.pts.astype(np.int64).sum())]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [np.load(tmp_path / f"r{r}.npy") for r in range(world)]
    for r in res:
        assert r[0] == pytest.approx(1.5)  # max(0.5, 1.5)
        assert r[1] == pytest.approx(world * 1000 / 1.5 / 1e6)
    assert res[0][2] != res[1][2]  # replica scenes differ between ranks
    from paper_1503_06029_gb300 import inputs

    for r in range(world):
        assert res[r][2] == float(inputs.planes_3d(n=256, ell=16, seed=2 + r).pts.astype(
            np.int64).sum())


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_value(1, 2_000_000, 0.5) == pytest.approx(4.0)


def test_host_description_names_the_cpu():
    sys.path.insert(0, ROOT)
    import bench

    h = bench.host_description()
    assert set(h) == {"machine", "model", "logical_cores"}
    assert h["logical_cores"] >= 1 and h["machine"]
