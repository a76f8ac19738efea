"""The multi-GPU path of the benchmark, on CPU: two gloo ranks.  Each rank
solves its own instance (the units are sharded, not replicated), the job
time is the slowest rank's, the value counts every rank's units, and the
reference arm runs on rank 0 only."""
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


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    inst = bench.make_instance(rank)  # the bench seeds each rank's instance by its rank
    mine = torch.tensor([float(inst["beta"].astype(np.float64).sum())], dtype=torch.float64)
    allv = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allv, mine)
    seconds = 1.0 + 0.5 * rank  # rank 1 is the slow one
    t = bench.max_over_ranks(seconds, world, "cpu")
    value = bench.job_value(world, 3, 10, t)
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([t, value] + [float(v.item()) for v in allv]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 1.5                  # the slowest rank's time
    assert r0[1] == r1[1] == 2 * 3 * 10 / 1.5     # every rank's units
    assert r0[2] != r0[3]                         # distinct instances per rank
    assert (r0[2:] == r1[2:]).all()


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        warmup, steps = 3, 1

    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
