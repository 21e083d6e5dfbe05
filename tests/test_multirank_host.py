"""The benchmark's multi-rank logic on CPU: two gloo ranks (world size 2) on
127.0.0.1. Every rank runs its own instance (weak scaling, no collective in the
data path); the only collective is the max over ranks of the timings, and rank
0 alone reports. The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r measured (r + 1) ms and (5 - r) s: the maximum wins element-wise
    got = bench.reduce_max([rank + 1.0, 5.0 - rank], device="cpu")
    value = bench.whole_job_value(world, 1000.0, got[0] * 1e-3)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{got[0]} {got[1]} {value}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        a, b, v = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert (a, b) == (2.0, 5.0)
        # 2 ranks x 1000 units in the slowest rank's 2 ms
        assert v == pytest.approx(2 * 1000.0 / 2e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup = "cellular32", 1, 0
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""


def test_world_size_one_is_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([3.0, 1.5]) == [3.0, 1.5]
