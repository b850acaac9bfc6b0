"""The multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1) reduce
their timed milliseconds (max) and steps (sum) the way the benchmark does,
and the reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    bench._init_ranks(world)
    assert dist.get_backend() == "gloo" and dist.get_world_size() == world
    ms, steps = bench._reduce_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1), "cpu")
    with open(f"{out}.{rank}", "w") as f:
        f.write(f"{ms} {steps}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_steps(tmp_path):
    if torch.cuda.is_available():
        pytest.skip("the gloo rank test runs on hosts without a GPU")
    port = _free_port()
    out = str(tmp_path / "rank")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        ms, steps = map(float, open(f"{out}.{r}").read().split())
        assert ms == 150.0 and steps == 3000.0


def test_single_rank_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    assert bench._reduce_ranks(12.5, 7, "cpu") == (12.5, 7.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup, gpus = "stencil3d_64", 1, 1, 2
    assert bench.run_reference(A()) == 0
