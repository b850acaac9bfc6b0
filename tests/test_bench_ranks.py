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


def test_reference_arm_takes_the_librarys_table_choice():
    """bench.py's reference arm runs the oracle with the table the library
    picks automatically: compact for stencils (at most six off-diagonals
    within 16383 columns), hybrid for long rows, cumulative for short rows
    that do not fit the compact record."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import synth
    assert bench._auto_table(synth.stencil3d_7pt(6, seed=1)) == 3
    assert bench._auto_table(synth.stencil2d_5pt(8, 8, seed=1)) == 3
    assert bench._auto_table(synth.powerlaw_random(2000, seed=2)) == 2
    # short rows, one column 20000 away: the compact record's offsets do not reach it
    n = 20001
    rows = np.concatenate([np.arange(n), [0]])
    cols = np.concatenate([np.arange(n), [20000]])
    vals = np.concatenate([np.full(n, 4.0), [1.0]])
    assert bench._auto_table(synth._from_coo(n, rows, cols, vals)) == 0


def test_reference_arm_line_on_a_small_workload(capsys):
    """The reference arm prints one JSON line with the oracle's rate on a
    row sample that the warm-up step may re-size but never beyond the
    matrix (here the whole 1024-row matrix fits the time budget)."""
    sys.path.insert(0, ROOT)
    import json
    import bench
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")

    class A:
        workload, steps, warmup, gpus = "stencil2d_32x32", 1, 1, 1
    assert bench.run_reference(A()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "steps/s"
    assert line["config"]["rows_per_step"] == 1024
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
