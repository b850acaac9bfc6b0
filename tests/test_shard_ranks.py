"""Row sharding of one build over ranks (Sec. IV-A): the partition, and the
gather of the ranks' CSR pieces, on two gloo ranks on the CPU (127.0.0.1).
Each rank computes its row range with the oracle (the CUDA build of a row
range is compared with the one-range build on the GPU in
test_gpu_parity.py); the gathered matrix must equal the one-rank build bit
for bit."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2409_03095_b300.shard import gather_csr, partition_rows  # noqa: E402


def test_partition_rows_even_and_weighted():
    assert partition_rows(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert partition_rows(2, 4) == [(0, 0), (0, 1), (1, 1), (1, 2)]
    assert partition_rows(0, 2) == [(0, 0), (0, 0)]
    w = np.array([1, 1, 1, 1, 10, 1, 1, 1], dtype=float)
    parts = partition_rows(len(w), 2, w)
    assert parts[0][0] == 0 and parts[-1][1] == len(w) and parts[0][1] == parts[1][0]
    # the heavy row ends the first half of the weight
    assert parts[0][1] == 5
    for world in (1, 2, 3, 7):
        for wts in (None, np.random.default_rng(world).random(50)):
            p = partition_rows(50, world, wts)
            assert p[0][0] == 0 and p[-1][1] == 50
            assert all(a[1] == b[0] for a, b in zip(p, p[1:])) and all(b >= a for a, b in p)
    with pytest.raises(ValueError):
        partition_rows(5, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import synth
    return synth.random_dd(301, 7, seed=12, diag_sign="mixed", dominance=0.85)


KW = dict(chains=64, max_len=64, delta=1e-3, seed=5, tau=2e-2, top_k=0, table=2)


def _rank_main(rank, world, port, out, weighted):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    m = _case()
    wts = np.diff(m.row_ptr) if weighted else None
    b, e = partition_rows(m.n, world, wts)[rank]
    rp, col, val, _ = oracle.build(m, rows=np.arange(b, e), **KW)
    g_rp, g_col, g_val = gather_csr(torch.from_numpy(rp.astype(np.int64)), torch.from_numpy(col.astype(np.int32)),
                                    torch.from_numpy(val), None)
    np.savez(f"{out}.{rank}.npz", rp=g_rp.numpy(), col=g_col.numpy(), val=g_val.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("weighted", [False, True])
def test_two_gloo_ranks_gather_the_one_rank_build(tmp_path, weighted):
    if torch.cuda.is_available():
        pytest.skip("the gloo rank test runs on hosts without a GPU")
    import oracle
    port = _free_port()
    out = str(tmp_path / "shard")
    mp.start_processes(_rank_main, args=(2, port, out, weighted), nprocs=2, join=True, start_method="spawn")
    rp, col, val, _ = oracle.build(_case(), **KW)
    for r in range(2):
        g = np.load(f"{out}.{r}.npz")
        assert np.array_equal(g["rp"], rp.astype(np.int64))
        assert np.array_equal(g["col"], col.astype(np.int32))
        assert np.array_equal(g["val"], val)
