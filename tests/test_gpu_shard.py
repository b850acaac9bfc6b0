"""Row sharding on the GPU: the CSR pieces of row-range builds, concatenated
in order, are the one-range build bit for bit (the kernel half of the
sharded build; the gather over ranks is covered on gloo ranks on the CPU),
and build_sharded on a one-rank NCCL group returns the plain build."""
import os
import socket

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402
from paper_2409_03095_b300.shard import build_sharded, partition_rows  # noqa: E402


def _csr(M):
    return [t.cpu().numpy() for t in M.to_torch()]


@pytest.mark.parametrize("name", ["powerlaw", "stencil"])
def test_row_range_pieces_concatenate_to_the_full_build(name):
    if name == "powerlaw":
        m = synth.powerlaw_random(20000, seed=8)
        p = mc.params(chains=128, max_len=256, delta=1e-3, filter_tau=5e-3, seed=3)
    else:
        m = synth.stencil3d_7pt(24, seed=8)
        p = mc.params(chains=256, max_len=128, delta=1e-2, top_k=16, seed=3)
    B = mc.DeviceCsr.from_host(m)
    full = _csr(mc.mcmi_build_ex(B, p))
    for world, wts in ((2, None), (3, np.diff(m.row_ptr))):
        rps, cols, vals = [], [], []
        for b, e in partition_rows(m.n, world, wts):
            q = type(p).from_buffer_copy(p)
            q.row_begin, q.row_end = b, e
            rp, col, val = _csr(mc.mcmi_build_ex(B, q))
            rps.append(np.diff(rp))
            cols.append(col)
            vals.append(val)
        rp = np.concatenate([[0], np.cumsum(np.concatenate(rps))])
        assert np.array_equal(rp, full[0])
        assert np.array_equal(np.concatenate(cols), full[1])
        assert np.array_equal(np.concatenate(vals), full[2])


def test_build_sharded_on_one_rank_is_the_plain_build():
    import torch.distributed as dist
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        m = synth.powerlaw_random(5000, seed=9)
        p = mc.params(chains=64, max_len=128, delta=1e-3, filter_tau=1e-2, seed=4)
        B = mc.DeviceCsr.from_host(m)
        rp, col, val, st = build_sharded(B, p)
        full = _csr(mc.mcmi_build_ex(B, p))
        assert np.array_equal(rp.cpu().numpy(), full[0])
        assert np.array_equal(col.cpu().numpy(), full[1]) and np.array_equal(val.cpu().numpy(), full[2])
        assert st.rows == m.n
    finally:
        dist.destroy_process_group()
