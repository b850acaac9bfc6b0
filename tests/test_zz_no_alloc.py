"""The allocation-free row-offset scan (mcmi_exclusive_scan_noalloc), called
through the C ABI, against the row pointers of mcmi_build_ex.

This entry point exists for callers that cannot allocate device memory at
the call site; its scratch is a fixed device array shared by all calls.  The
test runs it twice in a row (the array keeps the first call's partial sums)
and checks that sizes over its fixed limit are refused.  This file is
collected last so that a run that stops at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402


def _noalloc(counts):
    lib = mc.load()
    out = torch.full((counts.numel() + 1,), -7, dtype=torch.int64, device="cuda")
    st = lib.mcmi_exclusive_scan_noalloc(ctypes.c_void_p(counts.data_ptr()), counts.numel(),
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.mcmi_last_error().decode()
    torch.cuda.synchronize()
    return out


def test_noalloc_scan_matches_build_row_pointers_twice():
    # two builds of different sizes and sparsity: row pointers from the
    # library's own (allocating) path are the reference
    cases = [
        (synth.stencil3d_7pt(20, seed=3), mc.params(chains=256, max_len=128, delta=1e-2, top_k=16, seed=1)),
        (synth.powerlaw_random(6000, seed=4), mc.params(chains=64, max_len=64, delta=1e-3, filter_tau=1e-2, seed=2)),
    ]
    for m, p in cases:
        M = mc.mcmi_build_ex(mc.DeviceCsr.from_host(m), p)
        rp, _, _ = M.to_torch()
        torch.cuda.synchronize()
        counts = (rp[1:] - rp[:-1]).to(torch.int32).contiguous()
        got = _noalloc(counts)
        assert torch.equal(got, rp), "row pointers differ from mcmi_build_ex"


def test_noalloc_scan_large_and_limit():
    g = torch.Generator(device="cuda").manual_seed(5)
    counts = torch.randint(0, 1000, (3_000_001,), device="cuda", dtype=torch.int32, generator=g)
    ref = torch.zeros(counts.numel() + 1, dtype=torch.int64, device="cuda")
    ref[1:] = torch.cumsum(counts.to(torch.int64), 0)
    assert torch.equal(_noalloc(counts), ref)
    assert torch.equal(_noalloc(counts[:12345].contiguous()), ref[:12346])
    # exactly the limit: every tile of the fixed array, the last scratch word included
    full = torch.randint(0, 64, (33_554_432,), device="cuda", dtype=torch.int32, generator=g)
    ref_full = torch.zeros(full.numel() + 1, dtype=torch.int64, device="cuda")
    ref_full[1:] = torch.cumsum(full.to(torch.int64), 0)
    assert torch.equal(_noalloc(full), ref_full)
    del full, ref_full
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    assert _noalloc(empty).tolist() == [0]
    lib = mc.load()
    big_n = 33_554_432 + 1
    st = lib.mcmi_exclusive_scan_noalloc(ctypes.c_void_p(counts.data_ptr()), big_n, ctypes.c_void_p(ref.data_ptr()), None)
    assert st == mc.McmiError(1, "").status and b"fixed scratch limit" in lib.mcmi_last_error()
