"""Parity at the full benchmark sizes, in the launch configuration that
bench.py times (default launch shape, the benchmark's parameters and seed),
on sampled rows the oracle computes one by one.

For each configuration: the parity dump of the sampled rows has bit-exact
visited columns, visit counts and transition counts, with entries within
1e-5 (bounded where signed weights cancel). The rows of the timed build
(filter included) match the oracle's filtered rows. Each test prints its
errors: these are the per-configuration errors quoted in the design notes.
"""
import numpy as np
import pytest

import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402

SEED = 1000   # bench.py's seed on rank 0


def _orc():
    import oracle
    return oracle


def _sample(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1], rng.choice(n, min(n, k), replace=False)])).astype(np.int64)


def _csr_rows(M):
    rp, col, val = (t.cpu().numpy() for t in M.to_torch())
    torch.cuda.synchronize()
    return rp, col, val


def _check(name, m, B, p, M, rows, table, tau, top_k, alpha=0.0, theta=None, row_base=0, threads=0):
    """Dump parity and filtered-row parity of sampled rows; returns the errors.
    threads: oracle threads (0: all cores; each holds dense per-column sums)."""
    orc = _orc()
    orows, d, s = orc.walk(m, rows=rows, chains=p.chains, max_len=p.max_len, delta=p.delta, seed=p.seed,
                           table=table, alpha=alpha, theta=theta, threads=threads)
    cap = max(len(r["col"]) for r in orows) + 16
    grows = mc.mcmi_walk_dump(B, p, rows, cap)
    d_max, d_med, d_bnd = P.compare_dump(grows, orows, d)
    rp, col, val = _csr_rows(M)
    b_rel = b_bnd = 0.0
    for r in orows:
        i = r["row"]
        mvals = r["X"] / d[r["col"]]
        oc, ov = orc.filter_row(i, r["col"], mvals, tau=tau, top_k=top_k)
        gi = i + row_base
        gc, gv = col[rp[gi]:rp[gi + 1]], val[rp[gi]:rp[gi + 1]]
        rel, bnd = P.compare_rows(gc, gv.astype(np.float64), oc, ov, r["col"], mvals, r["A"] / np.abs(d[r["col"]]),
                                  i, tau, top_k)
        b_rel, b_bnd = max(b_rel, rel), max(b_bnd, bnd)
    print(f"{name}: {len(rows)} rows; walk entries max rel {d_max:.2e} median {d_med:.2e} bounded {d_bnd:.3f}; "
          f"filtered rows max rel {b_rel:.2e} bounded {b_bnd:.3f}")
    assert d_bnd <= 1.0 and b_bnd <= 1.0
    return d_max, d_bnd, b_rel, b_bnd


@pytest.mark.parametrize("name", ["stencil2d_32x32", "stencil3d_64", "powerlaw_1m"])
def test_full_size_sampled_rows(name):
    m, w = synth.workload(name)
    B = mc.DeviceCsr.from_host(m)
    p = mc.params(chains=w["chains"], max_len=w["max_len"], delta=w["delta"], filter_tau=w["tau"],
                  top_k=w["top_k"], seed=SEED)
    M = mc.mcmi_build_ex(B, p)
    assert M.stats.threads == 128 and M.stats.chains_per_thread == 1   # the benchmark's launch shape
    _check(name, m, B, p, M, _sample(m.n, 24, 7), M.stats.table, w["tau"], w["top_k"])


def test_full_size_fp64_stencil2d():
    """The FP64 build of the 2D configuration (its oracle precision)."""
    m, w = synth.workload("stencil2d_32x32")
    B = mc.DeviceCsr.from_host(m)
    p = mc.params(chains=w["chains"], max_len=w["max_len"], delta=w["delta"], filter_tau=w["tau"],
                  top_k=w["top_k"], seed=SEED, precision=64)
    M = mc.mcmi_build_ex(B, p)
    _check("stencil2d_32x32 fp64", m, B, p, M, _sample(m.n, 64, 8), M.stats.table, w["tau"], w["top_k"])


def test_full_size_batched_sampled_rows():
    """A slice of the batched family through the batched, graph-captured and
    autotuned launch; sampled rows of several matrices against the oracle."""
    mats = synth.batch_mix(24, seed=1004)
    Bs = [mc.DeviceCsr.from_host(m) for m in mats]
    p = mc.params(chains=128, max_len=128, delta=1e-3, top_k=16, seed=SEED)
    Ms, st = mc.mcmi_build_batched(Bs, p)
    for b in (0, 1, 2, 22, 23):
        # the table the batch gave this matrix: its own automatic choice (the
        # batch splits compact-table matrices from the others)
        tb = mc.mcmi_build_ex(Bs[b], mc.params(chains=1, max_len=0)).stats.table
        q = mc.params(chains=128, max_len=128, delta=1e-3, top_k=16, seed=SEED, table=tb,
                      threads=st.threads, chains_per_thread=st.chains_per_thread, hash_log2=st.hash_log2)
        _check(f"batch matrix {b} (n={mats[b].n})", mats[b], Bs[b], q, Ms[b], _sample(mats[b].n, 8, b),
               tb, 0.0, 16)


def test_full_size_learned_sampled_rows():
    """The anisotropic 1024^2 configuration with a learned proposal (seeded
    parameters): learned tables and walks against the oracle's BF16 network."""
    m = synth.aniso2d_9pt(1024, seed=1005)
    alpha = 0.25
    th = (np.random.default_rng(31).standard_normal(mc.MLP_PARAMS) * 0.3).astype(np.float32)
    prop = mc.Proposal(th)
    B = mc.DeviceCsr.from_host(m)
    p = mc.params(chains=128, max_len=256, delta=1e-3, seed=11, alpha=alpha, filter_tau=1e-2,
                  table=mc.TABLE_ALIAS, proposal=prop)
    M = mc.mcmi_build_ex(B, p)
    _check("aniso2d 1024^2 learned", m, B, p, M, _sample(m.n, 16, 9), mc.TABLE_ALIAS, 1e-2, 0, alpha=alpha,
           theta=th)
