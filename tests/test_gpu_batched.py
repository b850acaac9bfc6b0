"""Batched builds (one persistent, graph-captured walk over many matrices)
and the autotuner."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402


def _mats():
    return [synth.stencil2d_5pt(20, 17, seed=1, dominance=0.9),
            synth.stencil3d_7pt(9, seed=2, dominance=0.85),
            synth.powerlaw_random(1500, seed=3, dominance=0.8),
            synth.random_dd(1, 0, seed=4),
            synth.stencil2d_5pt(31, 40, seed=5, dominance=0.95),
            synth.powerlaw_random(777, seed=6, dominance=0.92)]


def _csr(M):
    out = [t.cpu().numpy() for t in M.to_torch()]
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("table", [0, 1, 2])
def test_batched_equals_individual_builds(table):
    mats = _mats()
    Bs = [mc.DeviceCsr.from_host(m) for m in mats]
    p = mc.params(chains=96, max_len=100, delta=1e-3, filter_tau=1e-2, top_k=8, seed=77, table=table)
    Ms, st = mc.mcmi_build_batched(Bs, p)
    assert st.rows == sum(m.n for m in mats)
    total_steps = 0
    for B, M in zip(Bs, Ms):
        Mi = mc.mcmi_build_ex(B, mc.params(chains=96, max_len=100, delta=1e-3, filter_tau=1e-2, top_k=8, seed=77,
                                           table=table))
        total_steps += Mi.stats.steps
        for u, v in zip(_csr(M), _csr(Mi)):
            assert np.array_equal(u, v)
    assert st.steps == total_steps


@pytest.mark.parametrize("table", [mc.TABLE_COMPACT, mc.TABLE_AUTO])
def test_batched_compact_equals_individual_builds(table):
    """Stencils only: the block-diagonal batch fits the compact table (column
    offsets stay inside each block), and AUTO picks it for the batch as for
    each matrix alone."""
    mats = [m for k, m in enumerate(_mats()) if k in (0, 1, 3, 4)]
    Bs = [mc.DeviceCsr.from_host(m) for m in mats]
    # a fixed launch shape: no autotuner, so AUTO resolves as in a single build
    kw = dict(chains=96, max_len=100, delta=1e-3, filter_tau=1e-2, top_k=8, seed=77, table=table, threads=128,
              chains_per_thread=1, hash_log2=11)
    Ms, st = mc.mcmi_build_batched(Bs, mc.params(**kw))
    assert st.table == mc.TABLE_COMPACT
    for B, M in zip(Bs, Ms):
        Mi = mc.mcmi_build_ex(B, mc.params(**kw))
        assert Mi.stats.table == mc.TABLE_COMPACT
        for u, v in zip(_csr(M), _csr(Mi)):
            assert np.array_equal(u, v)


def test_batched_split_by_table_type_equals_individual_builds():
    """A batch of stencils and power-law matrices with the table left to AUTO:
    the stencils take the compact table and the others the hybrid one, each
    group in its own batch; every M equals the matrix's own AUTO build."""
    mats = _mats()
    Bs = [mc.DeviceCsr.from_host(m) for m in mats]
    kw = dict(chains=96, max_len=100, delta=1e-3, filter_tau=1e-2, top_k=8, seed=77, threads=128,
              chains_per_thread=1, hash_log2=11)
    Ms, st = mc.mcmi_build_batched(Bs, mc.params(**kw))
    assert st.rows == sum(m.n for m in mats)
    tables, steps = set(), 0
    for B, M in zip(Bs, Ms):
        Mi = mc.mcmi_build_ex(B, mc.params(**kw))
        tables.add(Mi.stats.table)
        steps += Mi.stats.steps
        for u, v in zip(_csr(M), _csr(Mi)):
            assert np.array_equal(u, v)
    assert tables == {mc.TABLE_COMPACT, mc.TABLE_HYBRID} and st.steps == steps


def test_batched_fixed_shape_and_errors():
    mats = _mats()[:3]
    Bs = [mc.DeviceCsr.from_host(m) for m in mats]
    p = mc.params(chains=64, max_len=64, delta=1e-3, top_k=4, seed=5, table=0, threads=256, chains_per_thread=1,
                  hash_log2=10)
    Ms, st = mc.mcmi_build_batched(Bs, p)
    assert len(Ms) == 3 and st.hash_log2 == 10
    bad = synth.random_dd(30, 3, seed=9)
    bad.val[bad.row_ptr[4]] = np.nan
    with pytest.raises(mc.McmiError) as e:
        mc.mcmi_build_batched(Bs + [mc.DeviceCsr.from_host(bad)], p)
    assert e.value.status == 2
    with pytest.raises(mc.McmiError):
        mc.mcmi_build_batched(Bs, mc.params(row_begin=1, row_end=3))


def test_autotune_picks_a_valid_shape_with_identical_results():
    m = synth.stencil3d_7pt(24, seed=8)
    B = mc.DeviceCsr.from_host(m)
    base = dict(chains=128, max_len=128, delta=1e-2, top_k=16, seed=3, table=0)
    p = mc.params(**base)
    rep = mc.mcmi_autotune(B, p)
    assert rep.trials >= 8 and rep.best_ms > 0 and rep.best_ms <= rep.default_ms * 1.0001
    # a trial replaces the default plan only when 2% faster
    assert rep.best_ms == rep.default_ms or rep.best_ms < 0.98 * rep.default_ms
    assert p.threads in (64, 128, 256) and p.chains_per_thread in (1, 2) and 9 <= p.hash_log2 <= 13
    assert p.load_depth in (4, 8) and rep.load_depth == p.load_depth
    # walks do not depend on the launch shape; fixed-point sums are exact
    a = _csr(mc.mcmi_build_ex(B, p))
    b = _csr(mc.mcmi_build_ex(B, mc.params(**base)))
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
