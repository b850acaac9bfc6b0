"""Matrix reduction (Algorithm 1, step 2) on the GPU against the oracle:
the reduced CSR is bit-identical (an integer selection) for both modes,
with ties at the cut, and a build on it equals a build on the oracle's."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402


def _orc():
    import oracle
    return oracle


def _tied(m, decimals=1):
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    off = m.col != rows
    m.val[off] = np.round(m.val[off], decimals)
    return m


def _cases():
    return {
        "rand_tied": _tied(synth.random_dd(2000, 9, seed=21, diag_sign="mixed")),
        "powerlaw_tied": _tied(synth.powerlaw_random(1 << 17, seed=22), 2),
        "stencil3d": synth.stencil3d_7pt(24, seed=23),
    }


def _same(R, ref):
    rp, col, val = (t.cpu().numpy() for t in R.to_torch())
    torch.cuda.synchronize()
    assert R.n == ref.n and R.nnz == ref.nnz
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    assert np.array_equal(val.view(np.uint64), ref.val.view(np.uint64))


@pytest.mark.parametrize("name", list(_cases()))
@pytest.mark.parametrize("mode", [0, 1])
def test_reduced_csr_bit_identical(name, mode):
    orc = _orc()
    m = _cases()[name]
    B = mc.DeviceCsr.from_host(m)
    for f in (0.0, 0.02, 0.075, 0.3, 0.5, 0.999, 1.0):
        ref, keep, d = orc.reduce(m, f, mode)
        R = mc.mcmi_reduce(B, f, mode)
        assert R.dropped == d, (name, mode, f, R.dropped, d)
        _same(R, ref)
        R.close()


def test_build_on_the_reduced_matrix_equals_build_on_the_oracles():
    orc = _orc()
    m = synth.powerlaw_random(4096, seed=24, dominance=0.85)
    ref, _, _ = orc.reduce(m, 0.06, mc.REDUCE_RANGE)
    R = mc.mcmi_reduce(mc.DeviceCsr.from_host(m), 0.06, mc.REDUCE_RANGE)
    p = mc.params(chains=128, max_len=128, delta=1e-3, filter_tau=5e-3, seed=3)
    a = [t.cpu().numpy() for t in mc.mcmi_build_ex(R, p).to_torch()]
    b = [t.cpu().numpy() for t in mc.mcmi_build_ex(mc.DeviceCsr.from_host(ref), p).to_torch()]
    torch.cuda.synchronize()
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_reduce_edge_cases_and_errors():
    orc = _orc()
    one = synth._from_coo(1, np.array([0]), np.array([0]), np.array([3.0]))
    for f in (0.0, 1.0):
        for mode in (0, 1):
            R = mc.mcmi_reduce(mc.DeviceCsr.from_host(one), f, mode)
            ref, _, _ = orc.reduce(one, f, mode)
            _same(R, ref)
    empty = mc.DeviceCsr(0, torch.zeros(1, dtype=torch.int64, device="cuda"),
                         torch.zeros(0, dtype=torch.int32, device="cuda"),
                         torch.zeros(0, dtype=torch.float64, device="cuda"))
    R = mc.mcmi_reduce(empty, 0.5)
    assert R.n == 0 and R.nnz == 0 and R.dropped == 0
    B = mc.DeviceCsr.from_host(synth.random_dd(30, 3, seed=1))
    for f, mode in ((1.5, 0), (-0.1, 1), (0.5, 7)):
        with pytest.raises(mc.McmiError) as e:
            mc.mcmi_reduce(B, f, mode)
        assert e.value.status == 1
