"""General (not diagonally dominant) matrices through the Eq. 1 augmentation
bhat_ii = b_ii + alpha ||B||_inf sgn(b_ii) (Sec. V-C): the unaugmented
build is refused, augmented walks match the oracle, and the walk cost
follows the closed-form chain length as alpha changes (the paper reports
about 20% longer runs at alpha = 4 than at alpha = 5)."""
import numpy as np
import pytest

import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402


def _orc():
    import oracle
    return oracle


def _steps(m, B, alpha, chains=64, delta=1e-6):
    p = mc.params(chains=chains, max_len=1000, delta=delta, alpha=alpha, seed=5, top_k=8)
    return mc.mcmi_build_ex(B, p).stats.steps


@pytest.mark.parametrize("alpha", [1.0, 2.0, 4.0, 5.0])
def test_every_chain_has_the_closed_form_length(alpha):
    """Equal row norms: every augmented row has the same s, so every chain
    makes exactly T*(alpha) transitions (the FP32 stop rule of the oracle)."""
    orc = _orc()
    m = synth.equal_rows(3000, 8, seed=41)
    d, s = orc.split(m, alpha)
    assert np.all(s == s[0])
    T = orc.max_walk_len(s[0], 1e-6, 1000)
    assert _steps(m, mc.DeviceCsr.from_host(m), alpha) == m.n * 64 * T


def test_alpha_sensitivity_of_the_walk_cost():
    orc = _orc()
    m = synth.equal_rows(3000, 8, seed=41)
    B = mc.DeviceCsr.from_host(m)
    t4 = orc.max_walk_len(orc.split(m, 4.0)[1][0], 1e-6, 1000)
    t5 = orc.max_walk_len(orc.split(m, 5.0)[1][0], 1e-6, 1000)
    s4, s5 = _steps(m, B, 4.0), _steps(m, B, 5.0)
    assert s4 / s5 == pytest.approx(t4 / t5) and s4 > s5
    print(f"alpha 4 vs 5: {s4 / s5:.3f}x the transitions")


def test_general_matrix_needs_alpha_and_matches_the_oracle():
    orc = _orc()
    m = synth.random_dd(5000, 9, seed=42, dominance=1.4, diag_sign="mixed")
    B = mc.DeviceCsr.from_host(m)
    with pytest.raises(mc.McmiError) as e:
        mc.mcmi_build_ex(B, mc.params(chains=32, max_len=64, delta=1e-3))
    assert e.value.status == 4          # MCMI_ERR_NOT_CONTRACTIVE
    alpha, N, L, delta, seed = 0.5, 128, 200, 1e-4, 17
    p = mc.params(chains=N, max_len=L, delta=delta, alpha=alpha, seed=seed, filter_tau=1e-2)
    M = mc.mcmi_build_ex(B, p)
    rows = np.unique(np.concatenate([[0, m.n - 1], np.random.default_rng(3).choice(m.n, 30, replace=False)]))
    orows, d, s = orc.walk(m, rows=rows, chains=N, max_len=L, delta=delta, seed=seed, table=M.stats.table,
                           alpha=alpha)
    assert np.max(s) < 1.0
    grows = mc.mcmi_walk_dump(B, p, rows, max(len(r["col"]) for r in orows) + 16)
    mx, med, bounded = P.compare_dump(grows, orows, d)
    print(f"general matrix, alpha {alpha}: max rel {mx:.2e} median {med:.2e} bounded {bounded:.3f}")
    assert bounded <= 1.0
    rp, col, val = (t.cpu().numpy() for t in M.to_torch())
    torch.cuda.synchronize()
    for r in orows:
        i = r["row"]
        mvals = r["X"] / d[r["col"]]
        oc, ov = orc.filter_row(i, r["col"], mvals, tau=1e-2, top_k=0)
        gc, gv = col[rp[i]:rp[i + 1]], val[rp[i]:rp[i + 1]]
        rel, b = P.compare_rows(gc, gv.astype(np.float64), oc, ov, r["col"], mvals, r["A"] / np.abs(d[r["col"]]),
                                i, 1e-2, 0)
        assert b <= 1.0
