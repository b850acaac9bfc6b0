"""Learned proposal on the GPU against the oracle: tables and walks bit-exact
(seeded, untrained parameters), row moments, loss and gradients against
FP64 central differences, training, unbiasedness."""
import numpy as np
import pytest

import synth
from tests import _parity as Pp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402


def _orc():
    import oracle
    return oracle


def _theta(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(1377) * scale).astype(np.float32)


CASES = {
    "rand": (lambda: synth.random_dd(400, 7, seed=3, diag_sign="mixed", zero_frac=0.05, dominance=0.8), 0.0),
    "aniso": (lambda: synth.aniso2d_9pt(20, seed=2001), 0.3),
    "powerlaw": (lambda: synth.powerlaw_random(1500, seed=5, dominance=0.8), 0.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_learned_tables_bit_exact(name):
    orc = _orc()
    gen, alpha = CASES[name]
    m = gen()
    th = _theta(7)
    P = mc.Proposal(th)
    B = mc.DeviceCsr.from_host(m)
    g = mc.mcmi_debug_tables(B, mc.params(proposal=P, alpha=alpha))
    lt = orc.learned_tables(m, th, alpha=alpha)
    assert np.array_equal(g["slot"][:, 0], lt["Q"].astype(np.uint32))
    for i in range(m.n):
        a, b = lt["off"][i], lt["off"][i + 1]
        deg = b - a
        assert g["slot"][i, 3] == (deg | (1 << 31))
        if deg == 0:
            continue
        o = g["slot"][i, 4]
        prob, al = orc.alias_build(lt["q"][a:b], int(lt["Q"][i]))
        assert np.array_equal(g["a"][o:o + deg], prob)
        own = g["b"][o:o + deg]
        assert np.array_equal(g["c"][o:o + deg], own[al])


@pytest.mark.parametrize("name", list(CASES))
def test_learned_walks_bit_exact(name):
    orc = _orc()
    gen, alpha = CASES[name]
    m = gen()
    th = _theta(9, scale=0.7)
    P = mc.Proposal(th)
    B = mc.DeviceCsr.from_host(m)
    rows = np.arange(0, m.n, max(1, m.n // 40))
    N, L, delta, seed = 128, 60, 1e-3, 31
    p = mc.params(chains=N, max_len=L, delta=delta, seed=seed, alpha=alpha, proposal=P)
    orows, d, s = orc.walk(m, rows=rows, chains=N, max_len=L, delta=delta, seed=seed, table=1, alpha=alpha, theta=th)
    grows = mc.mcmi_walk_dump(B, p, rows, max(len(r["col"]) for r in orows) + 16)
    mx, med, bounded = Pp.compare_dump(grows, orows, d)
    print(f"learned {name}: max rel {mx:.2e} median {med:.2e} bounded {bounded:.3f}")
    assert bounded <= 1.0


@pytest.mark.parametrize("learned", [False, True])
def test_row_moments_match_oracle(learned):
    orc = _orc()
    m = synth.aniso2d_9pt(16, seed=2002)
    th = _theta(4) if learned else None
    P = mc.Proposal(th) if learned else None
    B = mc.DeviceCsr.from_host(m)
    kw = dict(chains=64, max_len=80, delta=1e-3, seed=5, alpha=0.3)
    mg = mc.mcmi_row_moments(B, mc.params(proposal=P, table=1, **kw) if learned else mc.params(table=1, **kw))
    mo = orc.row_moments(m, chains=64, max_len=80, delta=1e-3, seed=5, table=1, alpha=0.3, theta=th)
    assert np.allclose(mg.cpu().numpy(), mo, rtol=2e-5)


def _fd_grad(orc, th, feat, row, p, mt, idx, h=1e-3):
    out = []
    for k in idx:
        tp, tm = th.astype(np.float64).copy(), th.astype(np.float64).copy()
        tp[k] += h
        tm[k] -= h
        out.append((orc.proposal_loss(tp, feat, row, p, mt) - orc.proposal_loss(tm, feat, row, p, mt)) / (2 * h))
    return np.array(out)


def test_loss_and_gradient_match_central_differences():
    orc = _orc()
    m = synth.aniso2d_9pt(14, seed=2003)
    alpha = 0.3
    B = mc.DeviceCsr.from_host(m)
    th = _theta(12, scale=0.3)
    P = mc.Proposal(th)
    wp = mc.params(chains=64, max_len=80, delta=1e-3, seed=2, alpha=alpha, table=1)
    mrow = orc.row_moments(m, chains=64, max_len=80, delta=1e-3, seed=2, table=1, alpha=alpha)
    feat, pe, tgt, row = orc.train_edges(m, alpha=alpha)
    mt = mrow[tgt]
    m_dev = torch.from_numpy(mrow.astype(np.float32)).cuda()
    # FP32 network: loss and gradient against FP64 central differences
    loss, grad = mc.mcmi_proposal_loss_grad(B, m_dev, wp, P, round_bf16=0)
    ref = orc.proposal_loss(th, feat, row, pe, mt)
    assert abs(loss - ref) <= 1e-4 * ref, (loss, ref)
    rng = np.random.default_rng(0)
    idx = np.concatenate([np.arange(1344, 1377), rng.choice(1344, 80, replace=False)])
    fd = _fd_grad(orc, th, feat, row, pe, mt, idx)
    err = np.linalg.norm(grad[idx] - fd) / np.linalg.norm(fd)
    print(f"gradient rel err (FP32 net) {err:.2e}")
    assert err < 2e-3
    # BF16 network (as trained and used): within BF16 precision
    loss16, grad16 = mc.mcmi_proposal_loss_grad(B, m_dev, wp, P, round_bf16=1)
    assert abs(loss16 - ref) <= 2e-2 * ref
    err16 = np.linalg.norm(grad16[idx] - fd) / np.linalg.norm(fd)
    print(f"gradient rel err (BF16 net) {err16:.2e}")
    assert err16 < 5e-2


def test_training_lowers_the_loss_and_keeps_unbiasedness():
    mats = [synth.aniso2d_9pt(int(nx), seed=2100 + k) for k, nx in enumerate([16, 20, 24, 16, 20, 24])]
    Bs = [mc.DeviceCsr.from_host(m) for m in mats]
    P = mc.Proposal()
    tp = mc.mcmi_train_params(steps=150, lr=3e-3, chains=64, max_len=200, delta=1e-4, alpha=0.3, seed=7,
                              round_bf16=1)
    hist = mc.mcmi_proposal_train(Bs, tp, P)
    print("loss", hist[0], "->", hist[-1])
    assert hist[-1] < hist[0] and hist[-1] >= 1.0 - 1e-3
    # the trained proposal still estimates (I - C)^-1 D^-1 without bias
    m = synth.aniso2d_9pt(12, seed=2999)
    B = mc.DeviceCsr.from_host(m)
    rows = np.arange(0, m.n, 13)
    for prop in (None, P):
        p = mc.params(chains=20000, max_len=400, delta=1e-6, seed=3, alpha=0.3, table=1, proposal=prop)
        got = mc.mcmi_walk_dump(B, p, rows, m.n + 1)
        orc = _orc()
        d, s = orc.split(m, alpha=0.3)
        Bh = m.to_scipy().toarray()
        Bh[np.diag_indices(m.n)] = d
        inv = np.linalg.inv(Bh)
        for r, g in zip(rows, got):
            est = np.zeros(m.n)
            est[g["col"]] = g["val"]
            assert np.linalg.norm(est - inv[r]) / np.linalg.norm(inv[r]) < 0.03


def test_trained_proposal_needs_fewer_steps_on_heterogeneous_rows():
    """Where the rows' own walk lengths differ a lot (s_i from 0.1 to 0.97),
    |c| is far from the best proposal: after training, the learned proposal
    reaches the |c| proposal's estimator error with measurably fewer walk
    steps (errors against the exact inverse, same chains and cutoff)."""
    rng = np.random.default_rng(0)
    train = [synth.random_dd(int(n), 6, seed=3000 + k, dominance=0.97, dominance_jitter=0.9, diag_sign="mixed")
             for k, n in enumerate(rng.integers(1000, 4000, 40))]
    P = mc.Proposal()
    tp = mc.mcmi_train_params(steps=150, lr=3e-3, chains=64, max_len=300, delta=1e-4, alpha=0.0, seed=7,
                              round_bf16=1)
    hist = mc.mcmi_proposal_train([mc.DeviceCsr.from_host(m) for m in train], tp, P)
    assert hist[-1] < hist[0]
    m = synth.random_dd(3000, 6, seed=3999, dominance=0.97, dominance_jitter=0.9, diag_sign="mixed")
    B = mc.DeviceCsr.from_host(m)
    inv = np.linalg.inv(m.to_scipy().toarray())
    rows = np.arange(0, m.n, 29)
    res = {}
    for name, prop in (("plain", None), ("learned", P)):
        p = mc.params(chains=128, max_len=300, delta=1e-4, seed=5, table=mc.TABLE_ALIAS, proposal=prop)
        errs, steps = [], 0
        for k in range(6):
            p.seed = 100 + k
            for r, g in zip(rows, mc.mcmi_walk_dump(B, p, rows, m.n + 1)):
                est = np.zeros(m.n)
                est[g["col"]] = g["val"]
                errs.append(np.linalg.norm(est - inv[r]) / np.linalg.norm(inv[r]))
                steps += g["steps"]
        res[name] = (float(np.mean(errs)), steps)
    (ep, sp), (el, sl) = res["plain"], res["learned"]
    ratio = (el / ep) ** 2 * sl / sp    # steps the learned proposal needs at the plain one's error (error ~ N^-1/2)
    print(f"loss {hist[0]:.4f} -> {hist[-1]:.4f}; eps plain {ep:.4f} learned {el:.4f}; steps at equal error {ratio:.3f}")
    assert ratio < 0.97
