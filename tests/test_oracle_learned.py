"""Pins of the oracle's learned-proposal functions (CPU).

- the BF16 MLP against an independent emulation built on torch's bfloat16
  conversion, and against the same network in FP64;
- learned tables: q/Q follows |c| g, and f = c Q / q undoes the proposal;
- unbiasedness: the learned estimator's exact expectation (path
  enumeration) equals the truncated Neumann series sum_t C^t, and its Monte
  Carlo estimate has z-scores < 5 against it;
- the second moments m_i against their closed form (equal row norms);
- the training loss is >= 1 and equals 1 when g is proportional to sqrt(m).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def _theta(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(1377) * scale).astype(np.float32)


def _bf16(x):
    return torch.tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _mlp_bf16(theta, f):
    th = np.asarray(theta, dtype=np.float32)
    W1, b1 = _bf16(th[:256]).reshape(32, 8), th[256:288]
    W2, b2 = _bf16(th[288:1312]).reshape(32, 32), th[1312:1344]
    w3, b3 = _bf16(th[1344:1376]), th[1376]
    x = _bf16(f)
    h1 = np.zeros(32, np.float32)
    for o in range(32):
        acc = np.float32(b1[o])
        for k in range(8):
            acc = np.float32(acc + np.float32(W1[o, k] * x[k]))
        h1[o] = max(acc, np.float32(0))
    h1 = _bf16(h1)
    h2 = np.zeros(32, np.float32)
    for o in range(32):
        acc = np.float32(b2[o])
        for k in range(32):
            acc = np.float32(acc + np.float32(W2[o, k] * h1[k]))
        h2[o] = max(acc, np.float32(0))
    h2 = _bf16(h2)
    z = np.float32(b3)
    for k in range(32):
        z = np.float32(z + np.float32(w3[k] * h2[k]))
    g = np.float32(np.float32(0.5) * np.float32(z + np.sqrt(np.float32(np.float32(z * z) + np.float32(4)))))
    return float(np.clip(g, np.float32(0.0625), np.float32(16.0)))


def test_mlp_matches_bf16_emulation_and_fp64(orc):
    rng = np.random.default_rng(0)
    for trial in range(40):
        th = _theta(trial, scale=float(rng.choice([0.1, 0.5, 1.0])))
        f = (rng.standard_normal(8) * rng.choice([0.1, 1.0, 3.0])).astype(np.float32)
        g = orc.mlp_g(th, f)
        assert g == _mlp_bf16(th, f)
        # FP64 network without rounding: same g within BF16 precision
        t = th.astype(np.float64)
        h1 = np.maximum(t[:256].reshape(32, 8) @ f + t[256:288], 0)
        h2 = np.maximum(t[288:1312].reshape(32, 32) @ h1 + t[1312:1344], 0)
        z = t[1344:1376] @ h2 + t[1376]
        g64 = np.clip(0.5 * (z + np.sqrt(z * z + 4)), 0.0625, 16.0)
        assert abs(g - g64) <= 0.05 * g64 + 0.02


def test_learned_tables_follow_g_and_undo_the_proposal(orc):
    m = synth.random_dd(80, 6, seed=7, diag_sign="mixed", zero_frac=0.1, dominance=0.8)
    th = _theta(3)
    lt = orc.learned_tables(m, th)
    B = m.to_scipy().toarray()
    C = np.eye(m.n) - B / np.diag(B)[:, None]
    for i in range(m.n):
        a, b = lt["off"][i], lt["off"][i + 1]
        cols = [c for c in m.col[m.row_ptr[i]:m.row_ptr[i + 1]] if c != i]
        c = C[i, cols]
        q = lt["q"][a:b].astype(np.float64)
        Q = float(lt["Q"][i])
        assert Q == float(lt["q"][a:b].astype(np.uint64).sum())
        w = np.abs(c) * lt["g"][a:b].astype(np.float64)
        if w.sum() == 0:
            continue
        assert np.all((q == 0) == (w == 0))
        assert np.all(np.abs(q / Q - w / w.sum()) <= (len(q) + 1) / Q)
        nz = q > 0
        assert np.allclose(lt["fac"][a:b][nz] * q[nz] / Q, c[nz], rtol=1e-14, atol=0)
        assert np.all((lt["g"][a:b][nz] >= 0.0625) & (lt["g"][a:b][nz] <= 16.0))


def _enumerate_learned(m, lt, i, L, second=False):
    """Exact E[Y] (and E[Y^2]) of one learned chain (no cutoff, length L)."""
    n = m.n
    EY = np.zeros(n)
    EY2 = np.zeros(n)
    off = lt["off"]

    def rec(state, w, t, prob, Y):
        Y = Y.copy()
        Y[state] += w
        if t == L or lt["Q"][state] == 0:
            EY[:] += prob * Y
            EY2[:] += prob * Y * Y
            return
        cols = [c for c in m.col[m.row_ptr[state]:m.row_ptr[state + 1]] if c != state]
        a = off[state]
        Q = float(lt["Q"][state])
        for k, c in enumerate(cols):
            p = lt["q"][a + k] / Q
            if p > 0:
                rec(c, w * lt["fac"][a + k], t + 1, prob * p, Y)

    rec(i, 1.0, 0, 1.0, np.zeros(n))
    return (EY, EY2) if second else EY


@pytest.mark.parametrize("table", [0, 1])
def test_learned_estimator_is_unbiased(orc, table):
    m = synth.random_dd(5, 3, seed=21, dominance=0.85, diag_sign="mixed")
    th = _theta(11, scale=1.0)
    lt = orc.learned_tables(m, th)
    B = m.to_scipy().toarray()
    C = np.eye(m.n) - B / np.diag(B)[:, None]
    L = 4
    P = sum(np.linalg.matrix_power(C, t) for t in range(L + 1))
    for i in range(m.n):   # the exact expectation equals the Neumann sum
        assert np.allclose(_enumerate_learned(m, lt, i, L), P[i], rtol=1e-9, atol=1e-12)
    N = 200_000
    res, _, _ = orc.walk(m, chains=N, max_len=L, delta=0.0, seed=9, table=table, theta=th)
    worst = 0.0
    for r in res:
        X = np.zeros(m.n)
        X[r["col"]] = r["X"]
        EY, EY2 = _enumerate_learned(m, lt, r["row"], L, second=True)
        var = np.maximum(EY2 - EY * EY, 0.0)
        ok = var > 0
        worst = max(worst, float(np.max(np.abs(X[ok] - P[r["row"]][ok]) / np.sqrt(var[ok] / N), initial=0.0)))
        assert np.allclose(X[~ok], P[r["row"]][~ok], rtol=1e-9, atol=1e-12)
    assert worst < 5.0, worst


def test_row_moments_closed_form(orc):
    m = synth.random_dd(30, 4, seed=8, signs="negative", dominance=0.7)
    delta, L = 1e-3, 200
    w = np.float32(1.0)
    T = 0
    while T < L and not (float(abs(w)) < delta):
        w = np.float32(w * np.float32(0.7))
        T += 1
    mm = orc.row_moments(m, chains=16, max_len=L, delta=delta, seed=3)
    assert np.allclose(mm, sum(0.7 ** (2 * t) for t in range(T + 1)), rtol=1e-12)


def test_training_loss_bounds(orc):
    rng = np.random.default_rng(5)
    nrow, per = 50, 6
    r = np.repeat(np.arange(nrow), per)
    p = rng.random(nrow * per)
    p /= np.bincount(r, p)[r]
    mm = rng.random(nrow * per) * 3 + 0.1
    feat = rng.standard_normal((nrow * per, 8)).astype(np.float32)
    for s in range(5):
        assert orc.proposal_loss(_theta(s), feat, r, p, mm) >= 1.0 - 1e-12
    # g proportional to sqrt(m) inside each row reaches 1: only the bias of
    # the last layer acts (other weights zero), one row, m constant
    th = np.zeros(1377, np.float32)
    th[1376] = 1.3
    one = np.zeros(per, np.int64)
    assert abs(orc.proposal_loss(th, feat[:per], one, p[:per] / p[:per].sum(), np.full(per, 2.0)) - 1.0) < 1e-12



def _mixed_degree_matrix(n, seed):
    """Mixed-sign rows of 1-8 off-diagonals (some explicit zeros), diagonal of
    random sign and dominance, so that s_i, deg_i and |d_i| differ between
    the two ends of most edges."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        deg = int(rng.integers(1, 9))
        js = rng.choice(np.setdiff1d(np.arange(n), [i]), deg, replace=False)
        v = rng.standard_normal(deg) * rng.choice([0.1, 1.0, 10.0])
        v[rng.random(deg) < 0.1] = 0.0
        diag = (np.abs(v).sum() or 1.0) / rng.uniform(0.5, 0.95) * rng.choice([-1.0, 1.0])
        rows += [i] * (deg + 1)
        cols += list(js) + [i]
        vals += list(v) + [diag]
    return synth._from_coo(n, rows, cols, vals)


def _closed_form_features(orc, m):
    """Per stored off-diagonal (i, j): the eight features from the dense
    C = I - D^-1 B (s_i from the oracle's split, which its own pin checks
    against the dense row sums; numpy's pairwise sum may differ by an ulp)."""
    B = m.to_scipy().toarray()
    dd = np.diag(B).copy()
    C = -B / dd[:, None]
    np.fill_diagonal(C, 0.0)
    _, s = orc.split(m)
    assert np.allclose(s, np.abs(C).sum(axis=1), rtol=1e-14, atol=0)
    stored = np.zeros((m.n, m.n), bool)
    stored[np.repeat(np.arange(m.n), np.diff(m.row_ptr)), m.col] = True
    np.fill_diagonal(stored, False)
    deg = stored.sum(axis=1)
    out = {}
    for i in range(m.n):
        maxabs = np.abs(C[i, stored[i]]).max()
        for j in np.flatnonzero(stored[i]):
            c = C[i, j]
            if c == 0.0:
                out[(i, j)] = None
                continue
            out[(i, j)] = np.array([abs(c) / s[i], s[i], s[j], 1.0 / deg[i], 1.0 / deg[j],
                                    abs(dd[i]) / (abs(dd[i]) + abs(dd[j])), abs(c) / maxabs,
                                    -1.0 if c < 0 else 1.0]).astype(np.float32)
    return out, C, s, deg, dd


def test_edge_features_match_their_closed_forms(orc):
    """orc_train_edges' eight features of edge (i, j) equal |c_ij|/s_i, s_i,
    s_j, 1/deg_i, 1/deg_j, |d_i|/(|d_i|+|d_j|), |c_ij|/max_k|c_ik| and
    sign(c_ij) recomputed from the dense matrix (FP64, then FP32).  The
    matrix is built so that swapping i and j in any two-sided feature
    changes it on most edges."""
    m = _mixed_degree_matrix(60, seed=17)
    want, C, s, deg, dd = _closed_form_features(orc, m)
    feat, p, tgt, row = orc.train_edges(m)
    checked = swaps = 0
    for k in range(len(tgt)):
        i, j = int(row[k]), int(tgt[k])
        if i == j or want[(i, j)] is None:
            assert np.all(feat[k] == 0.0) and p[k] == 0.0
            continue
        assert np.array_equal(feat[k], want[(i, j)]), (i, j, feat[k], want[(i, j)])
        assert p[k] == abs(C[i, j]) / s[i]
        checked += 1
        swaps += (abs(s[i] - s[j]) > 1e-3 * s[i]) and deg[i] != deg[j] and abs(dd[i]) != abs(dd[j])
    assert checked > 200 and swaps > 0.6 * checked, (checked, swaps)
    assert len(want) == sum(1 for k in range(len(tgt)) if row[k] != tgt[k])


def test_learned_tables_evaluate_the_network_on_the_closed_form_features(orc):
    """orc_learned_tables' g equals the independent BF16 emulation of the MLP
    evaluated on the features recomputed from the dense matrix."""
    m = _mixed_degree_matrix(24, seed=5)
    th = _theta(9)
    lt = orc.learned_tables(m, th)
    want, _, _, _, _ = _closed_form_features(orc, m)
    e = 0
    for i in range(m.n):
        for j in m.col[m.row_ptr[i]:m.row_ptr[i + 1]]:
            if j == i:
                continue
            f = want[(i, int(j))]
            assert lt["g"][e] == (0.0 if f is None else _mlp_bf16(th, f)), (i, j)
            e += 1
    assert e == len(lt["g"])
