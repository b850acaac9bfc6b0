"""Pins of the CPU oracle to things other than itself.

Each test checks an oracle function against mathematics or an independent
library: cuRAND's host Philox generator, dense matrix algebra (numpy),
exact path enumeration, closed forms of zero-variance cases, the 1/sqrt(N)
law, numpy sorting and scipy's SpMV.  A plausible slip in the oracle (a
dropped j = 0 term, a wrong sign of c, a transposed index, an off-by-one in
the sampler or the stop rule) fails at least one of them.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import synth

# ---------------------------------------------------------------- Philox


def _curand_host_blocks(seed, nblocks):
    """cuRAND's host PHILOX4_32_10 generator, read through its public C API.
    Its output block i equals Philox4x32-10(counter=(0,0,i,0), key=seed)."""
    path = None
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            path = ctypes.CDLL(p)
            break
        except OSError:
            continue
    if path is None:
        pytest.skip("libcurand not available")
    lib = path
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        lib.curandSetPseudoRandomGeneratorSeed.argtypes = [ctypes.c_void_p, ctypes.c_ulonglong]
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        lib.curandGenerate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), out.size) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(nblocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 2**64 - 1, 20240903])
def test_philox_matches_curand_host(orc, seed):
    ref = _curand_host_blocks(seed, 40)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(40):
        got = orc.philox4x32_10([0, 0, i, 0], key)
        assert np.array_equal(got, ref[i]), (seed, i)


# ---------------------------------------------------------------- split


@pytest.mark.parametrize("diag_sign", ["positive", "mixed"])
def test_split_matches_dense_jacobi(orc, diag_sign):
    m = synth.random_dd(40, 5, seed=3, diag_sign=diag_sign, zero_frac=0.1)
    B = m.to_scipy().toarray()
    d, s = orc.split(m)
    assert np.array_equal(d, np.diag(B))
    C = np.eye(m.n) - B / np.diag(B)[:, None]          # C = I - D^-1 B
    assert np.allclose(np.diag(C), 0.0)
    assert np.allclose(s, np.abs(C).sum(axis=1), rtol=1e-14, atol=0)
    # Eq. 1 augmentation with alpha ||B||_inf sgn(b_ii) (Sec. V-C)
    alpha = 0.3
    da, sa = orc.split(m, alpha=alpha)
    bn = np.abs(B).sum(axis=1).max()
    assert np.allclose(da, np.diag(B) + alpha * bn * np.where(np.diag(B) < 0, -1, 1), rtol=1e-15)
    assert np.all(sa < s)


def test_split_zero_diagonal_is_an_error(orc):
    m = synth.random_dd(10, 3, seed=1)
    dpos = [int(np.flatnonzero(m.col[m.row_ptr[i]:m.row_ptr[i + 1]] == i)[0] + m.row_ptr[i]) for i in range(m.n)]
    m.val[dpos[4]] = 0.0
    with pytest.raises(orc.OracleError) as e:
        orc.split(m)
    assert e.value.status == 3 and "row 4" in str(e.value)


# ---------------------------------------------------------------- tables


def _exact_cumulative_counts(q):
    """Number of 32-bit r that the cumulative rule maps to each entry:
    floor(r Q / 2^32) < T  <=>  r < ceil(T 2^32 / Q)."""
    Q = int(sum(int(v) for v in q))
    T = np.cumsum([int(v) for v in q])
    bounds = [0] + [-(-int(t) * 2**32 // Q) for t in T]
    return np.diff(bounds), bounds, Q


def test_table_weights_follow_transition_probabilities(orc):
    m = synth.random_dd(60, 7, seed=5, zero_frac=0.15)
    d, s = orc.split(m)
    tb = orc.tables(m, d, s)
    B = m.to_scipy().toarray()
    C = np.eye(m.n) - B / np.diag(B)[:, None]
    for i in range(m.n):
        a, b = tb["off"][i], tb["off"][i + 1]
        q = tb["q"][a:b].astype(np.float64)
        cols = [c for c in m.col[m.row_ptr[i]:m.row_ptr[i + 1]] if c != i]
        p = np.abs(C[i, cols]) / np.abs(C[i]).sum()
        Q = int(tb["Q"][i])
        assert Q == int(tb["q"][a:b].astype(np.uint64).sum())
        assert abs(Q - 2**31) <= len(q)
        assert np.all((q == 0) == (p == 0))                 # zero c never sampled, others kept
        assert np.all(np.abs(q / Q - p) <= (len(q) + 1) / Q)


def test_compact_table_weights(orc):
    """The compact table's weights at the scale 2^20: against the dense
    transition probabilities, and against the 2^31 table (dropping 11 bits
    of floor(x 2^31) is floor(x 2^20); both floor at 1 and keep zeros)."""
    m = synth.random_dd(60, 6, seed=6, zero_frac=0.15, diag_sign="mixed")
    d, s = orc.split(m)
    tc = orc.tables(m, d, s, table=orc.TABLE_COMPACT)
    t31 = orc.tables(m, d, s)
    assert np.array_equal(tc["off"], t31["off"])
    q31 = t31["q"].astype(np.int64)
    want = np.where(q31 == 0, 0, np.maximum(1, q31 >> 11))
    assert np.array_equal(tc["q"].astype(np.int64), want)
    B = m.to_scipy().toarray()
    C = np.eye(m.n) - B / np.diag(B)[:, None]
    for i in range(m.n):
        a, b = tc["off"][i], tc["off"][i + 1]
        q = tc["q"][a:b].astype(np.float64)
        cols = [c for c in m.col[m.row_ptr[i]:m.row_ptr[i + 1]] if c != i]
        p = np.abs(C[i, cols]) / np.abs(C[i]).sum()
        Q = int(tc["Q"][i])
        assert Q == int(tc["q"][a:b].astype(np.uint64).sum())
        assert abs(Q - 2**20) <= len(q) and Q < 2**21
        assert np.all((q == 0) == (p == 0))
        assert np.all(np.abs(q / Q - p) <= (len(q) + 1) / Q)


def test_cumulative_pick_boundaries_are_exact(orc):
    rng = np.random.default_rng(0)
    for trial in range(30):
        deg = int(rng.integers(1, 12))
        q = rng.integers(0, 2**28, deg).astype(np.uint32)
        q[rng.random(deg) < 0.2] = 0
        if q.sum() == 0:
            q[0] = 1
        counts, bounds, Q = _exact_cumulative_counts(q)
        # the pick switches exactly at the boundaries
        probe, want = [], []
        for m in range(deg):
            if counts[m] == 0:
                continue
            probe += [bounds[m], bounds[m + 1] - 1]
            want += [m, m]
        got = orc.pick_cumulative(q, np.array(probe, dtype=np.uint64).astype(np.uint32))
        assert np.array_equal(got, want)
        assert np.all(np.abs(counts / 2**32 - q / Q) <= 1.0 / Q + 2**-32)
        # random r against numpy's searchsorted ('smallest m with x < T_m')
        r = rng.integers(0, 2**32, 2000, dtype=np.uint64)
        x = (r * np.uint64(Q)) >> np.uint64(32)
        ref = np.searchsorted(np.cumsum(q.astype(np.uint64)), x, side="right")
        assert np.array_equal(orc.pick_cumulative(q, r.astype(np.uint32)), ref)


def _alias_exact_probs(prob, al, Q):
    """Exact probability of each pick of the alias rule, by counting r in
    closed form per bucket: r in [ceil(b 2^32/deg), ceil((b+1) 2^32/deg)),
    own entry iff (r deg - b 2^32) < ceil(prob_b 2^32 / Q)."""
    deg = len(prob)
    cnt = np.zeros(deg, dtype=object)
    for b in range(deg):
        lo = -(-b * 2**32 // deg)
        hi = -(-(b + 1) * 2**32 // deg)
        F = -(-int(prob[b]) * 2**32 // Q)
        own_hi = -(-(F + b * 2**32) // deg)            # r < own_hi <=> frac < F
        own = max(0, min(hi, own_hi) - lo)
        cnt[b] += own
        cnt[int(al[b])] += (hi - lo) - own
    return np.array([c / 2**32 for c in cnt]), cnt


def test_alias_table_conserves_mass_and_samples_p(orc):
    rng = np.random.default_rng(1)
    for trial in range(40):
        deg = int(rng.integers(1, 40))
        q = rng.integers(0, 2**26, deg).astype(np.uint32)
        q[rng.random(deg) < 0.2] = 0
        if q.sum() == 0:
            q[-1] = 5
        Q = int(q.astype(np.uint64).sum())
        prob, al = orc.alias_build(q)
        mass = np.zeros(deg, dtype=object)
        for b in range(deg):
            assert 0 <= int(prob[b]) <= Q
            mass[b] += int(prob[b])
            mass[int(al[b])] += Q - int(prob[b])
        assert all(int(mass[j]) == int(q[j]) * deg for j in range(deg))
        p, cnt = _alias_exact_probs(prob, al, Q)
        assert np.all(np.abs(p - q / Q) <= (deg + 2) / 2**32 + 1.0 / Q)
        # the oracle's pick agrees with the closed-form count on random r
        r = rng.integers(0, 2**32, 4000, dtype=np.uint64).astype(np.uint32)
        picks = orc.pick_alias(prob, al, Q, r)
        assert np.all(q[picks] > 0)
        # and at bucket edges
        for b in range(deg):
            lo = -(-b * 2**32 // deg)
            got = orc.pick_alias(prob, al, Q, np.array([lo], dtype=np.uint64).astype(np.uint32))[0]
            assert got == (b if int(prob[b]) > 0 else int(al[b]))


# ---------------------------------------------------------------- walks


def _dense_C(m):
    B = m.to_scipy().toarray()
    return np.eye(m.n) - B / np.diag(B)[:, None], np.diag(B)


def test_diagonal_matrix_gives_inverse_diagonal(orc):
    n = 17
    d = np.linspace(-3.0, 5.0, n)
    d[d == 0] = 1.5
    m = synth._from_coo(n, np.arange(n), np.arange(n), d)
    res, dd, s = orc.walk(m, chains=50, max_len=10, delta=1e-3, seed=3)
    for r in res:
        assert list(r["col"]) == [r["row"]] and r["X"][0] == 1.0 and r["V"][0] == 50 and r["steps"] == 0
    rp, col, val, steps = orc.build(m, chains=50, max_len=10, delta=1e-3, seed=3, tau=0.5, top_k=3)
    assert np.array_equal(col, np.arange(n)) and np.array_equal(val, 1.0 / d)


def _fp32_stop_len(factors, delta, L):
    """Transitions taken under the stop rule, with the single-precision shadow
    weight (numpy float32 arithmetic)."""
    w = np.float32(1.0)
    t = 0
    while t < L and not (float(abs(w)) < delta):
        w = np.float32(w * np.float32(factors[t]))
        t += 1
    return t


def test_scaled_permutation_is_a_deterministic_path(orc):
    """One off-diagonal per row: every chain follows the same path, and X is
    the truncated Neumann sum sum_t C^t of Eq. 2 exactly."""
    n = 9
    rng = np.random.default_rng(4)
    perm = rng.permutation(n)
    while np.any(perm == np.arange(n)):
        perm = rng.permutation(n)
    b = rng.uniform(0.3, 0.8, n) * np.where(rng.random(n) < 0.5, -1, 1)
    d = rng.uniform(1.0, 1.2, n) * np.where(rng.random(n) < 0.3, -1, 1)
    rows = np.concatenate([np.arange(n), np.arange(n)])
    cols = np.concatenate([perm, np.arange(n)])
    m = synth._from_coo(n, rows, cols, np.concatenate([b, d]))
    C, dd = _dense_C(m)
    delta, L = 1e-3, 25
    res, _, s = orc.walk(m, chains=7, max_len=L, delta=delta, seed=9)
    for r in res:
        i = r["row"]
        path = [i]
        for _ in range(L):
            path.append(perm[path[-1]])
        T = _fp32_stop_len([s[path[t]] for t in range(L)], delta, L)
        expect = np.zeros(n)
        Ct = np.eye(n)
        for t in range(T + 1):
            expect += Ct[i]
            Ct = Ct @ C
        X = np.zeros(n)
        X[r["col"]] = r["X"]
        assert np.allclose(X, expect, rtol=1e-13, atol=1e-15)
        assert r["steps"] == 7 * T
        assert r["V"].sum() == 7 * (T + 1)


def test_equal_row_norms_fix_every_chain_length(orc):
    """Nonnegative C with s_i = s for all i: every chain carries weights s^t
    and stops after the same T* transitions (visit invariants)."""
    m = synth.random_dd(30, 4, seed=8, signs="negative", dominance=0.7)
    d, s = orc.split(m)
    assert np.allclose(s, 0.7)
    assert len(np.unique(s.astype(np.float32))) == 1
    delta, L, N = 1e-3, 200, 40
    Tstar = _fp32_stop_len([s[0]] * L, delta, L)
    res, _, _ = orc.walk(m, chains=N, max_len=L, delta=delta, seed=2)
    for r in res:
        assert r["steps"] == N * Tstar
        assert int(r["V"].sum()) == N * (Tstar + 1)
        # all weights positive here, so A == X and sum_j X_ij = sum_t s^t
        assert np.allclose(r["A"], r["X"])
        assert np.isclose(r["X"].sum(), sum(0.7 ** t for t in range(Tstar + 1)), rtol=1e-12)
    assert orc.max_walk_len(s.max(), delta, L) == Tstar


def _enumerate_paths(m, q_tab, i, L, delta, use_true_p=False):
    """Exact E[Y] and E[Y^2] of one chain's contribution Y_j = sum_{t: s_t=j} W_t
    by enumerating every path (with the table's probabilities q/Q, or the
    exact |c|/s), applying the stop rule with the float32 shadow weight."""
    C, dd = _dense_C(m)
    n = m.n
    s = np.abs(C).sum(axis=1)
    EY = np.zeros(n)
    EY2 = np.zeros(n)
    offs = q_tab["off"]

    def rec(state, w, w32, t, prob, Y):
        Y = Y.copy()
        Y[state] += w
        stop = t == L or float(abs(w32)) < delta or s[state] == 0.0
        if stop:
            EY[:] += prob * Y
            EY2[:] += prob * Y * Y
            return
        cols = [c for c in m.col[m.row_ptr[state]:m.row_ptr[state + 1]] if c != state]
        a = offs[state]
        Q = float(q_tab["Q"][state])
        for k, c in enumerate(cols):
            p = abs(C[state, c]) / s[state] if use_true_p else q_tab["q"][a + k] / Q
            if p == 0:
                continue
            f = np.sign(C[state, c]) * s[state]
            w32n = np.float32(w32 * np.float32(np.sign(C[state, c]) * np.float32(s[state])))
            rec(c, w * f, w32n, t + 1, prob * p, Y)

    rec(i, 1.0, np.float32(1.0), 0, 1.0, np.zeros(n))
    return EY, EY2


def test_path_enumeration_reproduces_neumann_powers(orc):
    """Without cutoff, E[X_i.] over all paths with p = |c|/s is the truncated
    Neumann row sum_{t<=L} (C^t)_i. (checks the enumerator used below)."""
    m = synth.random_dd(5, 3, seed=11, dominance=0.8, diag_sign="mixed")
    C, _ = _dense_C(m)
    d, s = orc.split(m)
    tb = orc.tables(m, d, s)
    L = 4
    P = sum(np.linalg.matrix_power(C, t) for t in range(L + 1))
    for i in range(m.n):
        EY, _ = _enumerate_paths(m, tb, i, L, 0.0, use_true_p=True)
        assert np.allclose(EY, P[i], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("delta,L,table", [(0.0, 4, 0), (0.2, 6, 0), (0.05, 5, 1), (0.05, 5, 3)])
def test_estimator_mean_matches_exact_expectation(orc, delta, L, table):
    """z-scores of the oracle's Eq. 2 estimate against the exact expectation
    and variance from path enumeration (n = 5), with the probabilities q/Q
    of the table the walks sample (the compact table's are coarser)."""
    m = synth.random_dd(5, 3, seed=21, dominance=0.85, diag_sign="mixed")
    d, s = orc.split(m)
    tb = orc.tables(m, d, s, table=table if table == 3 else 0)
    N = 200_000
    res, _, _ = orc.walk(m, chains=N, max_len=L, delta=delta, seed=77, table=table)
    worst = 0.0
    for r in res:
        EY, EY2 = _enumerate_paths(m, tb, r["row"], L, delta)
        var = np.maximum(EY2 - EY * EY, 0.0)
        X = np.zeros(m.n)
        X[r["col"]] = r["X"]
        ok = var > 0
        z = np.abs(X[ok] - EY[ok]) / np.sqrt(var[ok] / N)
        worst = max(worst, z.max(initial=0.0))
        assert np.allclose(X[~ok], EY[~ok], rtol=1e-12, atol=1e-14)   # zero-variance entries exact
    assert worst < 5.0


def test_estimate_converges_to_inverse(orc):
    """With a tiny cutoff and long walks, X D^-1 -> B^-1 (Eq. 2 + phase 4)."""
    m = synth.random_dd(16, 3, seed=31, dominance=0.5, diag_sign="mixed")
    B = m.to_scipy().toarray()
    res, d, s = orc.walk(m, chains=100_000, max_len=200, delta=1e-12, seed=5)
    M = np.zeros((m.n, m.n))
    for r in res:
        M[r["row"], r["col"]] = r["X"] / d[r["col"]]
    Binv = np.linalg.inv(B)
    assert np.linalg.norm(M - Binv) / np.linalg.norm(Binv) < 0.01


def test_error_decays_as_inverse_sqrt_chains(orc):
    m = synth.random_dd(8, 3, seed=41, dominance=0.5, diag_sign="mixed")
    B = m.to_scipy().toarray()
    Binv = np.linalg.inv(B)
    Ns = [100, 400, 1600, 6400, 25600, 102400]
    rms = []
    for N in Ns:
        errs = []
        for seed in range(16):
            res, d, s = orc.walk(m, chains=N, max_len=200, delta=1e-10, seed=1000 + seed)
            M = np.zeros((m.n, m.n))
            for r in res:
                M[r["row"], r["col"]] = r["X"] / d[r["col"]]
            errs.append(np.mean((M - Binv) ** 2))
        rms.append(math.sqrt(np.mean(errs)))
    slope = np.polyfit(np.log(Ns), np.log(rms), 1)[0]
    # slope -1/2 within 0.05 (16 seeds per N: four seed bases gave -0.491 to -0.497)
    assert -0.55 < slope < -0.45, slope


def test_visit_counts_add_up_and_rows_are_independent(orc):
    m = synth.random_dd(50, 6, seed=13, dominance=0.9, diag_sign="mixed", dominance_jitter=0.5)
    full, _, _ = orc.walk(m, chains=64, max_len=40, delta=1e-3, seed=99)
    for r in full:
        assert int(r["V"].sum()) == 64 + r["steps"]
        assert r["row"] in set(r["col"].tolist())
    sub, _, _ = orc.walk(m, rows=[37, 2, 11], chains=64, max_len=40, delta=1e-3, seed=99)
    for r in sub:
        f = full[r["row"]]
        for k in ("col", "X", "A", "V"):
            assert np.array_equal(r[k], f[k])


def test_first_steps_follow_the_table(orc):
    """Chi-square of first transitions of row 0 against q/Q: walks of max
    length 1 visit the start and exactly one neighbour."""
    m = synth.random_dd(40, 12, seed=17, dominance=0.9)
    d, s = orc.split(m)
    tb = orc.tables(m, d, s)
    N = 100_000
    for table in (0, 1):
        res, _, _ = orc.walk(m, rows=[0], chains=N, max_len=1, delta=0.0, seed=3, table=table)
        r = res[0]
        cols = [c for c in m.col[m.row_ptr[0]:m.row_ptr[1]] if c != 0]
        q = tb["q"][tb["off"][0]:tb["off"][1]].astype(np.float64)
        exp = N * q / q.sum()
        obs = np.array([r["V"][list(r["col"]).index(c)] if c in set(r["col"]) else 0 for c in cols])
        chi2 = float(np.sum((obs - exp) ** 2 / exp))
        assert chi2 < 40.0, chi2      # 11 d.o.f.: p ~ 4e-5


@pytest.mark.parametrize("table", [0, 3])
def test_python_rewalk_of_a_few_chains(orc, table):
    """Brute force: re-walk two chains in Python from the oracle's Philox
    and numpy's searchsorted, and compare the visit counts (cumulative and
    compact tables)."""
    m = synth.random_dd(12, 4, seed=23, dominance=0.8, diag_sign="mixed")
    d, s = orc.split(m)
    tb = orc.tables(m, d, s, table=table)
    C, _ = _dense_C(m)
    seed, delta, L, N = 0xDEADBEEF12345, 1e-2, 30, 2
    key = [seed & 0xFFFFFFFF, seed >> 32]
    res, _, _ = orc.walk(m, rows=[5], chains=N, max_len=L, delta=delta, seed=seed, table=table)
    V = np.zeros(m.n, dtype=np.int64)
    X = np.zeros(m.n)
    for k in range(N):
        st, w, w32, t = 5, 1.0, np.float32(1.0), 0
        V[st] += 1; X[st] += w
        while t < L and not (float(abs(w32)) < delta):
            r = orc.philox4x32_10([t // 4, k, 5, 0], key)[t % 4]
            a, b = tb["off"][st], tb["off"][st + 1]
            q = tb["q"][a:b].astype(np.uint64)
            x = (np.uint64(r) * np.uint64(q.sum())) >> np.uint64(32)
            mm = int(np.searchsorted(np.cumsum(q), x, side="right"))
            cols = [c for c in m.col[m.row_ptr[st]:m.row_ptr[st + 1]] if c != st]
            nxt = cols[mm]
            sg = np.sign(C[st, nxt])
            w *= sg * s[st]
            w32 = np.float32(w32 * np.float32(sg * np.float32(s[st])))
            st = nxt; t += 1
            V[st] += 1; X[st] += w
    r = res[0]
    assert np.array_equal(np.flatnonzero(V), r["col"])
    assert np.array_equal(V[r["col"]], r["V"])
    assert np.allclose(X[r["col"]] / N, r["X"], rtol=1e-15)


# ---------------------------------------------------------------- filter, spmv


def test_filter_matches_numpy_ranking(orc):
    rng = np.random.default_rng(7)
    for trial in range(200):
        cnt = int(rng.integers(1, 60))
        cols = np.sort(rng.choice(500, cnt, replace=False)).astype(np.int32)
        i = int(cols[rng.integers(0, cnt)]) if rng.random() < 0.9 else 1000
        vals = rng.choice([-2.0, -1.0, -0.5, 0.25, 0.5, 1.0, 3.0], cnt) * rng.choice([1.0, 1.0, 1e-3], cnt)
        tau = float(rng.choice([0.0, 1e-2, 0.3]))
        k = int(rng.choice([0, 1, 4, 16]))
        oc, ov = orc.filter_row(i, cols, vals, tau=tau, top_k=k)
        mx = np.abs(vals).max()
        off = cols != i
        cand = np.flatnonzero(off & ((tau == 0.0) | (np.abs(vals) >= tau * mx)))
        if k > 0 and len(cand) > k:
            order = np.lexsort((cols[cand], -np.abs(vals[cand])))
            cand = cand[order[:k]]
        keep = np.sort(np.concatenate([cand, np.flatnonzero(~off)]))
        assert np.array_equal(oc, cols[keep]) and np.array_equal(ov, vals[keep])


def test_spmv_matches_scipy(orc):
    m = synth.random_dd(300, 9, seed=2)
    x = np.random.default_rng(0).standard_normal(m.n)
    assert np.allclose(orc.spmv(m.row_ptr, m.col, m.val, x), m.to_scipy() @ x, rtol=1e-13)


# ---------------------------------------------------------------- matrix reduction (Algorithm 1, step 2)


def _offdiag(m):
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    return m.col != rows


@pytest.mark.parametrize("fraction", [0.0, 0.1, 0.37, 0.5, 0.93, 1.0])
def test_reduce_entries_drops_the_smallest_ties_by_position(fraction):
    import oracle
    m = synth.random_dd(300, 7, seed=11, diag_sign="mixed")
    off = _offdiag(m)
    # many equal magnitudes, both signs: ties at the cut
    m.val[off] = np.round(m.val[off], 1)
    r, keep, d = oracle.reduce(m, fraction, oracle.REDUCE_ENTRIES)
    noff = int(off.sum())
    a = np.abs(m.val)
    assert d == int(np.floor(fraction * noff)) and int((~keep).sum()) == d
    assert keep[~off].all()                                    # the diagonal stays
    if 0 < d < noff:
        assert a[off & ~keep].max() <= a[off & keep].min()     # every dropped entry <= every kept one
        b = a[off & ~keep].max()
        tie = np.flatnonzero(off & (a == b))
        assert np.all(np.diff(keep[tie].astype(int)) >= 0)     # equal magnitudes: earlier entries dropped first
    # the same set from numpy's lexsort on (|b|, position)
    pos = np.flatnonzero(off)
    first = pos[np.lexsort((pos, a[off]))][:d]
    assert set(first.tolist()) == set(np.flatnonzero(~keep).tolist())
    # the reduced CSR keeps the remaining entries in order
    assert np.array_equal(r.col, m.col[keep]) and np.array_equal(r.val, m.val[keep])
    assert np.array_equal(np.diff(r.row_ptr), [keep[m.row_ptr[i]:m.row_ptr[i + 1]].sum() for i in range(m.n)])


def test_reduce_range_closed_form():
    """Off-diagonal magnitudes 1..100 (alternating signs): the cut at
    lo + f (hi - lo) = 1 + 99 f drops exactly the values below it."""
    import oracle
    n = 101
    rows, cols, vals = [], [], []
    for i in range(n):
        rows.append(i); cols.append(i); vals.append(1000.0)
        if i < 100:
            rows.append(i); cols.append((i + 7) % n); vals.append((i + 1.0) * (-1) ** i)
    m = synth._from_coo(n, np.array(rows), np.array(cols), np.array(vals))
    for f, expect in [(0.0, 0), (0.5, 50), (0.25, 25), (1.0, 99), (0.004, 1), (0.011, 2)]:
        r, keep, d = oracle.reduce(m, f, oracle.REDUCE_RANGE)
        assert d == expect, (f, d)
        kept = np.abs(r.val[_offdiag(r)])
        assert kept.min(initial=np.inf) >= 1 + 99 * f - 1e-12
    # the 0.5 cut: values 1..50 go, 51..100 stay
    r, keep, d = oracle.reduce(m, 0.5, oracle.REDUCE_RANGE)
    assert sorted(np.abs(r.val[_offdiag(r)]).tolist()) == [float(v) for v in range(51, 101)]


def test_reduce_keeps_the_diagonal_and_handles_diagonal_matrices():
    import oracle

    def csr(n, r, c, v):
        return synth._from_coo(n, np.array(r), np.array(c), np.array(v, dtype=np.float64))
    m = csr(4, [0, 1, 2, 3, 0], [0, 1, 2, 3, 3], [2.0, 3.0, -4.0, 5.0, 0.5])
    r, keep, d = oracle.reduce(m, 1.0, oracle.REDUCE_ENTRIES)      # every off-diagonal entry goes
    assert d == 1 and r.nnz == 4 and np.array_equal(r.col, [0, 1, 2, 3])
    r, keep, d = oracle.reduce(m, 1.0, oracle.REDUCE_RANGE)        # the largest off-diagonal |b| stays
    assert d == 0 and r.nnz == 5
    d0 = csr(3, [0, 1, 2], [0, 1, 2], [1.0, 2.0, 3.0])
    r, keep, d = oracle.reduce(d0, 0.5, oracle.REDUCE_ENTRIES)
    assert d == 0 and r.nnz == 3
    with pytest.raises(ValueError):
        oracle.reduce(d0, 1.5, oracle.REDUCE_ENTRIES)


# ---------------------------------------------------------------- recovery of B^-1 (Eq. 3, Algorithm 1 step 5)


@pytest.mark.parametrize("alpha", [0.3, 1.0, 4.0])
def test_recovery_of_the_exact_inverse_is_the_inverse(alpha):
    """Sherman-Morrison is exact: from Bhat^-1 (numpy) the n rank-one
    updates of Eq. 3 give B^-1 (numpy) up to rounding."""
    import oracle
    m = synth.random_dd(80, 6, seed=5, dominance=1.3, diag_sign="mixed")
    s = oracle.augmentation(m, alpha)
    B = m.to_scipy().toarray()
    d1, _ = oracle.split(m, alpha)
    Bh = B.copy()
    Bh[np.diag_indices(m.n)] = d1
    assert np.array_equal(np.diag(Bh) - np.diag(B), s)
    X = oracle.recover_dense(np.linalg.inv(Bh), s)
    ref = np.linalg.inv(B)
    assert np.abs(X - ref).max() <= 1e-9 * np.abs(ref).max()


def test_recovery_without_augmentation_changes_nothing():
    import oracle
    rng = np.random.default_rng(1)
    X = rng.standard_normal((30, 30))
    Y = oracle.recover_dense(X, np.zeros(30))
    assert np.array_equal(X, Y)


def test_recovery_of_one_diagonal_change():
    """One nonzero s_i: the recovery inverts Bhat - s_i e_i e_i^T (numpy)."""
    import oracle
    rng = np.random.default_rng(2)
    A = rng.standard_normal((25, 25)) + 25 * np.eye(25)
    s = np.zeros(25)
    s[7] = 3.5
    X = oracle.recover_dense(np.linalg.inv(A), s)
    ref = np.linalg.inv(A - np.diag(s))
    assert np.abs(X - ref).max() <= 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------- hybrid table (per-row table type)


def test_hybrid_table_is_cumulative_on_short_rows_and_alias_on_long_rows():
    import oracle
    short = synth.stencil3d_7pt(6, seed=3)                     # every row has at most 6 transitions
    long_ = synth.random_dd(300, 12, seed=4, dominance=0.8)     # every row has 12
    kw = dict(chains=64, max_len=40, delta=1e-3, seed=9)
    for m, same in ((short, oracle.TABLE_CUMULATIVE), (long_, oracle.TABLE_ALIAS)):
        a, _, _ = oracle.walk(m, table=oracle.TABLE_HYBRID, **kw)
        b, _, _ = oracle.walk(m, table=same, **kw)
        for x, y in zip(a, b):
            assert np.array_equal(x["col"], y["col"]) and np.array_equal(x["V"], y["V"])
            assert np.array_equal(x["X"], y["X"]) and x["steps"] == y["steps"]


def test_hybrid_table_on_mixed_rows_is_unbiased():
    """Rows of 4 to 256 transitions: the hybrid table's estimate converges to
    the same expectation as the others (z-scores against the exact Neumann
    sum of the table's probabilities are checked by the estimator pins; here
    the three tables agree within their Monte Carlo error)."""
    import oracle
    m = synth.powerlaw_random(300, seed=8, dominance=0.7)
    deg = np.diff(m.row_ptr) - 1
    assert (deg <= 6).any() and (deg > 6).any()
    rows = np.arange(0, 300, 23)
    est = {}
    for t in (oracle.TABLE_CUMULATIVE, oracle.TABLE_ALIAS, oracle.TABLE_HYBRID):
        orows, d, s = oracle.walk(m, rows=rows, chains=20000, max_len=60, delta=1e-6, seed=17, table=t)
        est[t] = orows
    for k in range(len(rows)):
        xc = np.zeros(m.n); xc[est[0][k]["col"]] = est[0][k]["X"]
        xh = np.zeros(m.n); xh[est[2][k]["col"]] = est[2][k]["X"]
        xa = np.zeros(m.n); xa[est[1][k]["col"]] = est[1][k]["X"]
        scale = np.linalg.norm(xc)
        assert np.linalg.norm(xh - xc) / scale < 0.02 and np.linalg.norm(xh - xa) / scale < 0.02


# ---------------------------------------------------------------- chains from epsilon


@pytest.mark.parametrize("smax,eps", [(0.3, 0.01), (0.6, 0.02), (0.9, 0.05)])
def test_chains_from_eps_meets_its_probable_error_on_the_extremal_estimator(orc, smax, eps):
    """The rule claims: with N chains the probable error (the median of
    |error|) of an estimate whose single-chain contribution has standard
    deviation at most 1/(1 - ||C||) is at most eps.  A fair coin of
    +-1/(1 - smax) attains that deviation, so the mean of N of them must fall
    inside +-eps with probability 1/2 (exact binomial law; the lattice of
    the mean moves it by a few 1e-3 at these N).  Half or twice the chains
    must be clearly on either side."""
    from scipy.stats import binom
    a = 1.0 / (1.0 - smax)

    def p_inside(N):
        # |mean| = a |2K - N| / N < eps  <=>  |2K - N| < eps N / a
        lim = eps * N / a
        k_lo = math.floor((N - lim) / 2) + 1
        k_hi = math.ceil((N + lim) / 2) - 1
        return float(binom.cdf(k_hi, N, 0.5) - binom.cdf(k_lo - 1, N, 0.5))

    N = orc.chains_from_eps(eps, smax)
    assert N > 2000
    assert abs(p_inside(N) - 0.5) < 0.02, (N, p_inside(N))
    assert p_inside(N // 2) < 0.4 and p_inside(2 * N) > 0.6


def test_chains_from_eps_bounds_the_walks_per_entry_error(orc):
    """With N from the rule, the walks' per-entry error against the exact
    expectation (path enumeration, n = 5, no cutoff, L = 6) is below eps in
    at least half of independent trials: one binomial sample per (row,
    seed), the entry of the row with the largest single-chain variance, and
    a one-sided bound three standard deviations below 1/2."""
    m = synth.random_dd(5, 3, seed=23, dominance=0.6, diag_sign="mixed")
    d, s = orc.split(m)
    tb = orc.tables(m, d, s)
    L, eps = 6, 0.02
    N = orc.chains_from_eps(eps, float(s.max()))
    mean, col = {}, {}
    for i in range(m.n):
        EY, EY2 = _enumerate_paths(m, tb, i, L, 0.0)
        var = EY2 - EY * EY
        # the single-chain deviation the rule bounds
        assert np.sqrt(var.max()) <= sum(float(s.max()) ** t for t in range(L + 1)) + 1e-12
        col[i] = int(np.argmax(var))
        mean[i] = EY[col[i]]
    T = inside = 0
    for seed in range(120):
        res, _, _ = orc.walk(m, chains=N, max_len=L, delta=0.0, seed=9000 + seed)
        for r in res:
            i = int(r["row"])
            X = dict(zip(r["col"].tolist(), r["X"].tolist()))
            inside += abs(X.get(col[i], 0.0) - mean[i]) < eps
            T += 1
    assert inside / T - 3.0 * math.sqrt(0.25 / T) >= 0.5, (inside, T, N)


# ---------------------------------------------------------------- compact table bias


@pytest.mark.parametrize("table,scale", [(3, 2.0 ** 20), (0, 2.0 ** 31)])
def test_table_expectation_is_within_the_quantisation_bound_of_neumann(orc, table, scale):
    """The walks sample p^ = q/Q (q = max(1, floor(p scale))) but multiply by
    sign(c) s, so their exact expectation (path enumeration) is the Neumann
    sum of C^ = p^ sign(c) s, not of C.  With ||C^ - C||_inf <= eta =
    s_max 2 deg_max / (scale - deg_max) and ||C^||_inf = ||C||_inf = s_max,
    each row's L1 distance to sum_{t<=L} C^t is at most
    eta sum_{t=1}^{L} t s_max^(t-1).  The compact table's bias must also be
    visible (above 2^-31-level noise), so the enumeration sees its q."""
    m = synth.random_dd(5, 3, seed=29, dominance=0.8, diag_sign="mixed")
    C, _ = _dense_C(m)
    d, s = orc.split(m)
    tb = orc.tables(m, d, s, table=table)
    L = 5
    P = sum(np.linalg.matrix_power(C, t) for t in range(L + 1))
    degmax = int(max(np.count_nonzero(C[i]) for i in range(m.n)))
    smax = float(s.max())
    eta = smax * 2 * degmax / (scale - degmax)
    bound = eta * sum(t * smax ** (t - 1) for t in range(1, L + 1))
    worst = 0.0
    for i in range(m.n):
        EY, _ = _enumerate_paths(m, tb, i, L, 0.0)
        dist = float(np.abs(EY - P[i]).sum())
        assert dist <= bound, (i, dist, bound)
        worst = max(worst, dist)
    if table == 3:
        assert worst > 1e-3 * bound and worst > 1e-8, worst
