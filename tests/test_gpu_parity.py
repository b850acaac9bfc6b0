"""CUDA path vs the CPU oracle, through the C ABI.

Bit-exact: the split (d, s), the integer tables, every walk's visited
columns, visit counts and transition counts.  Floating point: entries within
1e-5 relative (bounded by (1/N) sum |W| / |d_j| where signed weights cancel).
Filtered patterns equal except entries inside the rounding band of a cut.
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


def _orc():
    import oracle
    return oracle


def _cases_small():
    return {
        "rand_mixed": synth.random_dd(300, 5, seed=1, diag_sign="mixed", zero_frac=0.1, dominance=0.85),
        "rand_long": synth.random_dd(500, 23, seed=2, dominance=0.8, dominance_jitter=0.3),
        "stencil2d": synth.stencil2d_5pt(32, 32, seed=1001),
        "stencil3d_12": synth.stencil3d_7pt(12, seed=7),
        "powerlaw_4k": synth.powerlaw_random(4096, seed=3),
    }


# ------------------------------------------------------------------ tables


@pytest.mark.parametrize("name", list(_cases_small()))
@pytest.mark.parametrize("table", [0, 1, 2])
def test_tables_bit_exact(name, table):
    """Table 2 (hybrid): rows of at most 6 transitions hold the inline
    cumulative record (flag bit 30), longer rows the alias buckets."""
    orc = _orc()
    m = _cases_small()[name]
    B = mc.DeviceCsr.from_host(m)
    g = mc.mcmi_debug_tables(B, mc.params(table=table))
    d, s = orc.split(m)
    assert np.array_equal(g["d"], d) and np.array_equal(g["s"], s)
    tbc = orc.tables(m, d, s, alias=False)
    tba = orc.tables(m, d, s, alias=True)
    tb = tba if table == 1 else tbc
    slot = g["slot"]
    assert np.array_equal(slot[:, 0], tb["Q"].astype(np.uint32))
    assert np.array_equal(slot[:, 1], s.astype(np.float32).view(np.uint32))
    assert np.array_equal(slot[:, 2], (1.0 / d).astype(np.float32).view(np.uint32))
    for i in range(m.n):
        a, b = tb["off"][i], tb["off"][i + 1]
        deg = b - a
        cols = np.array([c for c in m.col[m.row_ptr[i]:m.row_ptr[i + 1]] if c != i], dtype=np.int64)
        vals = np.array([v for c, v in zip(m.col[m.row_ptr[i]:m.row_ptr[i + 1]], m.val[m.row_ptr[i]:m.row_ptr[i + 1]]) if c != i])
        cs = (cols | np.where(-vals / d[i] < 0, 1 << 31, 0)).astype(np.uint32)
        kind = table if table != 2 else (0 if deg <= 6 else 1)
        tb = tbc if kind == 0 else tba
        inline = deg <= (6 if kind == 0 else 4)
        assert slot[i, 3] == (deg | (0 if inline else 1 << 31) | (1 << 30 if table == 2 and kind == 0 else 0))
        if kind == 0:
            T = np.cumsum(tb["q"][a:b].astype(np.uint64)).astype(np.uint32)
            if inline:
                assert np.array_equal(slot[i, 4:4 + 2 * deg:2], T) and np.array_equal(slot[i, 5:5 + 2 * deg:2], cs)
                assert np.all(slot[i, 4 + 2 * deg:16:2] == 0xFFFFFFFF)
            else:
                o = slot[i, 4]
                assert np.array_equal(g["a"][o:o + deg], T) and np.array_equal(g["b"][o:o + deg], cs)
        else:
            prob, al = tb["prob"][a:b], tb["alias"][a:b]
            if inline:
                got = slot[i, 4:4 + 3 * deg].reshape(deg, 3) if deg else np.zeros((0, 3), np.uint32)
            else:
                o = slot[i, 4]
                got = np.stack([g["a"][o:o + deg], g["b"][o:o + deg], g["c"][o:o + deg]], axis=1)
            assert np.array_equal(got[:, 0], prob) and np.array_equal(got[:, 1], cs) and np.array_equal(got[:, 2], cs[al])


@pytest.mark.parametrize("table", [0, 1, 2])
def test_tables_independent_of_row_order(table):
    """From 2^16 rows on, the split and table kernels take the rows in order
    of CSR row length.  A row's split and table depend only on its own entries
    (and its offset), so the 4096 power-law rows (checked against the oracle
    by test_tables_bit_exact) must come out the same when they open a matrix
    of 2^16 + 4096 rows whose other rows are diagonal only."""
    small = _cases_small()["powerlaw_4k"]
    n = (1 << 16) + small.n
    extra = n - small.n
    big = synth.Csr(n, np.concatenate([small.row_ptr, small.nnz + np.arange(1, extra + 1, dtype=np.int64)]),
                    np.concatenate([small.col, np.arange(small.n, n, dtype=np.int32)]),
                    np.concatenate([small.val, np.ones(extra)]))
    gs = mc.mcmi_debug_tables(mc.DeviceCsr.from_host(small), mc.params(table=table))
    gb = mc.mcmi_debug_tables(mc.DeviceCsr.from_host(big), mc.params(table=table))
    k, z = small.n, small.nnz
    assert np.array_equal(gb["d"][:k], gs["d"]) and np.array_equal(gb["s"][:k], gs["s"])
    assert np.array_equal(gb["slot"][:k], gs["slot"])
    for a in ("a", "b", "c"):
        assert np.array_equal(gb[a][:z], gs[a][:z])


@pytest.mark.parametrize("name", ["stencil2d", "stencil3d_12"])
def test_compact_tables_bit_exact(name):
    """The compact table's 32-byte records against the oracle's weights at
    the scale 2^20: fl32(s_i), Q and the cumulative thresholds in 21-bit
    fields (thresholds past the last transition hold Q), and per transition
    (j - i) << 1 | sign(c_ij) in 16 bits."""
    orc = _orc()
    m = _cases_small()[name]
    B = mc.DeviceCsr.from_host(m)
    g = mc.mcmi_debug_tables(B, mc.params(table=mc.TABLE_COMPACT))
    d, s = orc.split(m)
    tb = orc.tables(m, d, s, table=orc.TABLE_COMPACT)
    rec = g["rec32"].astype(np.uint64)
    assert np.array_equal(rec[:, 0].astype(np.uint32), s.astype(np.float32).view(np.uint32))
    A = rec[:, 1] | (rec[:, 2] << np.uint64(32))
    Bt = rec[:, 3] | (rec[:, 4] << np.uint64(32))
    f = lambda x, k: ((x >> np.uint64(21 * k)) & np.uint64(0x1FFFFF)).astype(np.int64)
    assert np.array_equal(f(A, 0), tb["Q"].astype(np.int64))
    for i in range(m.n):
        a, b = tb["off"][i], tb["off"][i + 1]
        deg = b - a
        T = np.cumsum(tb["q"][a:b].astype(np.int64))
        Q = int(tb["Q"][i])
        got_T = [f(A, 1)[i], f(A, 2)[i], f(Bt, 0)[i], f(Bt, 1)[i], f(Bt, 2)[i]]
        want_T = [int(T[k]) if k < deg else Q for k in range(5)]
        assert got_T == want_T, (i, got_T, want_T)
        cols = np.array([c for c in m.col[m.row_ptr[i]:m.row_ptr[i + 1]] if c != i], dtype=np.int64)
        vals = np.array([v for c, v in zip(m.col[m.row_ptr[i]:m.row_ptr[i + 1]], m.val[m.row_ptr[i]:m.row_ptr[i + 1]]) if c != i])
        h = [(int(rec[i, 5 + k // 2]) >> (16 * (k % 2))) & 0xFFFF for k in range(deg)]
        off = [((x ^ 0x8000) - 0x8000) >> 1 for x in h]
        neg = [x & 1 for x in h]
        assert off == list(cols - i) and neg == [int(-v / d[i] < 0) for v in vals]


def _banded(n, far, seed):
    """Tridiagonal plus one entry `far` columns to the right of every row that
    has room (and one to the left of the rows it reaches), signs mixed."""
    rng = np.random.default_rng(seed)
    r, c, v = [], [], []
    for i in range(n):
        nb = [j for j in (i - 1, i + 1, i + far, i - far) if 0 <= j < n]
        w = rng.uniform(0.2, 1.0, len(nb)) * rng.choice([-1.0, 1.0], len(nb))
        r += [i] * (len(nb) + 1)
        c += nb + [i]
        v += list(w) + [np.abs(w).sum() / 0.8]
    return synth._from_coo(n, r, c, v)


def test_compact_table_column_offset_limit():
    """|j - i| = 16383 fits the compact record's 16-bit offsets (walks
    bit-exact against the oracle, both signs of the offset); 16384 does not
    (AUTO takes the cumulative table, an explicit request is refused)."""
    orc = _orc()
    m = _banded(20000, 16383, seed=3)
    B = mc.DeviceCsr.from_host(m)
    p = mc.params(chains=64, max_len=64, delta=1e-3, seed=9)
    assert mc.mcmi_build_ex(B, p).stats.table == mc.TABLE_COMPACT
    rows = np.array([0, 1, 3616, 16382, 16383, 16384, 19999], dtype=np.int64)
    orows, d, _ = orc.walk(m, rows=rows, chains=64, max_len=64, delta=1e-3, seed=9, table=orc.TABLE_COMPACT)
    grows = mc.mcmi_walk_dump(B, mc.params(chains=64, max_len=64, delta=1e-3, seed=9, table=mc.TABLE_COMPACT),
                              rows, max(len(r["col"]) for r in orows) + 16)
    assert P.compare_dump(grows, orows, d)[2] <= 1.0
    m2 = _banded(20000, 16384, seed=3)
    B2 = mc.DeviceCsr.from_host(m2)
    assert mc.mcmi_build_ex(B2, p).stats.table == mc.TABLE_CUMULATIVE
    with pytest.raises(mc.McmiError) as e:
        mc.mcmi_build_ex(B2, mc.params(chains=8, max_len=8, table=mc.TABLE_COMPACT))
    assert e.value.status == 1


def test_compact_table_refuses_rows_that_do_not_fit():
    for name in ("rand_long", "powerlaw_4k"):
        B = mc.DeviceCsr.from_host(_cases_small()[name])
        with pytest.raises(mc.McmiError) as e:
            mc.mcmi_build_ex(B, mc.params(chains=8, max_len=8, table=mc.TABLE_COMPACT))
        assert e.value.status == 1
    B = mc.DeviceCsr.from_host(_cases_small()["stencil2d"])
    with pytest.raises(mc.McmiError) as e:
        mc.mcmi_build_ex(B, mc.params(chains=8, max_len=8, table=mc.TABLE_COMPACT, accumulator=1))
    assert e.value.status == 1
    # the automatic choice: compact for the stencil, not for the long rows
    assert mc.mcmi_build_ex(B, mc.params(chains=8, max_len=8)).stats.table == mc.TABLE_COMPACT
    R = mc.DeviceCsr.from_host(_cases_small()["rand_long"])
    assert mc.mcmi_build_ex(R, mc.params(chains=8, max_len=8)).stats.table != mc.TABLE_COMPACT
    assert mc.mcmi_build_ex(B, mc.params(chains=8, max_len=8, accumulator=1)).stats.table == mc.TABLE_CUMULATIVE


# ------------------------------------------------------------------ walks


WALK_CASES = [
    # name, precision, table, N, L, delta, extra params
    ("stencil2d", 64, 0, 1000, 64, 1e-3, {}),
    ("stencil2d", 32, 0, 1000, 64, 1e-3, {}),
    ("stencil3d_12", 32, 0, 256, 128, 1e-2, {}),
    ("stencil3d_12", 32, 1, 256, 128, 1e-2, {}),
    ("rand_mixed", 32, 0, 300, 80, 1e-4, {}),
    ("rand_mixed", 64, 1, 100, 80, 1e-4, {}),
    ("rand_long", 32, 1, 128, 256, 1e-3, {}),
    ("rand_long", 32, 0, 128, 256, 1e-3, {"threads": 128}),
    ("rand_long", 32, 1, 300, 256, 1e-3, {"threads": 64, "chains_per_thread": 2}),   # refill: 300 chains on 128 slots
    ("stencil3d_12", 32, 0, 256, 128, 1e-2, {"threads": 256, "chains_per_thread": 1}),
    ("stencil2d", 64, 1, 1000, 64, 1e-3, {"threads": 128, "chains_per_thread": 2}),
    ("powerlaw_4k", 32, 1, 128, 256, 1e-3, {}),
    ("powerlaw_4k", 32, 0, 128, 256, 1e-3, {"hash_log2": 6}),      # forces the overflow log
    # hybrid table: inline cumulative rows (<= 6 transitions) and alias rows in one walk
    ("powerlaw_4k", 32, 2, 128, 256, 1e-3, {}),
    ("powerlaw_4k", 64, 2, 128, 256, 1e-3, {"hash_log2": 6}),
    ("rand_mixed", 32, 2, 300, 80, 1e-4, {"threads": 64, "chains_per_thread": 2}),
    ("rand_long", 32, 2, 128, 256, 1e-3, {"accumulator": 1}),
    ("powerlaw_4k", 64, 1, 128, 256, 1e-3, {"hash_log2": 6}),
    ("rand_long", 32, 1, 300, 256, 1e-3, {"hash_log2": 8, "threads": 64, "chains_per_thread": 2}),
    ("stencil2d", 32, 0, 1000, 64, 1e-3, {"hash_log2": 7, "threads": 64}),
    # compact table: 32-byte records, weights at the scale 2^20
    ("stencil2d", 64, 3, 1000, 64, 1e-3, {}),
    ("stencil2d", 32, 3, 1000, 64, 1e-3, {"hash_log2": 7, "threads": 64}),   # log entries look up 1/d_j
    ("stencil3d_12", 32, 3, 256, 128, 1e-2, {"threads": 128, "chains_per_thread": 2}),
    ("stencil3d_12", 64, 3, 256, 128, 1e-2, {"hash_log2": 6}),
    # the FP32 Kahan accumulator
    ("stencil3d_12", 32, 0, 256, 128, 1e-2, {"accumulator": 1}),
    ("rand_mixed", 32, 1, 300, 80, 1e-4, {"accumulator": 1}),
    ("powerlaw_4k", 32, 1, 128, 256, 1e-3, {"accumulator": 1, "hash_log2": 6}),
]


@pytest.mark.parametrize("case", WALK_CASES, ids=lambda c: f"{c[0]}-fp{c[1]}-t{c[2]}-{c[6]}")
def test_walk_paths_and_visits_bit_exact(case):
    orc = _orc()
    name, prec, table, N, L, delta, extra = case
    m = _cases_small()[name]
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([[0, m.n - 1], rng.choice(m.n, min(m.n, 48), replace=False)]))
    seed = 0x5EED0000 + N
    B = mc.DeviceCsr.from_host(m)
    p = mc.params(chains=N, max_len=L, delta=delta, seed=seed, precision=prec, table=table, **extra)
    orows, d, s = orc.walk(m, rows=rows, chains=N, max_len=L, delta=delta, seed=seed, table=table)
    cap = max(len(r["col"]) for r in orows) + 16
    grows = mc.mcmi_walk_dump(B, p, rows, cap)
    mx, med, bounded = P.compare_dump(grows, orows, d)
    print(f"{name} fp{prec} table{table}: max rel {mx:.2e} median {med:.2e} bounded {bounded:.3f}")
    assert bounded <= 1.0


def test_sharded_rows_equal_one_launch():
    """Counter-keyed RNG: a row's walks do not depend on which launch, block
    or row subset it runs in."""
    m = _cases_small()["rand_long"]
    B = mc.DeviceCsr.from_host(m)
    p = mc.params(chains=200, max_len=100, delta=1e-3, seed=9, table=1)
    a = mc.mcmi_walk_dump(B, p, np.arange(m.n), 4000)
    b = mc.mcmi_walk_dump(B, p, np.arange(m.n)[::-1].copy(), 4000)[::-1]
    c = mc.mcmi_walk_dump(B, p, np.arange(7, 19), 4000)
    for x, y in zip(a, b):
        assert np.array_equal(x["col"], y["col"]) and np.array_equal(x["visits"], y["visits"])
        # the fixed-point accumulator sums exactly: bit-identical values
        assert np.array_equal(x["val"], y["val"])
    for k, r in enumerate(c):
        assert np.array_equal(r["col"], a[7 + k]["col"]) and np.array_equal(r["visits"], a[7 + k]["visits"])
        assert np.array_equal(r["val"], a[7 + k]["val"])
    # the FP32 Kahan accumulator sums in a timing-dependent order: equal up to
    # a few ulps of the row's largest partial sums (entries may cancel)
    pk = mc.params(chains=200, max_len=100, delta=1e-3, seed=9, table=1, accumulator=1)
    x1 = mc.mcmi_walk_dump(B, pk, np.arange(m.n), 4000)
    x2 = mc.mcmi_walk_dump(B, pk, np.arange(m.n), 4000)
    for x, y in zip(x1, x2):
        assert np.array_equal(x["visits"], y["visits"])
        assert np.allclose(x["val"], y["val"], rtol=1e-6, atol=1e-6 * np.abs(x["val"]).max())


def test_builds_are_bit_reproducible():
    m = synth.stencil3d_7pt(10, seed=4)
    B = mc.DeviceCsr.from_host(m)
    p = mc.params(chains=256, max_len=128, delta=1e-2, top_k=16, seed=3)
    r1 = [t.cpu().numpy() for t in mc.mcmi_build_ex(B, p).to_torch()]
    r2 = [t.cpu().numpy() for t in mc.mcmi_build_ex(B, p).to_torch()]
    for u, v in zip(r1, r2):
        assert np.array_equal(u, v)


# ------------------------------------------------------------------ build (filter + CSR)


def _gpu_rows(M):
    rp, col, val = (t.cpu().numpy() for t in M.to_torch())
    torch.cuda.synchronize()
    return rp, col, val


def _check_build(m, rows, N, L, delta, tau, top_k, prec=32, table=-1, seed=11, extra=None):
    orc = _orc()
    extra = extra or {}
    B = mc.DeviceCsr.from_host(m)
    p = mc.params(chains=N, max_len=L, delta=delta, seed=seed, precision=prec, table=table,
                  filter_tau=tau, top_k=top_k, **extra)
    M = mc.mcmi_build_ex(B, p)
    used_table = M.stats.table
    rp, col, val = _gpu_rows(M)
    rb = p.row_begin
    orows, d, s = orc.walk(m, rows=rows, chains=N, max_len=L, delta=delta, seed=seed, table=used_table)
    worst_rel = worst_b = 0.0
    for r in orows:
        i = r["row"]
        mvals = r["X"] / d[r["col"]]
        oc, ov = orc.filter_row(i, r["col"], mvals, tau=tau, top_k=top_k)
        gi = i - rb
        gc, gv = col[rp[gi]:rp[gi + 1]], val[rp[gi]:rp[gi + 1]]
        assert np.all(np.diff(gc) > 0), "row not sorted by column"
        rel, b = P.compare_rows(gc, gv.astype(np.float64), oc, ov, r["col"], mvals, r["A"] / np.abs(d[r["col"]]),
                                i, tau, top_k)
        worst_rel, worst_b = max(worst_rel, rel), max(worst_b, b)
    print(f"build n={m.n} fp{prec} table{used_table}: max rel {worst_rel:.2e} bounded {worst_b:.3f} "
          f"steps {M.stats.steps} spilled {M.stats.spilled}")
    assert worst_b <= 1.0
    return M, rp, col, val


def test_build_stencil2d_full_fp64_and_fp32():
    m = synth.stencil2d_5pt(32, 32, seed=1001)
    for prec in (64, 32):
        _check_build(m, np.arange(m.n), 1000, 64, 1e-3, 1e-2, 0, prec=prec)


def test_build_topk_and_tau_combinations():
    m = synth.random_dd(400, 9, seed=4, diag_sign="mixed", dominance=0.85)
    rows = np.arange(m.n)
    for tau, k in [(0.0, 0), (0.0, 3), (5e-2, 0), (1e-2, 4), (0.3, 16)]:
        _check_build(m, rows, 150, 60, 1e-3, tau, k, table=1)


def test_build_staging_regrowth_reruns_rows():
    # tau = 0 keeps every visited column: far more than the first staging buffer
    m = synth.powerlaw_random(2048, seed=8)
    M, rp, col, val = _check_build(m, np.arange(0, m.n, 37), 64, 40, 1e-3, 0.0, 0)
    assert M.stats.deferred_rows > 0
    # re-run rows are counted once
    orows, _, _ = _orc().walk(m, chains=64, max_len=40, delta=1e-3, seed=11, table=M.stats.table)
    assert M.stats.steps == sum(r["steps"] for r in orows)


def test_build_rows_of_every_length_class():
    """The CSR assembly orders a row by column in ways that depend on its
    length (up to a warp by shuffle ranks, up to 1024 entries by a warp in
    shared memory, padded to 64 ... 1024, one 4096-entry tile, several
    tiles): rows of each class against the oracle, and every row of the
    build strictly increasing in column."""
    m = synth.powerlaw_random(4096, seed=9)
    B = mc.DeviceCsr.from_host(m)
    p = mc.params(chains=256, max_len=64, delta=1e-4, seed=11, filter_tau=3e-3)
    rp, col, _ = (t.cpu().numpy() for t in mc.mcmi_build_ex(B, p).to_torch())
    ln = np.diff(rp)
    inner = np.ones(col.size, dtype=bool)
    inner[rp[:-1][ln > 0]] = False          # first entry of each row
    assert np.all(np.diff(col.astype(np.int64))[inner[1:]] > 0)
    picks = []
    for lo, hi in ((0, 32), (33, 64), (65, 128), (129, 256), (257, 512), (513, 1024), (1025, 1 << 30)):
        idx = np.flatnonzero((ln >= lo) & (ln <= hi))
        assert idx.size > 0, (lo, hi, ln.min(), ln.max())
        picks += [idx[0], idx[-1], idx[idx.size // 2]]
    picks.append(int(np.argmax(ln)))
    _check_build(m, np.unique(picks), 256, 64, 1e-4, 3e-3, 0)
    # rows beyond one 4096-entry shared-memory tile: merged in global memory
    m = synth.powerlaw_random(1 << 15, seed=9)
    p = mc.params(chains=512, max_len=64, delta=1e-4, seed=11, filter_tau=1e-4)
    ln = np.diff(mc.mcmi_build_ex(mc.DeviceCsr.from_host(m), p).to_torch()[0].cpu().numpy())
    assert ln.max() > 8192
    big = np.flatnonzero(ln > 4096)
    picks = [big[0], big[-1], int(np.argmax(ln)), int(np.argmin(ln))]
    _check_build(m, np.unique(picks), 512, 64, 1e-4, 1e-4, 0)


def test_build_rows_with_crowded_columns():
    """Rows of several hundred entries whose columns crowd into narrow
    ranges far apart (a chain with long walks plus a link 20000 columns
    away), sorted by the assembly's bitonic network.  Rows against the
    oracle."""
    n, far = 40000, 20000
    rng = np.random.default_rng(12)
    r, c, v = [], [], []
    for i in range(n):
        nb = [j for j in (i - 1, i + 1, i + far, i - far) if 0 <= j < n]
        w = rng.uniform(0.5, 1.0, len(nb))
        r += [i] * (len(nb) + 1)
        c += nb + [i]
        v += list(-w) + [w.sum() / 0.99]
    m = synth._from_coo(n, r, c, v)
    # FP64 walks: chains of ~1600 transitions would take an FP32 weight
    # product past the 1e-5 parity bound (about 2t 2^-24 relative)
    M, rp, _, _ = _check_build(m, np.array([0, 10000, 19999, 20000, 39999]), 256, 2000, 1e-7, 0.0, 0, prec=64)
    assert np.diff(rp).max() > 300


def test_build_through_the_overflow_log():
    """Rows that reach far more columns than a 64-slot on-chip table: visits
    go to the log and are reduced in several hash-range passes."""
    m = _cases_small()["powerlaw_4k"]
    rows = np.arange(0, m.n, 41)
    # 2^6 slots (< 128 threads): hash-range passes only; 2^8 and 2^11 slots:
    # per-warp bucket reduction, passes for the rare buckets above 32 entries
    for prec, log2h in [(32, 6), (64, 6), (32, 8), (64, 8), (32, 11)]:
        for tau, k in [(5e-3, 0), (0.0, 8)]:
            M, *_ = _check_build(m, rows, 128, 256, 1e-3, tau, k, prec=prec, extra={"hash_log2": log2h},
                                 seed=17)
            # with 2^11 slots the FP32 top-k build's sketch may prove every log column below the bound
            if log2h <= 8 or prec == 64 or k == 0:
                assert M.stats.spilled > 0


def test_load_depth_leaves_the_result_unchanged():
    """The load depth batches the loads after the walks, and the FP32 depth-8
    variant drops log columns that a magnitude sketch proves below the tau or
    top-k bound: builds at depth 4 and 8 are bit-identical (log-heavy rows,
    both precisions, 1 and 2 chains per thread, tau, top-k and both); auto
    picks 8 only for FP32 on long-row matrices."""
    m = _cases_small()["powerlaw_4k"]
    B = mc.DeviceCsr.from_host(m)
    for prec in (32, 64):
        for cpt in (1, 2):
            for tau, k in ((5e-3, 0), (0.0, 8), (1e-3, 24)):
                out = {}
                for depth in (4, 8):
                    p = mc.params(chains=128, max_len=256, delta=1e-3, filter_tau=tau, top_k=k, seed=17,
                                  precision=prec, hash_log2=8, chains_per_thread=cpt, load_depth=depth)
                    M = mc.mcmi_build_ex(B, p)
                    assert M.stats.load_depth == depth and (depth == 8 or M.stats.spilled > 0)
                    out[depth] = [t.cpu().numpy() for t in M.to_torch()]
                for u, v in zip(out[4], out[8]):
                    assert np.array_equal(u, v)
    # compact table through the log (1/d_j looked up by column), sketch at depth 8
    S12 = mc.DeviceCsr.from_host(_cases_small()["stencil3d_12"])
    out = {}
    for depth in (4, 8):
        p = mc.params(chains=256, max_len=128, delta=1e-2, filter_tau=1e-2, seed=5, table=mc.TABLE_COMPACT,
                      hash_log2=6, load_depth=depth)
        out[depth] = [t.cpu().numpy() for t in mc.mcmi_build_ex(S12, p).to_torch()]
    for u, v in zip(out[4], out[8]):
        assert np.array_equal(u, v)
    assert mc.mcmi_build_ex(B, mc.params(chains=8, max_len=8)).stats.load_depth == 8
    assert mc.mcmi_build_ex(B, mc.params(chains=8, max_len=8, precision=64)).stats.load_depth == 4
    S = mc.DeviceCsr.from_host(synth.stencil3d_7pt(8, seed=1))
    assert mc.mcmi_build_ex(S, mc.params(chains=8, max_len=8)).stats.load_depth == 4
    with pytest.raises(mc.McmiError):
        mc.mcmi_build_ex(S, mc.params(chains=8, max_len=8, load_depth=6))


def test_build_row_range():
    m = synth.stencil3d_7pt(10, seed=3)
    a = _check_build(m, np.arange(200, 420), 256, 128, 1e-2, 0.0, 16, extra=dict(row_begin=200, row_end=420))
    assert a[0].shape()[0] == 220


def test_apply_matches_oracle_spmv():
    orc = _orc()
    m = synth.stencil3d_7pt(16, seed=5)
    B = mc.DeviceCsr.from_host(m)
    M = mc.mcmi_build_ex(B, mc.params(chains=256, max_len=128, delta=1e-2, top_k=16))
    rp, col, val = _gpu_rows(M)
    x = torch.randn(m.n, device="cuda", dtype=torch.float32)
    y = torch.empty(m.n, device="cuda", dtype=torch.float32)
    mc.mcmi_apply(M, x, y)
    ref = orc.spmv(rp, col, val.astype(np.float64), x.cpu().numpy().astype(np.float64))
    assert np.allclose(y.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)


# ------------------------------------------------------------------ edge cases


def _csr(n, rows, cols, vals):
    return synth._from_coo(n, np.array(rows), np.array(cols), np.array(vals, dtype=np.float64))


def test_edge_diagonal_only_and_single_row():
    for m in (_csr(1, [0], [0], [2.0]), _csr(5, range(5), range(5), [1.0, -2.0, 3.0, 4.0, -0.5])):
        B = mc.DeviceCsr.from_host(m)
        M = mc.mcmi_build_ex(B, mc.params(chains=33, max_len=10, delta=1e-3, top_k=2))
        rp, col, val = _gpu_rows(M)
        d = m.to_scipy().diagonal()
        assert np.array_equal(col, np.arange(m.n)) and np.allclose(val, (1.0 / d).astype(np.float32), rtol=1e-7)
        assert M.stats.steps == 0


def test_edge_zero_length_and_huge_cutoff():
    m = synth.random_dd(50, 4, seed=2)
    B = mc.DeviceCsr.from_host(m)
    d = m.to_scipy().diagonal()
    for kw in (dict(max_len=0, delta=1e-3), dict(max_len=50, delta=2.0)):
        M = mc.mcmi_build_ex(B, mc.params(chains=64, **kw))
        rp, col, val = _gpu_rows(M)
        assert M.stats.steps == 0 and np.array_equal(col, np.arange(m.n))
        assert np.allclose(val, 1.0 / d, rtol=1e-6)


def test_edge_empty_matrix_and_empty_range():
    m = _csr(0, [], [], [])
    B = mc.DeviceCsr(0, torch.zeros(1, dtype=torch.int64, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"),
                     torch.zeros(0, dtype=torch.float64, device="cuda"))
    M = mc.mcmi_build_ex(B, mc.params())
    assert M.shape() == (0, 0, 0)
    m = synth.random_dd(20, 3, seed=1)
    M = mc.mcmi_build_ex(mc.DeviceCsr.from_host(m), mc.params(row_begin=5, row_end=5))
    assert M.shape() == (0, 5, 0)


@pytest.mark.parametrize("defect,status", [("zero_diag", 3), ("unsorted", 2), ("nan", 2), ("col_range", 2),
                                           ("not_dd", 4), ("row_ptr", 2)])
def test_edge_invalid_inputs_report_status(defect, status):
    m = synth.random_dd(30, 4, seed=3)
    rp, col, val = m.row_ptr.copy(), m.col.copy(), m.val.copy()
    dpos = [int(rp[i] + np.flatnonzero(col[rp[i]:rp[i + 1]] == i)[0]) for i in range(m.n)]
    if defect == "zero_diag":
        val[dpos[7]] = 0.0
    elif defect == "unsorted":
        a = int(rp[4])
        col[a], col[a + 1] = col[a + 1], col[a]
    elif defect == "nan":
        val[int(rp[9]) + 1] = np.nan
    elif defect == "col_range":
        col[int(rp[3]) + 1] = m.n + 5
    elif defect == "not_dd":
        val[dpos[11]] *= 0.5
    elif defect == "row_ptr":
        rp[6] = rp[7] + 1
    bad = synth.Csr(m.n, rp, col, val)
    B = mc.DeviceCsr.from_host(bad)
    with pytest.raises(mc.McmiError) as e:
        mc.mcmi_build_ex(B, mc.params(chains=16, max_len=20))
    assert e.value.status == status, str(e.value)


def test_edge_bad_parameters():
    m = synth.random_dd(10, 3, seed=1)
    B = mc.DeviceCsr.from_host(m)
    for kw in (dict(precision=16), dict(chains=-1), dict(delta=-1.0), dict(table=5), dict(row_begin=3, row_end=2),
               dict(threads=96), dict(chains=0, eps=0.0)):
        with pytest.raises(mc.McmiError) as e:
            mc.mcmi_build_ex(B, mc.params(**kw))
        assert e.value.status == 1, kw


def test_mcmi_build_signature_and_eps_rule():
    m = synth.random_dd(64, 4, seed=6, dominance=0.5)
    B = mc.DeviceCsr.from_host(m)
    M = mc.mcmi_build(B, 0.05, 1e-3, 64, 1e-2, 5)
    assert M.shape()[0] == m.n
    M2 = mc.mcmi_build_ex(B, mc.params(chains=0, eps=0.05, delta=1e-3))
    assert M2.stats.chains == _orc().chains_from_eps(0.05, float(M2.stats.max_s))
