"""CPU oracle of the (MC)^2MI hot path: plain FP64 C, loaded with ctypes.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA product
path never imports it, and it imports nothing from the product package.

Each function cites the passage of the paper it follows; the arithmetic lives
in ``mcmi_oracle.c`` (see its header for the readings of the points the paper
leaves open).  ``chains_from_eps`` is *parity unpinned* (the paper does not
state the rule).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcmi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TABLE_CUMULATIVE = 0
TABLE_ALIAS = 1
TABLE_HYBRID = 2   # per row: cumulative for at most 6 transitions, alias for longer rows
TABLE_COMPACT = 3  # cumulative sampling from weights at the scale 2^20 instead of 2^31


def compile_lib(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        compile_lib()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        i64, u64, f64, i32 = C.c_int64, C.c_uint64, C.c_double, C.c_int
        lib.orc_philox4x32_10.argtypes = [P, P, P]
        lib.orc_split.argtypes = [i64, P, P, P, f64, P, P, P]
        lib.orc_split.restype = i32
        lib.orc_alias_build.argtypes = [P, i64, u64, P, P]
        lib.orc_pick_cumulative_many.argtypes = [P, i64, P, i64, P]
        lib.orc_pick_alias_many.argtypes = [P, P, i64, u64, P, i64, P]
        lib.orc_tables.argtypes = [i64, P, P, P, P, P, P, P, P, P, P]
        lib.orc_tables.restype = i32
        lib.orc_tables_ex.argtypes = [i64, P, P, P, P, P, i32, P, P, P, P, P]
        lib.orc_tables_ex.restype = i32
        lib.orc_max_walk_len.argtypes = [f64, f64, i64]
        lib.orc_max_walk_len.restype = i64
        lib.orc_chains_from_eps.argtypes = [f64, f64]
        lib.orc_chains_from_eps.restype = i64
        lib.orc_walk_rows.argtypes = [i64, P, P, P, P, P, i32, P, i64, i64, i64, f64, u64, i64, i32,
                                      P, P, P, P, P, P, P]
        lib.orc_walk_rows.restype = i32
        lib.orc_build_rows.argtypes = [i64, P, P, P, P, P, i32, P, i64, i64, i64, f64, u64, f64, i64,
                                       i64, i32, P, P, P, P, P]
        lib.orc_build_rows.restype = i32
        lib.orc_learned_tables.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_learned_tables.restype = i32
        lib.orc_mlp_g.argtypes = [P, P]
        lib.orc_mlp_g.restype = C.c_float
        lib.orc_row_moments.argtypes = [i64, P, P, P, P, P, i32, P, i64, i64, i64, f64, u64, i32, P, P]
        lib.orc_row_moments.restype = i32
        lib.orc_train_edges.argtypes = [i64, P, P, P, P, P, P, P, P, P]
        lib.orc_train_edges.restype = i32
        lib.orc_filter_row.argtypes = [i64, P, P, i64, f64, i64, P, P]
        lib.orc_filter_row.restype = i64
        lib.orc_spmv.argtypes = [i64, P, P, P, P, P]
        lib.orc_reduce_mask.argtypes = [i64, P, P, P, f64, i32, P]
        lib.orc_reduce_mask.restype = i64
        lib.orc_recover_dense.argtypes = [i64, P, P]
        lib.orc_recover_dense.restype = i32
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _csr(m):
    rp = np.ascontiguousarray(m.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(m.col, dtype=np.int32)
    val = np.ascontiguousarray(m.val, dtype=np.float64)
    return rp, col, val


class OracleError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"oracle status {status} {msg}")
        self.status = status


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _L().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def split(m, alpha: float = 0.0):
    """Eq. 1 split (with the Sec. V-C augmentation when alpha > 0) and the
    Jacobi scaling: returns (d, s), d_i = bhat_ii, s_i = ||c_i||_1."""
    rp, col, val = _csr(m)
    d = np.zeros(m.n)
    s = np.zeros(m.n)
    bad = np.zeros(1, dtype=np.int64)
    st = _L().orc_split(m.n, _p(rp), _p(col), _p(val), alpha, _p(d), _p(s), _p(bad))
    if st:
        raise OracleError(st, f"row {int(bad[0])}")
    return d, s


def tables(m, d, s, alias: bool = False, table: int = TABLE_CUMULATIVE):
    """Integer sampling tables of every row (p of Eq. 2 as integers).
    Returns dict(off, Q, q[, prob, alias]) over off-diagonals in CSR order;
    table=TABLE_COMPACT gives the weights at the scale 2^20."""
    rp, col, val = _csr(m)
    noff = int(rp[-1]) - int(np.sum(col == np.repeat(np.arange(m.n), np.diff(rp))))
    off = np.zeros(m.n + 1, dtype=np.int64)
    Q = np.zeros(m.n, dtype=np.uint64)
    q = np.zeros(max(noff, 1), dtype=np.uint32)
    prob = np.zeros(max(noff, 1), dtype=np.uint32) if alias else None
    al = np.zeros(max(noff, 1), dtype=np.int32) if alias else None
    _L().orc_tables_ex(m.n, _p(rp), _p(col), _p(val), _p(np.ascontiguousarray(d)),
                       _p(np.ascontiguousarray(s)), int(table), _p(off), _p(Q), _p(q),
                       _p(prob) if alias else None, _p(al) if alias else None)
    out = dict(off=off, Q=Q, q=q[:noff])
    if alias:
        out["prob"] = prob[:noff]
        out["alias"] = al[:noff]
    return out


def alias_build(q, Q=None):
    q = np.ascontiguousarray(q, dtype=np.uint32)
    Q = int(q.astype(np.uint64).sum()) if Q is None else int(Q)
    prob = np.zeros(len(q), dtype=np.uint32)
    al = np.zeros(len(q), dtype=np.int32)
    _L().orc_alias_build(_p(q), len(q), Q, _p(prob), _p(al))
    return prob, al


def pick_cumulative(q, r):
    q = np.ascontiguousarray(q, dtype=np.uint32)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    out = np.zeros(len(r), dtype=np.int64)
    _L().orc_pick_cumulative_many(_p(q), len(q), _p(r), len(r), _p(out))
    return out


def pick_alias(prob, al, Q, r):
    prob = np.ascontiguousarray(prob, dtype=np.uint32)
    al = np.ascontiguousarray(al, dtype=np.int32)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    out = np.zeros(len(r), dtype=np.int64)
    _L().orc_pick_alias_many(_p(prob), _p(al), len(prob), int(Q), _p(r), len(r), _p(out))
    return out


def max_walk_len(smax, delta, max_len):
    return int(_L().orc_max_walk_len(float(smax), float(delta), int(max_len)))


def chains_from_eps(eps, smax):
    """N from epsilon: the rule of the earlier (MC)^2MI papers (not stated in
    this one), N = ceil((0.6745 / (eps (1 - smax)))^2): probable error <= eps."""
    return int(_L().orc_chains_from_eps(float(eps), float(smax)))


def _rows(m, rows):
    if rows is None:
        rows = np.arange(m.n, dtype=np.int64)
    return np.ascontiguousarray(rows, dtype=np.int64)


def _theta(theta):
    return None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)


def _tp(theta):
    return _p(theta) if theta is not None else None


def walk(m, rows=None, chains=100, max_len=64, delta=1e-3, seed=1, table=TABLE_CUMULATIVE,
         alpha=0.0, threads=0, theta=None):
    """Eq. 2 estimator, unfiltered: for each listed row a dict with the visited
    columns (sorted), X = (1/N) sum W, A = (1/N) sum |W|, V = visit counts,
    and the number of transitions taken.  theta: learned-proposal parameters
    (see learned_tables), None for p = |c|/s."""
    rp, col, val = _csr(m)
    d, s = split(m, alpha)
    rows = _rows(m, rows)
    theta = _theta(theta)
    tb = max_walk_len(s.max() if m.n else 0.0, delta, max_len) if theta is None else max_len
    cap = int(min(m.n, chains * (tb + 1)))
    nr = len(rows)
    count = np.zeros(nr, dtype=np.int64)
    steps = np.zeros(nr, dtype=np.uint64)
    oc = np.zeros(nr * cap, dtype=np.int32)
    oX = np.zeros(nr * cap)
    oA = np.zeros(nr * cap)
    oV = np.zeros(nr * cap, dtype=np.uint32)
    st = _L().orc_walk_rows(m.n, _p(rp), _p(col), _p(val), _p(d), _p(s), table, _p(rows), nr,
                            chains, max_len, delta, seed, cap, threads, _p(count), _p(steps),
                            _p(oc), _p(oX), _p(oA), _p(oV), _tp(theta))
    if st:
        raise OracleError(st)
    out = []
    for p in range(nr):
        a, b = p * cap, p * cap + int(count[p])
        out.append(dict(row=int(rows[p]), col=oc[a:b].copy(), X=oX[a:b].copy(), A=oA[a:b].copy(),
                        V=oV[a:b].copy(), steps=int(steps[p])))
    return out, d, s


def filter_row(i, cols, mvals, tau=0.0, top_k=0):
    """Sec. IV-B filter of one column-scaled row (cols sorted)."""
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    mvals = np.ascontiguousarray(mvals, dtype=np.float64)
    oc = np.zeros(max(len(cols), 1), dtype=np.int32)
    ov = np.zeros(max(len(cols), 1))
    k = _L().orc_filter_row(int(i), _p(cols), _p(mvals), len(cols), float(tau), int(top_k), _p(oc), _p(ov))
    return oc[:k].copy(), ov[:k].copy()


def build(m, rows=None, chains=100, max_len=64, delta=1e-3, seed=1, tau=0.0, top_k=0,
          table=TABLE_CUMULATIVE, alpha=0.0, threads=0, theta=None):
    """Preconditioner rows: Eq. 2 walks, column scaling by 1/d_j (phase 4),
    Sec. IV-B filter.  Returns (row_ptr, col, val, steps_per_row) for the
    listed rows (in the given order)."""
    rp, col, val = _csr(m)
    d, s = split(m, alpha)
    rows = _rows(m, rows)
    theta = _theta(theta)
    tb = max_walk_len(s.max() if m.n else 0.0, delta, max_len) if theta is None else max_len
    cap = int(min(m.n, chains * (tb + 1)))
    if top_k > 0:
        cap = min(cap, top_k + 1)
    nr = len(rows)
    count = np.zeros(nr, dtype=np.int64)
    steps = np.zeros(nr, dtype=np.uint64)
    oc = np.zeros(nr * cap, dtype=np.int32)
    ov = np.zeros(nr * cap)
    st = _L().orc_build_rows(m.n, _p(rp), _p(col), _p(val), _p(d), _p(s), table, _p(rows), nr,
                             chains, max_len, delta, seed, tau, top_k, cap, threads,
                             _p(count), _p(steps), _p(oc), _p(ov), _tp(theta))
    if st:
        raise OracleError(st)
    orp = np.zeros(nr + 1, dtype=np.int64)
    np.cumsum(count, out=orp[1:])
    keep = np.concatenate([np.arange(p * cap, p * cap + count[p]) for p in range(nr)]) if nr else np.zeros(0, int)
    return orp, oc[keep], ov[keep], steps


def spmv(rp, col, val, x):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(len(rp) - 1)
    _L().orc_spmv(len(rp) - 1, _p(rp), _p(col), _p(val), _p(x), _p(y))
    return y


# ---------------------------------------------------------------- learned proposal
# (an extension of the method: |c_ij| reweighted by an MLP g_ij > 0, weight
#  update c_ij / p_ij with the table's own probability, so Eq. 2 stays unbiased)

MLP_NPARAM = 32 * 8 + 32 + 32 * 32 + 32 + 32 + 1


def learned_tables(m, theta, alpha=0.0):
    """Integer weights q, factors f = c Q / q and MLP outputs g of every
    off-diagonal entry (CSR order) under the learned proposal theta."""
    rp, col, val = _csr(m)
    d, s = split(m, alpha)
    theta = _theta(theta)
    noff = int(rp[-1]) - int(np.sum(col == np.repeat(np.arange(m.n), np.diff(rp))))
    off = np.zeros(m.n + 1, dtype=np.int64)
    Q = np.zeros(m.n, dtype=np.uint64)
    q = np.zeros(max(noff, 1), dtype=np.uint32)
    fac = np.zeros(max(noff, 1))
    g = np.zeros(max(noff, 1), dtype=np.float32)
    _L().orc_learned_tables(m.n, _p(rp), _p(col), _p(val), _p(d), _p(s), _p(theta), _p(off), _p(Q), _p(q),
                            _p(fac), _p(g))
    return dict(off=off, Q=Q, q=q[:noff], fac=fac[:noff], g=g[:noff], d=d, s=s)


def mlp_g(theta, feat):
    """The BF16 MLP of the learned proposal on one FP32 feature vector."""
    theta = _theta(theta)
    f = np.ascontiguousarray(feat, dtype=np.float32)
    return float(_L().orc_mlp_g(_p(theta), _p(f)))


def row_moments(m, rows=None, chains=64, max_len=64, delta=1e-3, seed=1, table=TABLE_CUMULATIVE, alpha=0.0,
                theta=None, threads=0):
    """m_i = (1/N) sum over the N chains of row i of sum_t W_t^2."""
    rp, col, val = _csr(m)
    d, s = split(m, alpha)
    rows = _rows(m, rows)
    theta = _theta(theta)
    out = np.zeros(len(rows))
    _L().orc_row_moments(m.n, _p(rp), _p(col), _p(val), _p(d), _p(s), table, _p(rows), len(rows), chains,
                         max_len, delta, seed, threads, _p(out), _tp(theta))
    return out


def proposal_loss(theta, feat, row_of_edge, p_edge, m_edge):
    """FP64 training loss of the learned proposal (no BF16 rounding):
    mean over rows of (sum_j p g)(sum_j p m / g) / (sum_j p sqrt(m))^2, which
    is >= 1 with equality iff g is proportional to sqrt(m) within each row
    (Cauchy-Schwarz); p = |c|/s per edge, m = second moment of the target row."""
    th = np.asarray(theta, dtype=np.float64)
    W1, b1 = th[:256].reshape(32, 8), th[256:288]
    W2, b2 = th[288:1312].reshape(32, 32), th[1312:1344]
    w3, b3 = th[1344:1376], th[1376]
    x = np.asarray(feat, dtype=np.float64)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    z = h2 @ w3 + b3
    g = np.clip(0.5 * (z + np.sqrt(z * z + 4.0)), 0.0625, 16.0)
    r = np.asarray(row_of_edge, dtype=np.int64)
    nr = int(r.max()) + 1 if r.size else 0
    A = np.bincount(r, p_edge * g, nr)
    Bv = np.bincount(r, p_edge * m_edge / g, nr)
    Cv = np.bincount(r, p_edge * np.sqrt(m_edge), nr) ** 2
    ok = Cv > 0
    return float(np.mean(A[ok] * Bv[ok] / Cv[ok]))


def train_edges(m, alpha=0.0):
    """Training edges in CSR order: features (FP32), p = |c|/s (FP64), target
    column and row (diagonal slots: p = 0)."""
    rp, col, val = _csr(m)
    d, s = split(m, alpha)
    E = int(rp[-1])
    feat = np.zeros((max(E, 1), 8), dtype=np.float32)
    p = np.zeros(max(E, 1))
    tgt = np.zeros(max(E, 1), dtype=np.int64)
    row = np.zeros(max(E, 1), dtype=np.int64)
    _L().orc_train_edges(m.n, _p(rp), _p(col), _p(val), _p(d), _p(s), _p(feat), _p(p), _p(tgt), _p(row))
    return feat[:E], p[:E], tgt[:E], row[:E]


REDUCE_ENTRIES, REDUCE_RANGE = 0, 1


def reduce(m, fraction, mode=REDUCE_ENTRIES):
    """Matrix reduction (Algorithm 1 step 2; Sec. III "Matrix Reduction"):
    drop a share of the smallest off-diagonal entries before the split.
    mode 0: floor(fraction * nnz_off) smallest |b_ij|, ties by CSR position;
    mode 1: |b_ij| < lo + fraction (hi - lo) over the off-diagonal range.
    Returns (reduced Csr, keep mask over the stored entries, dropped count)."""
    from synth import Csr
    rp, col, val = _csr(m)
    keep = np.ones(max(len(col), 1), dtype=np.uint8)
    d = _L().orc_reduce_mask(m.n, _p(rp), _p(col), _p(val), float(fraction), int(mode), _p(keep))
    if d < 0:
        raise ValueError("bad reduction arguments")
    keep = keep[:len(col)].astype(bool)
    counts = np.array([keep[rp[i]:rp[i + 1]].sum() for i in range(m.n)], dtype=np.int64)
    nrp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return Csr(m.n, nrp, col[keep].astype(np.int32), val[keep].astype(np.float64)), keep, int(d)


def augmentation(m, alpha):
    """Diagonal of S = Bhat - B for the Eq. 1 augmentation: alpha ||B||_inf sgn(b_ii)."""
    d0, _ = split(m, 0.0)
    d1, _ = split(m, alpha)
    return d1 - d0


def recover_dense(X, s):
    """Eq. 3 (Algorithm 1 step 5): B^-1 from a dense Bhat^-1 (or an
    approximation) by n Sherman-Morrison rank-one updates, k = n-1 .. 0."""
    X = np.ascontiguousarray(np.array(X, dtype=np.float64))
    s = np.ascontiguousarray(s, dtype=np.float64)
    if _L().orc_recover_dense(X.shape[0], _p(s), _p(X)) != 0:
        raise ValueError("zero denominator in the recovery")
    return X

