"""Seeded synthetic sparse matrices for the (MC)^2MI hot path.

This module only draws matrices; it contains none of the method's arithmetic
(no splitting, no tables, no walks).  Both the CPU oracle's tests and the CUDA
path's tests and benchmark take their inputs from here.

Every generator returns a ``Csr`` with int64 ``row_ptr``, int32 ``col``
(sorted, unique, diagonal present) and float64 ``val``.  The paper's own
matrices (Table I: a cubic-FE stiffness matrix, two climate-model matrices and
rdb2048) are not available; the families below stand in for them at the same
scales (2e4 to 1e6 rows, 6 to ~256 entries per row), as the paper's Sec. VI
workloads are sparse, diagonally dominant after the split of Eq. 1, and come
from PDE discretisations or random sparsity.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Csr", "stencil2d_5pt", "stencil3d_7pt", "powerlaw_random", "random_dd",
    "aniso2d_9pt", "batch_mix", "workload",
]


@dataclasses.dataclass
class Csr:
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[nnz]
    val: np.ndarray      # float64[nnz]
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def row_slice(self, i: int):
        a, b = int(self.row_ptr[i]), int(self.row_ptr[i + 1])
        return self.col[a:b], self.val[a:b]


def _from_coo(n, rows, cols, vals):
    """Assemble a CSR with columns sorted inside each row (no duplicates allowed)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], np.asarray(vals, dtype=np.float64)[order]
    key = rows * n + cols
    if key.size > 1 and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate entries")
    counts = np.bincount(rows, minlength=n)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return Csr(n, rp, cols.astype(np.int32), vals)


def _grid_neighbours(shape):
    """Directed neighbour pairs (i, j) of a regular grid, row-major numbering."""
    idx = np.arange(int(np.prod(shape))).reshape(shape)
    pairs = []
    for ax in range(len(shape)):
        lo = [slice(None)] * len(shape)
        hi = [slice(None)] * len(shape)
        lo[ax] = slice(0, shape[ax] - 1)
        hi[ax] = slice(1, shape[ax])
        a = idx[tuple(lo)].ravel()
        b = idx[tuple(hi)].ravel()
        pairs.append((a, b))
        pairs.append((b, a))
    i = np.concatenate([p[0] for p in pairs])
    j = np.concatenate([p[1] for p in pairs])
    return i, j


def stencil2d_5pt(nx=32, ny=32, seed=1001, dominance=0.95):
    """2D 5-point diffusion-like matrix with random coefficients.

    Diagonal 4 + U(0, 0.5); every off-diagonal entry independently -U(0.8, 1.0)
    (so the matrix is nonsymmetric).  The drawn diagonal alone does not
    guarantee ||C||_inf <= dominance (a row of four entries near 1.0 gives
    s_i near 1), so each diagonal is raised to at least (row abs-sum)/dominance;
    the number of raised rows is recorded in ``meta['clamped_rows']``.
    Draw order: diagonal for all rows, then off-diagonals in CSR order.
    """
    rng = np.random.default_rng(seed)
    n = nx * ny
    i, j = _grid_neighbours((ny, nx))
    diag = 4.0 + rng.uniform(0.0, 0.5, n)
    m = _from_coo(n, i, j, np.ones(i.size))
    m.val[:] = -rng.uniform(0.8, 1.0, m.nnz)
    absum = np.add.reduceat(np.abs(m.val), m.row_ptr[:-1]) if m.nnz else np.zeros(n)
    absum[np.diff(m.row_ptr) == 0] = 0.0
    need = absum / dominance
    clamped = int(np.sum(diag < need))
    diag = np.maximum(diag, need)
    out = _add_diagonal(m, diag)
    out.meta = dict(family="stencil2d_5pt", nx=nx, ny=ny, seed=seed, clamped_rows=clamped)
    return out


def _add_diagonal(m: Csr, diag):
    rows = np.repeat(np.arange(m.n, dtype=np.int64), np.diff(m.row_ptr))
    r = np.concatenate([rows, np.arange(m.n, dtype=np.int64)])
    c = np.concatenate([m.col.astype(np.int64), np.arange(m.n, dtype=np.int64)])
    v = np.concatenate([m.val, np.asarray(diag, dtype=np.float64)])
    return _from_coo(m.n, r, c, v)


def stencil3d_7pt(nx=64, seed=1002, dominance=0.9):
    """3D 7-point variable-coefficient diffusion on an nx^3 grid.

    One lognormal(0, 1) coefficient per cell face (Dirichlet boundary faces
    included); b_ij = -k(face ij), symmetric; diagonal = (sum of the six face
    coefficients of the cell) / dominance, so interior rows have
    ||c_i||_1 = dominance and boundary rows less.
    Draw order: x-faces, then y-faces, then z-faces, each as an
    (nx+1, nx, nx)-shaped array in C order (face index first along its axis).
    """
    rng = np.random.default_rng(seed)
    n = nx ** 3
    kx = rng.lognormal(0.0, 1.0, (nx + 1, nx, nx))  # faces normal to axis 2 (fastest index)
    ky = rng.lognormal(0.0, 1.0, (nx + 1, nx, nx))  # axis 1
    kz = rng.lognormal(0.0, 1.0, (nx + 1, nx, nx))  # axis 0 (slowest)
    idx = np.arange(n).reshape(nx, nx, nx)  # [z, y, x]
    rows, cols, vals = [], [], []
    diag = np.zeros((nx, nx, nx))
    # axis x: face f between x=f-1 and x=f; kx[f, z, y]
    fx = np.transpose(kx, (1, 2, 0))  # [z, y, f]
    diag += fx[:, :, :-1] + fx[:, :, 1:]
    a, b, k = idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel(), fx[:, :, 1:-1].ravel()
    rows += [a, b]; cols += [b, a]; vals += [-k, -k]
    fy = np.transpose(ky, (1, 0, 2))  # [z, f, x]
    diag += fy[:, :-1, :] + fy[:, 1:, :]
    a, b, k = idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel(), fy[:, 1:-1, :].ravel()
    rows += [a, b]; cols += [b, a]; vals += [-k, -k]
    fz = kz  # [f, y, x]
    diag += fz[:-1, :, :] + fz[1:, :, :]
    a, b, k = idx[:-1, :, :].ravel(), idx[1:, :, :].ravel(), fz[1:-1, :, :].ravel()
    rows += [a, b]; cols += [b, a]; vals += [-k, -k]
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(diag.ravel() / dominance)
    m = _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    m.meta = dict(family="stencil3d_7pt", nx=nx, seed=seed, dominance=dominance)
    return m


def _unique_cols(rng, n, row_of, deg_total):
    """Uniform columns without replacement per row, excluding the row itself."""
    cols = rng.integers(0, n - 1, deg_total, dtype=np.int64)
    cols += cols >= row_of
    for _ in range(64):
        key = row_of * n + cols
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(deg_total, dtype=bool)
        dup[order[1:][ks[1:] == ks[:-1]]] = True
        nd = int(dup.sum())
        if nd == 0:
            return cols
        c = rng.integers(0, n - 1, nd, dtype=np.int64)
        c += c >= row_of[dup]
        cols[dup] = c
    raise RuntimeError("could not draw unique columns")


def powerlaw_random(n=1 << 20, alpha=2.5, dmin=4, dmax=256, seed=1003, dominance=0.85):
    """Random sparse nonsymmetric matrix with power-law row lengths.

    Row length floor(k), k drawn from the continuous density proportional to
    k^-alpha on [dmin, dmax] (inverse CDF); columns uniform without
    replacement excluding the diagonal; values N(0, 1) in sorted-column order;
    diagonal = (row abs-sum) / dominance.  With alpha = 2.5 on [4, 256] the
    realised mean row length is about 10 (``meta['mean_deg']``).
    """
    rng = np.random.default_rng(seed)
    u = rng.random(n)
    e = 1.0 - alpha
    k = (dmin ** e - u * (dmin ** e - dmax ** e)) ** (1.0 / e)
    deg = np.clip(np.floor(k).astype(np.int64), dmin, min(dmax, n - 1))
    row_of = np.repeat(np.arange(n, dtype=np.int64), deg)
    cols = _unique_cols(rng, n, row_of, int(deg.sum()))
    order = np.lexsort((cols, row_of))
    cols = cols[order]
    vals = rng.standard_normal(cols.size)
    m = _from_coo(n, row_of, cols, vals)
    absum = np.add.reduceat(np.abs(m.val), m.row_ptr[:-1])
    out = _add_diagonal(m, absum / dominance)
    out.meta = dict(family="powerlaw_random", n=n, alpha=alpha, dmin=dmin, dmax=dmax,
                    seed=seed, dominance=dominance, mean_deg=float(deg.mean()))
    return out


def random_dd(n, deg, seed, dominance=0.8, signs="mixed", diag_sign="positive",
              zero_frac=0.0, dominance_jitter=0.0):
    """Small random diagonally dominant matrix for tests.

    ``deg`` off-diagonals per row (capped at n-1), columns uniform without
    replacement; values N(0,1) (``signs='mixed'``), |N(0,1)| (``'positive'``)
    or -|N(0,1)| (``'negative'``); a fraction ``zero_frac`` of them set to an
    explicit 0.0; diagonal = abs-sum / (dominance * (1 - U(0, jitter))) with
    sign + or random (``diag_sign='mixed'``).  Rows whose off-diagonals are
    all zero get diagonal 1.
    """
    rng = np.random.default_rng(seed)
    d = min(deg, n - 1)
    row_of = np.repeat(np.arange(n, dtype=np.int64), d)
    cols = _unique_cols(rng, n, row_of, n * d) if d > 0 else np.zeros(0, np.int64)
    order = np.lexsort((cols, row_of))
    cols = cols[order]
    v = rng.standard_normal(cols.size)
    if signs == "positive":
        v = np.abs(v)
    elif signs == "negative":
        v = -np.abs(v)
    if zero_frac > 0:
        v[rng.random(v.size) < zero_frac] = 0.0
    m = _from_coo(n, row_of, cols, v)
    absum = np.add.reduceat(np.abs(m.val), m.row_ptr[:-1]) if m.nnz else np.zeros(n)
    if m.nnz:
        absum[np.diff(m.row_ptr) == 0] = 0.0
    dom = dominance * (1.0 - rng.uniform(0.0, dominance_jitter, n))
    diag = np.where(absum > 0, absum / dom, 1.0)
    if diag_sign == "mixed":
        diag *= np.where(rng.random(n) < 0.5, -1.0, 1.0)
    out = _add_diagonal(m, diag)
    out.meta = dict(family="random_dd", n=n, deg=deg, seed=seed)
    return out


def equal_rows(n, deg, seed, diag=0.2):
    """General (not diagonally dominant) random matrix whose rows all have the
    same norms: ``deg`` off-diagonals of magnitude 1/deg with random signs
    (columns uniform without replacement) and a diagonal of magnitude
    ``diag`` with a random sign.  With the Eq. 1 augmentation every row then
    has the same s_i = 1 / (diag + alpha (1 + diag))."""
    rng = np.random.default_rng(seed)
    d = min(deg, n - 1)
    row_of = np.repeat(np.arange(n, dtype=np.int64), d)
    cols = _unique_cols(rng, n, row_of, n * d)
    order = np.lexsort((cols, row_of))
    cols = cols[order]
    v = np.where(rng.random(cols.size) < 0.5, -1.0, 1.0) / d
    m = _from_coo(n, row_of, cols, v)
    out = _add_diagonal(m, diag * np.where(rng.random(n) < 0.5, -1.0, 1.0))
    out.meta = dict(family="equal_rows", n=n, deg=deg, seed=seed)
    return out


def aniso2d_9pt(nx=1024, eps=1e-3, block=32, seed=1005):
    """2D anisotropic diffusion, 9-point finite differences of div(K grad u).

    K = R(theta) diag(1, eps) R(theta)^T with theta ~ U[0, pi) drawn per
    block x block tile (C order over tiles).  The stencil is the standard
    9-point discretisation with mixed derivative by central differences
    (coefficients from the cell's K, unit spacing):
      east/west  -kxx, north/south -kyy, corners -/+ kxy/2,
      centre 2(kxx + kyy).
    Off-diagonal entries are kept only inside the grid (Dirichlet boundary).
    The matrix need not be diagonally dominant; the split of Eq. 1 is chosen
    by the caller (alpha).
    """
    rng = np.random.default_rng(seed)
    nb = (nx + block - 1) // block
    theta = rng.uniform(0.0, math.pi, (nb, nb))
    yy, xx = np.meshgrid(np.arange(nx), np.arange(nx), indexing="ij")
    th = theta[yy // block, xx // block]
    c, s = np.cos(th), np.sin(th)
    kxx = c * c + eps * s * s
    kyy = s * s + eps * c * c
    kxy = (1.0 - eps) * c * s
    n = nx * nx
    idx = np.arange(n).reshape(nx, nx)
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [(2.0 * (kxx + kyy)).ravel()]
    offs = [((0, 1), -kxx), ((0, -1), -kxx), ((1, 0), -kyy), ((-1, 0), -kyy),
            ((1, 1), -0.5 * kxy), ((-1, -1), -0.5 * kxy), ((1, -1), 0.5 * kxy), ((-1, 1), 0.5 * kxy)]
    for (dy, dx), coef in offs:
        ys = slice(max(0, -dy), nx - max(0, dy))
        xs = slice(max(0, -dx), nx - max(0, dx))
        yt = slice(max(0, dy), nx - max(0, -dy))
        xt = slice(max(0, dx), nx - max(0, -dx))
        rows.append(idx[ys, xs].ravel())
        cols.append(idx[yt, xt].ravel())
        vals.append(coef[ys, xs].ravel())
    m = _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    m.meta = dict(family="aniso2d_9pt", nx=nx, eps=eps, block=block, seed=seed)
    return m


def batch_mix(count=512, nmin=1000, nmax=200_000, seed=1004):
    """Batch of uneven matrices: n log-uniform in [nmin, nmax], a mix of 2D
    5-point, 3D 7-point and power-law random rows, dominance U[0.8, 0.95].
    Returns a list of ``Csr`` (kind cycles 2D, 3D, power-law)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), count))
    doms = rng.uniform(0.8, 0.95, count)
    out = []
    for b in range(count):
        kind = b % 3
        sub = int(rng.integers(0, 2**31 - 1))
        if kind == 0:
            nx = max(2, int(round(math.sqrt(ns[b]))))
            m = stencil2d_5pt(nx, nx, seed=sub, dominance=doms[b])
        elif kind == 1:
            nx = max(2, int(round(ns[b] ** (1.0 / 3.0))))
            m = stencil3d_7pt(nx, seed=sub, dominance=doms[b])
        else:
            m = powerlaw_random(int(ns[b]), seed=sub, dominance=doms[b])
        out.append(m)
    return out


# Named workloads, with the walk parameters they are run with.
WORKLOADS = {
    "stencil2d_32x32": dict(gen=lambda: stencil2d_5pt(32, 32, seed=1001), chains=1000,
                            delta=1e-3, max_len=64, tau=1e-2, top_k=0),
    "stencil3d_64": dict(gen=lambda: stencil3d_7pt(64, seed=1002), chains=256,
                         delta=1e-2, max_len=128, tau=0.0, top_k=16),
    "stencil3d_32": dict(gen=lambda: stencil3d_7pt(32, seed=1002), chains=256,
                         delta=1e-2, max_len=128, tau=0.0, top_k=16),
    "powerlaw_1m": dict(gen=lambda: powerlaw_random(1 << 20, seed=1003), chains=128,
                        delta=1e-3, max_len=256, tau=5e-3, top_k=0),
    "powerlaw_128k": dict(gen=lambda: powerlaw_random(1 << 17, seed=1003), chains=128,
                          delta=1e-3, max_len=256, tau=5e-3, top_k=0),
    "general_128k": dict(gen=lambda: random_dd(1 << 17, 9, seed=1006, dominance=1.4, diag_sign="mixed"),
                         chains=128, delta=1e-3, max_len=256, tau=5e-3, top_k=0, alpha=0.5),
    "aniso2d_1024": dict(gen=lambda: aniso2d_9pt(1024, seed=1005), chains=128,
                         delta=1e-3, max_len=256, tau=1e-2, top_k=0, alpha=0.25),
}


def workload(name):
    w = dict(WORKLOADS[name])
    gen = w.pop("gen")
    return gen(), w
