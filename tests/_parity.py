"""Comparison helpers for the GPU-vs-oracle parity tests (test infrastructure)."""
import numpy as np

# Entry tolerance: FP32 walk weights accumulate at most ~t 2^-24 relative
# rounding over t transitions (t <= 64 here: 3.8e-6), plus FP32 rounding of
# 1/d_j and of the compensated sum; 1e-5 relative covers it.  Where signed
# weights cancel, the bound is taken relative to A = (1/N) sum |W| / |d_j|.
REL_TOL = 1e-5


def entry_errors(g_val, o_X, o_A, dcol):
    """Absolute error, plain relative error and the bounded error ratio
    |g - o| / (tol * max(|o|, A)) for D-scaled entries."""
    o = o_X / dcol
    a = o_A / np.abs(dcol)
    err = np.abs(g_val - o)
    rel = err / np.maximum(np.abs(o), 1e-300)
    bounded = err / (REL_TOL * np.maximum(np.abs(o), a))
    return err, rel, bounded


def compare_dump(gpu_rows, orc_rows, d):
    """Bit-exact columns, visit counts and step counts; bounded value error.
    Returns (max plain rel error, median plain rel error, max bounded ratio)."""
    rels, worst = [], 0.0
    for g, o in zip(gpu_rows, orc_rows):
        assert np.array_equal(g["col"], o["col"]), f"row {o['row']}: visited columns differ"
        assert np.array_equal(g["visits"].astype(np.uint64), o["V"].astype(np.uint64)), f"row {o['row']}: visits differ"
        assert g["steps"] == o["steps"], f"row {o['row']}: steps {g['steps']} vs {o['steps']}"
        err, rel, bounded = entry_errors(g["val"], o["X"], o["A"], d[o["col"]])
        rels.append(rel)
        worst = max(worst, float(bounded.max(initial=0.0)))
    rel = np.concatenate(rels) if rels else np.zeros(1)
    return float(rel.max(initial=0.0)), float(np.median(rel)), worst


def band_entries(cols, mvals, i, tau, top_k, band=REL_TOL):
    """Columns whose filter decision is within the rounding band of a cut:
    |M| within a relative band of 1e-5 of tau * max|M| or of the top_k-th
    value (the entry tolerance; the measured entry errors are below 2e-6,
    so an entry and the cut cannot move past each other outside it)."""
    mag = np.abs(mvals)
    amb = np.zeros(len(cols), dtype=bool)
    off = cols != i
    thr = tau * mag.max(initial=0.0)
    if tau > 0:
        amb |= off & (np.abs(mag - thr) <= band * np.maximum(thr, 1e-300))
    if top_k > 0:
        cand = off & ((tau == 0) | (mag >= thr * (1 - band)))
        cm = np.sort(mag[cand])[::-1]
        if len(cm) > top_k:
            kth = cm[top_k - 1]
            amb |= off & (np.abs(mag - kth) <= band * kth)
    return set(cols[amb].tolist())


def compare_rows(g_cols, g_vals, o_cols, o_vals, unf_cols, unf_m, unf_a, i, tau, top_k):
    """Kept patterns equal up to band entries; shared values within the
    tolerance (bounded by A where signed weights cancel).
    Returns (max plain relative error, max bounded ratio)."""
    gs, os_ = set(g_cols.tolist()), set(o_cols.tolist())
    diff = gs ^ os_
    if diff:
        amb = band_entries(unf_cols, unf_m, i, tau, top_k)
        assert diff <= amb, f"row {i}: pattern differs outside the band: {sorted(diff - amb)[:8]}"
    gi = dict(zip(g_cols.tolist(), g_vals.tolist()))
    oi = dict(zip(o_cols.tolist(), o_vals.tolist()))
    ai = dict(zip(unf_cols.tolist(), unf_a.tolist()))
    rel = bounded = 0.0
    for c in gs & os_:
        e = abs(gi[c] - oi[c])
        rel = max(rel, e / max(abs(oi[c]), 1e-300))
        bounded = max(bounded, e / (REL_TOL * max(abs(oi[c]), ai[c])))
    return rel, bounded
