"""Python binding of libmcmi, the B300 (sm_103a) (MC)^2MI preconditioner.

Argument marshalling only: every stage runs in the CUDA kernels of
``libmcmi.so`` behind the C ABI declared in ``include/mcmi.h``.  PyTorch
provides device memory and streams.  The names mirror the C entry points.
There is no CPU fallback: importing this package on a machine without the
built library raises, and every call needs a CUDA device.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmcmi.so")

MCMI_OK = 0
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_BAD_CSR", 3: "ERR_ZERO_DIAG", 4: "ERR_NOT_CONTRACTIVE",
          5: "ERR_OOM", 6: "ERR_CUDA", 7: "ERR_TIMEOUT", 8: "ERR_CAPACITY"}
TABLE_AUTO, TABLE_CUMULATIVE, TABLE_ALIAS, TABLE_HYBRID, TABLE_COMPACT = -1, 0, 1, 2, 3
TABLE_NAMES = {0: "cumulative", 1: "alias", 2: "hybrid", 3: "compact"}
ACC_FIXED64, ACC_KAHAN32 = 0, 1


class McmiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class mcmi_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class mcmi_params(C.Structure):
    _fields_ = [("eps", C.c_double), ("delta", C.c_double), ("filter_tau", C.c_double), ("alpha", C.c_double),
                ("seed", C.c_uint64), ("chains", C.c_int32), ("max_len", C.c_int32), ("top_k", C.c_int32),
                ("precision", C.c_int32), ("table", C.c_int32), ("threads", C.c_int32), ("hash_log2", C.c_int32),
                ("accumulator", C.c_int32), ("row_begin", C.c_int64), ("row_end", C.c_int64),
                ("chains_per_thread", C.c_int32), ("load_depth", C.c_int32), ("proposal", C.c_void_p)]


class mcmi_train_params(C.Structure):
    _fields_ = [("steps", C.c_int32), ("lr", C.c_float), ("chains", C.c_int32), ("max_len", C.c_int32),
                ("delta", C.c_double), ("alpha", C.c_double), ("seed", C.c_uint64), ("round_bf16", C.c_int32),
                ("reserved", C.c_int32)]


class mcmi_stats(C.Structure):
    _fields_ = [("steps", C.c_uint64), ("rows", C.c_int64), ("nnz", C.c_int64), ("max_s", C.c_double),
                ("chains", C.c_int32), ("max_len_bound", C.c_int32), ("table", C.c_int32), ("hash_log2", C.c_int32),
                ("spilled", C.c_int64), ("deferred_rows", C.c_int64), ("ms_prepare", C.c_float),
                ("ms_walk", C.c_float), ("ms_assemble", C.c_float), ("ms_walk_kernel", C.c_float),
                ("launches", C.c_int32), ("threads", C.c_int32), ("chains_per_thread", C.c_int32),
                ("load_depth", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class mcmi_tune_result(C.Structure):
    _fields_ = [("threads", C.c_int32), ("chains_per_thread", C.c_int32), ("hash_log2", C.c_int32),
                ("table", C.c_int32), ("trials", C.c_int32), ("best_ms", C.c_float), ("default_ms", C.c_float),
                ("load_depth", C.c_int32), ("sample_rows", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


_lib = None


def load():
    """Load libmcmi.so from the package directory (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmcmi.so not built ({LIB_PATH}); run python -m paper_2409_03095_b300.build")
    lib = C.CDLL(LIB_PATH)
    P, i32, i64, u64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    lib.mcmi_params_default.argtypes = [C.POINTER(mcmi_params)]
    lib.mcmi_params_default.restype = None
    lib.mcmi_build.argtypes = [C.POINTER(mcmi_csr), f64, f64, i32, f64, u64, P, C.POINTER(P)]
    lib.mcmi_build_ex.argtypes = [C.POINTER(mcmi_csr), C.POINTER(mcmi_params), P, C.POINTER(P), C.POINTER(mcmi_stats)]
    lib.mcmi_matrix_csr.argtypes = [P, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(P), C.POINTER(P),
                                    C.POINTER(P)]
    lib.mcmi_matrix_copy.argtypes = [P, P, P, P, P]
    lib.mcmi_apply.argtypes = [P, P, P, P]
    lib.mcmi_free.argtypes = [P]
    lib.mcmi_free.restype = None
    lib.mcmi_last_error.restype = C.c_char_p
    lib.mcmi_version.restype = C.c_char_p
    lib.mcmi_walk_dump.argtypes = [C.POINTER(mcmi_csr), C.POINTER(mcmi_params), P, i64, i64, P, P, P, P, P, P]
    lib.mcmi_debug_tables.argtypes = [C.POINTER(mcmi_csr), C.POINTER(mcmi_params), P, P, P, P, P, P, P]
    lib.mcmi_exclusive_scan_noalloc.argtypes = [P, i64, P, P]
    lib.mcmi_gather_roofline.argtypes = [u64, i32, i32, i32, i32, C.POINTER(f64), P]
    lib.mcmi_gather_roofline.restype = C.c_int
    lib.mcmi_gather_roofline_mix.argtypes = [u64, u64, f64, i32, i32, i32, C.POINTER(f64), P]
    lib.mcmi_gather_roofline_mix.restype = C.c_int
    lib.mcmi_solve.argtypes = [C.POINTER(mcmi_csr), P, P, P, C.c_int, f64, i32, i32, C.POINTER(i32), C.POINTER(f64), P]
    lib.mcmi_solve.restype = C.c_int
    lib.mcmi_autotune.argtypes = [C.POINTER(mcmi_csr), C.POINTER(mcmi_params), P, C.POINTER(mcmi_tune_result)]
    lib.mcmi_autotune.restype = C.c_int
    lib.mcmi_build_batched.argtypes = [P, i32, C.POINTER(mcmi_params), P, P, C.POINTER(mcmi_stats)]
    lib.mcmi_build_batched.restype = C.c_int
    lib.mcmi_proposal_create.argtypes = [P, C.POINTER(P)]
    lib.mcmi_proposal_get.argtypes = [P, P]
    lib.mcmi_proposal_free.argtypes = [P]
    lib.mcmi_proposal_free.restype = None
    lib.mcmi_row_moments.argtypes = [C.POINTER(mcmi_csr), C.POINTER(mcmi_params), P, P]
    lib.mcmi_proposal_loss_grad.argtypes = [C.POINTER(mcmi_csr), P, C.POINTER(mcmi_params), P, C.c_int,
                                            C.POINTER(C.c_float), P, P]
    lib.mcmi_proposal_train.argtypes = [P, i32, C.POINTER(mcmi_train_params), P, P, P]
    for f in ("mcmi_proposal_create", "mcmi_proposal_get", "mcmi_row_moments", "mcmi_proposal_loss_grad",
              "mcmi_proposal_train"):
        getattr(lib, f).restype = C.c_int
    lib.mcmi_recover_dense.argtypes = [C.POINTER(mcmi_csr), f64, P, P]
    lib.mcmi_recover_dense.restype = C.c_int
    lib.mcmi_matrix_dense.argtypes = [P, P, P]
    lib.mcmi_matrix_dense.restype = C.c_int
    lib.mcmi_reduce.argtypes = [C.POINTER(mcmi_csr), f64, i32, P, C.POINTER(P), C.POINTER(i64)]
    lib.mcmi_reduce.restype = C.c_int
    lib.mcmi_reduced_csr.argtypes = [P, C.POINTER(mcmi_csr)]
    lib.mcmi_reduced_csr.restype = C.c_int
    lib.mcmi_reduced_copy.argtypes = [P, P, P, P, P]
    lib.mcmi_reduced_copy.restype = C.c_int
    lib.mcmi_reduced_free.argtypes = [P]
    lib.mcmi_reduced_free.restype = None
    for f in ("mcmi_build", "mcmi_build_ex", "mcmi_matrix_csr", "mcmi_matrix_copy", "mcmi_apply",
              "mcmi_walk_dump", "mcmi_debug_tables", "mcmi_exclusive_scan_noalloc"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def _check(st):
    if st != MCMI_OK:
        raise McmiError(st, load().mcmi_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def params(**kw) -> mcmi_params:
    """mcmi_params with the library defaults, overridden by keyword."""
    p = mcmi_params()
    load().mcmi_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        if k == "proposal" and hasattr(v, "h"):
            v = v.h
        setattr(p, k, v)
    return p


class DeviceCsr:
    """A CSR matrix in device memory (torch tensors) and its mcmi_csr view."""

    def __init__(self, n, row_ptr, col, val):
        self.n = int(n)
        self.row_ptr, self.col, self.val = row_ptr, col, val
        self.c = mcmi_csr(self.n, int(col.numel()), row_ptr.data_ptr(), col.data_ptr(), val.data_ptr())

    @classmethod
    def from_host(cls, m, device="cuda"):
        import torch
        rp = torch.from_numpy(np.ascontiguousarray(m.row_ptr, dtype=np.int64)).to(device)
        col = torch.from_numpy(np.ascontiguousarray(m.col, dtype=np.int32)).to(device)
        val = torch.from_numpy(np.ascontiguousarray(m.val, dtype=np.float64)).to(device)
        return cls(m.n, rp, col, val)


class Matrix:
    """Library-owned preconditioner M (freed with the object or close())."""

    def __init__(self, handle, stats=None):
        self.h = handle
        self.stats = stats

    def close(self):
        if self.h:
            load().mcmi_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self):
        rows, rb, nnz = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().mcmi_matrix_csr(self.h, C.byref(rows), C.byref(rb), C.byref(nnz), None, None, None))
        return rows.value, rb.value, nnz.value

    def to_torch(self, stream=None):
        """Copy of M as (row_ptr int64, col int32, val float32) CUDA tensors."""
        import torch
        rows, rb, nnz = self.shape()
        rp = torch.empty(rows + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        val = torch.empty(max(nnz, 1), dtype=torch.float32, device="cuda")
        _check(load().mcmi_matrix_copy(self.h, _ptr(rp), _ptr(col), _ptr(val), _stream(stream)))
        return rp, col[:nnz], val[:nnz]


def mcmi_recover_dense(B: DeviceCsr, alpha, X, stream=None):
    """Eq. 3 recovery (Algorithm 1 step 5) in place on the dense row-major
    FP64 CUDA tensor X (n x n) holding Bhat^-1 or an approximation of it."""
    assert X.dtype.is_floating_point and X.element_size() == 8 and X.is_contiguous()
    _check(load().mcmi_recover_dense(C.byref(B.c), float(alpha), _ptr(X), _stream(stream)))
    return X


def mcmi_matrix_dense(M, n, stream=None):
    """Dense FP64 copy of M (its rows x the n columns of the matrix it was
    built from) as a CUDA tensor."""
    import torch
    rows, rb, nnz = M.shape()
    X = torch.empty((rows, n), dtype=torch.float64, device="cuda")
    _check(load().mcmi_matrix_dense(M.h, _ptr(X), _stream(stream)))
    return X


REDUCE_ENTRIES, REDUCE_RANGE = 0, 1


class Reduced:
    """Library-owned reduced input matrix (FP64 CSR, device); ``.c`` is its
    mcmi_csr view, so it can be passed to the builds as B."""

    def __init__(self, handle, dropped):
        self.h = handle
        self.dropped = dropped
        self.c = mcmi_csr()
        _check(load().mcmi_reduced_csr(self.h, C.byref(self.c)))
        self.n = int(self.c.n)

    @property
    def nnz(self):
        return int(self.c.nnz)

    def to_torch(self, stream=None):
        """Copy as (row_ptr int64, col int32, val float64) CUDA tensors."""
        import torch
        rp = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(self.nnz, 1), dtype=torch.int32, device="cuda")
        val = torch.empty(max(self.nnz, 1), dtype=torch.float64, device="cuda")
        _check(load().mcmi_reduced_copy(self.h, _ptr(rp), _ptr(col), _ptr(val), _stream(stream)))
        return rp, col[:self.nnz], val[:self.nnz]

    def close(self):
        if self.h:
            load().mcmi_reduced_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mcmi_reduce(B: DeviceCsr, fraction, mode=REDUCE_ENTRIES, stream=None) -> Reduced:
    """Matrix reduction of Algorithm 1 step 2 (drop the smallest off-diagonal
    entries: a share of the entries, or of the value range)."""
    h, d = C.c_void_p(), C.c_int64()
    _check(load().mcmi_reduce(C.byref(B.c), float(fraction), int(mode), _stream(stream), C.byref(h), C.byref(d)))
    return Reduced(h, d.value)


def mcmi_build(B: DeviceCsr, eps, delta, chains, filter_tau, seed, stream=None) -> Matrix:
    h = C.c_void_p()
    _check(load().mcmi_build(C.byref(B.c), eps, delta, chains, filter_tau, seed, _stream(stream), C.byref(h)))
    return Matrix(h)


def mcmi_build_ex(B: DeviceCsr, p: mcmi_params, stream=None) -> Matrix:
    h = C.c_void_p()
    st = mcmi_stats()
    _check(load().mcmi_build_ex(C.byref(B.c), C.byref(p), _stream(stream), C.byref(h), C.byref(st)))
    return Matrix(h, st)


def mcmi_build_batched(Bs, p: mcmi_params, stream=None):
    """Build preconditioners of several matrices in one batched launch.
    Returns (list of Matrix, aggregate mcmi_stats)."""
    arr = (mcmi_csr * len(Bs))(*[B.c for B in Bs])
    hs = (C.c_void_p * len(Bs))()
    st = mcmi_stats()
    _check(load().mcmi_build_batched(C.cast(arr, C.c_void_p), len(Bs), C.byref(p), _stream(stream),
                                     C.cast(hs, C.c_void_p), C.byref(st)))
    return [Matrix(C.c_void_p(h)) for h in hs], st


def mcmi_apply(M: Matrix, x, y, stream=None):
    _check(load().mcmi_apply(M.h, _ptr(x), _ptr(y), _stream(stream)))
    return y


def mcmi_walk_dump(B: DeviceCsr, p: mcmi_params, rows, cap, stream=None):
    """Unfiltered estimate of the listed rows (parity entry point); returns a
    list of dicts with col, val (D-scaled), visits, steps (host numpy)."""
    import torch
    rows_t = torch.as_tensor(np.asarray(rows, dtype=np.int64)).cuda()
    nr = rows_t.numel()
    cnt = torch.zeros(nr, dtype=torch.int32, device="cuda")
    steps = torch.zeros(nr, dtype=torch.int64, device="cuda")
    col = torch.zeros(nr * cap, dtype=torch.int32, device="cuda")
    val = torch.zeros(nr * cap, dtype=torch.float64, device="cuda")
    vis = torch.zeros(nr * cap, dtype=torch.int32, device="cuda")
    _check(load().mcmi_walk_dump(C.byref(B.c), C.byref(p), _ptr(rows_t), nr, cap, _ptr(cnt), _ptr(steps),
                                 _ptr(col), _ptr(val), _ptr(vis), _stream(stream)))
    cnt, steps = cnt.cpu().numpy(), steps.cpu().numpy().view(np.uint64)
    col, val, vis = col.cpu().numpy(), val.cpu().numpy(), vis.cpu().numpy().view(np.uint32)
    out = []
    for i in range(nr):
        a, b = i * cap, i * cap + int(cnt[i])
        o = np.argsort(col[a:b], kind="stable")
        out.append(dict(col=col[a:b][o], val=val[a:b][o], visits=vis[a:b][o], steps=int(steps[i])))
    return out


def mcmi_debug_tables(B: DeviceCsr, p: mcmi_params, stream=None):
    import torch
    n, nnz = B.n, int(B.col.numel())
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = torch.zeros(n, dtype=torch.float64, device="cuda")
    slot = torch.zeros(16 * n, dtype=torch.int32, device="cuda")
    a = torch.zeros(max(nnz, 1), dtype=torch.int32, device="cuda")
    b = torch.zeros(max(nnz, 1), dtype=torch.int32, device="cuda")
    c = torch.zeros(max(nnz, 1), dtype=torch.int32, device="cuda")
    _check(load().mcmi_debug_tables(C.byref(B.c), C.byref(p), _ptr(d), _ptr(s), _ptr(slot), _ptr(a), _ptr(b),
                                    _ptr(c), _stream(stream)))
    torch.cuda.synchronize()
    u = lambda t: t.cpu().numpy().view(np.uint32)
    out = dict(d=d.cpu().numpy(), s=s.cpu().numpy(), slot=u(slot).reshape(n, 16), a=u(a), b=u(b), c=u(c))
    # the compact table's 32-byte records are packed at the start
    out["rec32"] = u(slot)[:8 * n].reshape(n, 8)
    return out


def mcmi_exclusive_scan_noalloc(counts, offsets, stream=None):
    """offsets[i] = sum(counts[:i]) for i = 0..n, without any allocation in
    the library (for callers that cannot allocate device memory; scratch is a
    fixed 128 KB device array, n <= 33,554,432; overlapping calls race)."""
    _check(load().mcmi_exclusive_scan_noalloc(_ptr(counts), counts.numel(), _ptr(offsets), _stream(stream)))
    return offsets


def mcmi_autotune(B: DeviceCsr, p: mcmi_params, stream=None):
    """Times walk configurations on a row sample and writes the fastest into
    p (threads, chains_per_thread, hash_log2, table, load_depth); returns the
    report."""
    res = mcmi_tune_result()
    _check(load().mcmi_autotune(C.byref(B.c), C.byref(p), _stream(stream), C.byref(res)))
    return res


MLP_PARAMS = 1377


class Proposal:
    """Learned proposal (BF16 MLP over edge features); pass as
    params(proposal=P.h) or use P.params(...)."""

    def __init__(self, params=None):
        self.h = C.c_void_p()
        arr = None
        if params is not None:
            arr = np.ascontiguousarray(params, dtype=np.float32)
            assert arr.size == MLP_PARAMS
        _check(load().mcmi_proposal_create(arr.ctypes.data_as(C.c_void_p) if arr is not None else None,
                                           C.byref(self.h)))

    def get(self):
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(load().mcmi_proposal_get(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def close(self):
        if self.h:
            load().mcmi_proposal_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mcmi_row_moments(B: DeviceCsr, p: mcmi_params, stream=None):
    import torch
    m = torch.zeros(B.n, dtype=torch.float32, device="cuda")
    _check(load().mcmi_row_moments(C.byref(B.c), C.byref(p), _ptr(m), _stream(stream)))
    return m


def mcmi_proposal_loss_grad(B: DeviceCsr, m_rows, p: mcmi_params, P: Proposal, round_bf16=1, grad=True, stream=None):
    loss = C.c_float()
    g = np.zeros(MLP_PARAMS, dtype=np.float32) if grad else None
    _check(load().mcmi_proposal_loss_grad(C.byref(B.c), _ptr(m_rows), C.byref(p), P.h, round_bf16, C.byref(loss),
                                          g.ctypes.data_as(C.c_void_p) if grad else None, _stream(stream)))
    return loss.value, g


def mcmi_proposal_train(Bs, tp: mcmi_train_params, P: Proposal, stream=None):
    arr = (mcmi_csr * len(Bs))(*[B.c for B in Bs])
    hist = np.zeros(max(tp.steps, 1), dtype=np.float32)
    _check(load().mcmi_proposal_train(C.cast(arr, C.c_void_p), len(Bs), C.byref(tp), P.h,
                                      hist.ctypes.data_as(C.c_void_p), _stream(stream)))
    return hist[:tp.steps]


SOLVE_BICGSTAB, SOLVE_GMRES = 0, 1


def mcmi_solve(B: DeviceCsr, M, b, x, method=SOLVE_BICGSTAB, rtol=1e-8, maxit=10000, restart=30, stream=None):
    """Right-preconditioned BiCGstab / GMRES(restart) on the device (FP64).
    M: Matrix or None.  Returns (iterations, true relative residual)."""
    it, rr = C.c_int32(), C.c_double()
    _check(load().mcmi_solve(C.byref(B.c), M.h if M is not None else None, _ptr(b), _ptr(x), method, rtol, maxit,
                             restart, C.byref(it), C.byref(rr), _stream(stream)))
    return it.value, rr.value


def mcmi_gather_roofline(footprint_bytes, threads_per_block=128, blocks_per_sm=6, steps=64, stream=None,
                         record_bytes=64):
    """Random dependent record reads (64- or 32-byte records) per second over
    a buffer of the given size at the given occupancy (the walk's access
    pattern)."""
    r = C.c_double()
    _check(load().mcmi_gather_roofline(int(footprint_bytes), int(record_bytes), threads_per_block, blocks_per_sm,
                                       steps, C.byref(r), _stream(stream)))
    return r.value


def mcmi_gather_roofline_mix(record_footprint_bytes, bucket_footprint_bytes, bucket_share, threads_per_block=128,
                             blocks_per_sm=8, steps=64, stream=None):
    """Dependent 64-byte record reads per second where a share of them is
    followed by a dependent 16-byte bucket read (the hybrid table's walk)."""
    r = C.c_double()
    _check(load().mcmi_gather_roofline_mix(int(record_footprint_bytes), int(bucket_footprint_bytes),
                                           float(bucket_share), threads_per_block, blocks_per_sm, steps,
                                           C.byref(r), _stream(stream)))
    return r.value


def version() -> str:
    return load().mcmi_version().decode()
