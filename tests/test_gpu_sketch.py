"""The two forms of the log's magnitude sketch in the FP32 depth-8 kernel.

While at least 9 of the 32 bits of a column index are spare (n <= 2^23), a
log entry's column word also carries a rounded-up code of |1/d_j| and the
sketch is built after the walks in shared memory; with fewer spare bits the
walks add each logged visit's magnitude to global cells instead.  Either way
the sketch only decides which logged columns are reduced: the rows must match
the oracle.  The matrices hold power-law rows over their first 2^16 columns
(each row reaches more columns than the on-chip table holds, so most visits
are logged) inside an identity of 2^23 (9 spare bits, the narrowest code) or
2^23 + 64 rows (walk-time cells); the first 512 rows are built.
"""
import numpy as np
import pytest

import synth
from tests.test_gpu_full_size import SEED, _check, _sample

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402


def _embedded(n, seed):
    m0 = synth.powerlaw_random(n=1 << 16, seed=seed)
    n0, extra = m0.n, n - m0.n
    rp = np.concatenate([m0.row_ptr, m0.nnz + np.arange(1, extra + 1, dtype=np.int64)])
    col = np.concatenate([m0.col, np.arange(n0, n, dtype=np.int32)])
    val = np.concatenate([m0.val, np.ones(extra)])
    return synth.Csr(n, rp, col, val)


@pytest.mark.parametrize("n", [1 << 23, (1 << 23) + 64])
def test_sketch_forms_match_oracle(n):
    m = _embedded(n, 1011)
    B = mc.DeviceCsr.from_host(m)
    tau = 5e-3
    p = mc.params(chains=128, max_len=256, delta=1e-3, filter_tau=tau, top_k=0, seed=SEED)
    p.row_begin, p.row_end, p.load_depth = 0, 512, 8
    M = mc.mcmi_build_ex(B, p)
    assert M.stats.load_depth == 8
    _check(f"power-law rows in an identity of n = {n}", m, B, p, M, _sample(512, 24, 9), M.stats.table, tau, 0,
           threads=4)
