"""Recovery of B^-1 from Bhat^-1 (Eq. 3) on the GPU against the oracle:
bit-identical updates, the exact inverse recovered from the exact Bhat^-1,
and the diagnostic it serves: how far the recovered M is from B^-1."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402


def _orc():
    import oracle
    return oracle


@pytest.mark.parametrize("alpha", [0.4, 2.0])
def test_recovery_bit_identical_and_exact(alpha):
    orc = _orc()
    m = synth.random_dd(300, 7, seed=51, dominance=1.3, diag_sign="mixed")
    B = mc.DeviceCsr.from_host(m)
    s = orc.augmentation(m, alpha)
    d1, _ = orc.split(m, alpha)
    Bd = m.to_scipy().toarray()
    Bh = Bd.copy()
    Bh[np.diag_indices(m.n)] = d1
    X0 = np.linalg.inv(Bh)
    ref = orc.recover_dense(X0, s)
    X = torch.from_numpy(X0.copy()).cuda()
    mc.mcmi_recover_dense(B, alpha, X)
    got = X.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    inv = np.linalg.inv(Bd)
    assert np.abs(got - inv).max() <= 1e-9 * np.abs(inv).max()


def test_recovered_preconditioner_gap():
    """The diagnostic: M approximates Bhat^-1; Eq. 3 applied to M moves it
    toward B^-1 (GPU and oracle bit-identical from the same dense M)."""
    orc = _orc()
    m = synth.random_dd(400, 6, seed=52, dominance=1.2, diag_sign="mixed")
    alpha = 0.5
    B = mc.DeviceCsr.from_host(m)
    M = mc.mcmi_build_ex(B, mc.params(chains=4000, max_len=200, delta=1e-6, alpha=alpha, seed=9))
    Xd = mc.mcmi_matrix_dense(M, m.n)
    rp, col, val = (t.cpu().numpy() for t in M.to_torch())
    torch.cuda.synchronize()
    dense = np.zeros((m.n, m.n))
    for i in range(m.n):
        dense[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]].astype(np.float64)
    assert np.array_equal(Xd.cpu().numpy(), dense)
    ref = orc.recover_dense(dense, orc.augmentation(m, alpha))
    mc.mcmi_recover_dense(B, alpha, Xd)
    got = Xd.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    Bd = m.to_scipy().toarray()
    inv = np.linalg.inv(Bd)
    d1, _ = orc.split(m, alpha)
    Bh = Bd.copy()
    Bh[np.diag_indices(m.n)] = d1
    gap_m = np.linalg.norm(dense - inv) / np.linalg.norm(inv)
    gap_mhat = np.linalg.norm(dense - np.linalg.inv(Bh)) / np.linalg.norm(np.linalg.inv(Bh))
    gap_rec = np.linalg.norm(got - inv) / np.linalg.norm(inv)
    print(f"||M - Bhat^-1|| {gap_mhat:.3e}  ||M - B^-1|| {gap_m:.3e}  ||recovered - B^-1|| {gap_rec:.3e}")
    assert gap_rec < gap_m


def test_recover_errors():
    B = mc.DeviceCsr.from_host(synth.random_dd(20, 3, seed=1))
    X = torch.zeros((20, 20), dtype=torch.float64, device="cuda")
    with pytest.raises(mc.McmiError) as e:
        mc.mcmi_recover_dense(B, -1.0, X)
    assert e.value.status == 1
