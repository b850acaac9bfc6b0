"""Krylov judge (mcmi_solve) against scipy with the same preconditioner."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import scipy.sparse as sp  # noqa: E402
import scipy.sparse.linalg as spla  # noqa: E402

import paper_2409_03095_b300 as mc  # noqa: E402


def _scipy_M(M, n):
    rp, col, val = (t.cpu().numpy() for t in M.to_torch())
    torch.cuda.synchronize()
    return sp.csr_matrix((val.astype(np.float64), col, rp), shape=(n, n))


def _scipy_bicgstab_iters(A, b, Mop, rtol):
    it = [0]

    def cb(xk):
        it[0] += 1
    x, info = spla.bicgstab(A, b, rtol=rtol, atol=0.0, M=Mop, maxiter=10000, callback=cb)
    return x, it[0], info


@pytest.mark.parametrize("name", ["stencil3d", "nonsym"])
def test_bicgstab_matches_scipy(name):
    if name == "stencil3d":
        m = synth.stencil3d_7pt(16, seed=21)
        p = mc.params(chains=256, max_len=128, delta=1e-2, top_k=16, seed=4)
    else:
        m = synth.random_dd(3000, 8, seed=22, diag_sign="mixed", dominance=0.9)
        p = mc.params(chains=128, max_len=128, delta=1e-3, filter_tau=2e-2, seed=4)
    A = m.to_scipy()
    B = mc.DeviceCsr.from_host(m)
    M = mc.mcmi_build_ex(B, p)
    bh = np.random.default_rng(3).standard_normal(m.n)
    b = torch.from_numpy(bh).cuda()
    x = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    for Mh in (M, None):
        it, rr = mc.mcmi_solve(B, Mh, b, x, mc.SOLVE_BICGSTAB, rtol=1e-8)
        xs = x.cpu().numpy()
        assert rr <= 1e-8 * 1.5, rr
        assert np.linalg.norm(A @ xs - bh) / np.linalg.norm(bh) == pytest.approx(rr, rel=1e-3, abs=1e-12)
        Mop = _scipy_M(M, m.n) if Mh is not None else None
        xr, its, info = _scipy_bicgstab_iters(A, bh, Mop, 1e-8)
        assert info == 0
        # same algorithm (right-preconditioned BiCGstab), same M: iteration
        # counts within 2 of scipy's.  Unpreconditioned, the nonsymmetric
        # problem takes 100+ iterations whose count is chaotic in the
        # rounding: scipy's own count spreads over 112-144 when b is
        # perturbed by one unit in the last place, so there the count is
        # only held to a quarter of scipy's median over such perturbations
        if Mh is not None or name == "stencil3d":
            assert abs(it - its) <= 2, (it, its)
        else:
            rng = np.random.default_rng(7)
            own = [_scipy_bicgstab_iters(A, bh * (1 + rng.standard_normal(m.n) * 2.0 ** -52), None, 1e-8)[1]
                   for _ in range(8)] + [its]
            assert abs(it - np.median(own)) <= 0.25 * np.median(own), (it, own)
    it_m, _ = mc.mcmi_solve(B, M, b, x, mc.SOLVE_BICGSTAB, rtol=1e-8)
    it_0, _ = mc.mcmi_solve(B, None, b, x, mc.SOLVE_BICGSTAB, rtol=1e-8)
    assert it_m < it_0, (it_m, it_0)


def test_gmres_converges_and_preconditioning_helps():
    m = synth.random_dd(2500, 10, seed=31, diag_sign="mixed", dominance=0.92)
    A = m.to_scipy()
    B = mc.DeviceCsr.from_host(m)
    M = mc.mcmi_build_ex(B, mc.params(chains=128, max_len=128, delta=1e-3, filter_tau=1e-2, seed=2))
    bh = np.random.default_rng(4).standard_normal(m.n)
    b = torch.from_numpy(bh).cuda()
    x = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    ref = spla.spsolve(A.tocsc(), bh)
    its = {}
    for key, Mh in (("M", M), ("none", None)):
        it, rr = mc.mcmi_solve(B, Mh, b, x, mc.SOLVE_GMRES, rtol=1e-9, restart=30)
        assert rr <= 2e-9, rr
        assert np.allclose(x.cpu().numpy(), ref, rtol=1e-6, atol=1e-9 * np.abs(ref).max())
        its[key] = it
    assert its["M"] < its["none"]


def test_solve_bad_arguments():
    m = synth.random_dd(10, 3, seed=1)
    B = mc.DeviceCsr.from_host(m)
    b = torch.ones(10, dtype=torch.float64, device="cuda")
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(mc.McmiError):
        mc.mcmi_solve(B, None, b, x, method=7)
    with pytest.raises(mc.McmiError):
        mc.mcmi_solve(B, None, b, x, rtol=0.0)
