"""Least squares in the basis of statistically orthogonal polynomials (Sec. 2.1,
DPD_BASIS_ORTHOGONAL) against the FP64 oracle: the estimate is the same
least-squares solution (the basis change is invertible), returned in the
monomial stacking order, and the system it solves is far better conditioned."""
import numpy as np
import pytest

import dpd_synth as synth
import oracle
from oracle import basis

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1612_09001_gb300 as dpd  # noqa: E402


def _problem(P, Q, M, n, seed):
    u, theta = synth.ls_problem(n, P, Q, M, seed=seed)
    t = oracle.apply(u, theta, P, Q, M).astype(np.complex64)
    return u, t, theta


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("tf32x3", 1e-4), ("bf16x3", 1e-3)])
@pytest.mark.parametrize("P,Q,M,n", [(5, 3, 4, 50000), (9, 9, 4, 40000), (11, 11, 7, 70001), (3, 7, 2, 30011),
                                     (1, 0, 0, 1000)])
def test_orthogonal_estimate_matches_oracle(P, Q, M, n, precision, tol):
    u, t, theta = _problem(P, Q, M, n, seed=P + 10 * M)
    f = dpd.DPD(P, Q, M)
    h, st = f.estimate(torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda(), precision=precision,
                       refine_iters=3, basis="orthogonal")
    h = h.cpu().numpy().astype(np.complex128)
    ref = oracle.ls(u, t, P, Q, M)
    h_o, _, _ = basis.lstsq_orthogonal(u, t, P, Q, M)
    assert np.linalg.norm(ref - h_o) <= 1e-8 * np.linalg.norm(ref)   # the oracle's two routes agree
    e_ref = np.linalg.norm(h - ref) / np.linalg.norm(ref)
    e_true = np.linalg.norm(h - theta) / np.linalg.norm(theta)
    assert e_ref <= tol and e_true <= tol, (precision, e_ref, e_true, st)
    assert st["rel_residual"] < 1e-9


def test_orthogonal_basis_conditioning_and_bf16_accuracy():
    """P = Q = 11, M = 7 at 2^18 rows: the orthogonal system's condition number is
    orders of magnitude smaller and BF16x3 without refinement is far closer."""
    P, Q, M, n = 11, 11, 7, 1 << 18
    u, theta = synth.ls_problem(n, P, Q, M, seed=3)
    ud = torch.from_numpy(u).cuda()
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(theta)
    td = f.apply(ud)
    res = {}
    for b in ("monomial", "orthogonal"):
        h, st = f.estimate(ud, td, precision="bf16x3", refine_iters=0, basis=b)
        res[b] = (np.linalg.norm(h.cpu().numpy() - theta) / np.linalg.norm(theta), st["cond_est"])
    assert res["orthogonal"][1] < 1e-2 * res["monomial"][1], res
    assert res["orthogonal"][0] < 0.1 * res["monomial"][0], res
    assert res["orthogonal"][0] < 1e-3, res


def test_orthogonal_batched_matches_single():
    P, Q, M = 7, 7, 3
    us, ts, thetas = [], [], []
    for i in range(6):
        u, t, th = _problem(P, Q, M, 20000 + 977 * i, seed=100 + i)
        us.append(torch.from_numpy(u).cuda())
        ts.append(torch.from_numpy(t).cuda())
        thetas.append(th)
    f = dpd.DPD(P, Q, M)
    hb, info = f.estimate_batched(us, ts, precision="tf32x3", refine_iters=2, basis="orthogonal")
    assert all(i == 0 for i in info)
    for i in range(6):
        hs, _ = f.estimate(us[i], ts[i], precision="tf32x3", refine_iters=2, basis="orthogonal")
        e = np.linalg.norm(hb[i].cpu().numpy() - thetas[i]) / np.linalg.norm(thetas[i])
        assert e < 1e-5, (i, e)
        assert np.allclose(hb[i].cpu().numpy(), hs.cpu().numpy(), rtol=0, atol=1e-6)


def test_orthogonal_basis_degenerate_input_reports_not_spd():
    """All-zero input: the moment matrix is singular (the basis falls back to the
    monomials) and the Gram matrix is not positive definite."""
    f = dpd.DPD(5, 5, 2)
    u = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    t = torch.ones(4096, dtype=torch.complex64, device="cuda")
    with pytest.raises(dpd.DPDError) as e:
        f.estimate(u, t, basis="orthogonal")
    assert e.value.code == 6   # DPD_ERR_NOT_SPD


def test_estimate_basis_rejects_unknown():
    f = dpd.DPD(5, 5, 2)
    from paper_1612_09001_gb300 import _lib
    assert _lib.load().dpd_set_estimate_basis(f.handle, 7) == 1
