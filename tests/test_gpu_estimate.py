"""Least-squares estimation on the GPU (Sec. 2.2): the Gram matrix Psi^H Psi
and Psi^H t in every precision mode against the FP64 oracle, and the solved
coefficients against the FP64 oracle's solution and against the coefficients
that generated the data."""
import numpy as np
import pytest

import dpd_synth as synth
import oracle
from oracle import basis

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1612_09001_gb300 as dpd  # noqa: E402

# Element-wise bound of the Gram, relative to sqrt(G_aa G_bb) (Cauchy-Schwarz):
# FP32 accumulation for every mode; BF16 hi+lo keeps about 16 mantissa bits.
GRAM_TOL = {"fp32": 2e-6, "tf32x3": 2e-6, "bf16x3": 5e-5}


def _gram_check(P, Q, M, n, precision, seed):
    u = synth.clipped_gaussian(n, 0.4, key=(60, seed, 0))
    t = synth.ofdm2(n, key=(60, seed, 1))
    f = dpd.DPD(P, Q, M)
    G, g, tt = f.gram(torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda(), precision=precision)
    f.sync_status()
    Gr, gr = oracle.gram(u, t, P, Q, M)
    G = G.cpu().numpy()
    g = g.cpu().numpy()
    d = np.sqrt(np.abs(np.diag(Gr)))
    scale = np.outer(d, d)
    zero = scale == 0          # columns that are identically zero (taps beyond a short input)
    assert np.all(G[zero] == 0), "entries of all-zero columns must be exactly zero"
    err = np.abs(G - Gr)[~zero] / scale[~zero]
    tol = GRAM_TOL[precision]
    assert err.max() <= tol, (P, Q, M, n, precision, err.max())
    tts = float(np.sum(np.abs(t.astype(np.complex128)) ** 2))
    nz = d > 0
    assert np.all(g[~nz] == 0)
    gerr = np.abs(g - gr)[nz] / (d[nz] * np.sqrt(tts))
    assert gerr.max() <= tol, (precision, gerr.max())
    assert abs(tt - tts) <= tol * tts


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("P,Q,M,n", [(5, 3, 4, 5003), (1, 0, 0, 100), (9, 9, 4, 20011), (9, 9, 6, 3001),
                                     (11, 11, 7, 4099), (3, 1, 2, 63), (7, 7, 3, 1), (3, 7, 2, 2001),
                                     (1, 5, 3, 777), (11, 11, 7, 64 * 152 * 4 + 13)])
def test_gram_against_oracle(P, Q, M, n, precision):
    _gram_check(P, Q, M, n, precision, seed=P * 100 + M * 10 + n % 7)


def _ls_problem(P, Q, M, n, seed):
    u, theta = synth.ls_problem(n, P, Q, M, seed=seed)
    t = oracle.apply(u, theta, P, Q, M).astype(np.complex64)   # noise-free target from the model
    return u, t, theta


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("tf32x3", 1e-4), ("bf16x3", 1e-3)])
def test_estimate_recovers_model_coefficients(precision, tol):
    P, Q, M, n = 5, 3, 4, 50000
    u, t, theta = _ls_problem(P, Q, M, n, 1)
    f = dpd.DPD(P, Q, M)
    h, st = f.estimate(torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda(), precision=precision, refine_iters=3)
    h = h.cpu().numpy().astype(np.complex128)
    ref = oracle.ls(u, t, P, Q, M)
    e_ref = np.linalg.norm(h - ref) / np.linalg.norm(ref)
    e_true = np.linalg.norm(h - theta) / np.linalg.norm(theta)
    assert e_ref <= tol and e_true <= tol, (precision, e_ref, e_true, st)
    assert st["rel_residual"] < 1e-10 and st["cond_est"] >= 1.0


@pytest.mark.parametrize("P,Q,M", [(5, 3, 4), (9, 9, 4), (11, 11, 7)])
def test_condition_estimate_matches_numpy(P, Q, M):
    """stats["cond_est"] (power iterations on the device Cholesky factor) is the
    2-norm condition number of D G D, D = diag(G)^(-1/2), for the Gram matrix
    of the same precision: compared with numpy's SVD-based cond."""
    u, t, _ = _ls_problem(P, Q, M, 40000, 3)
    f = dpd.DPD(P, Q, M)
    ud, td = torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda()
    _, st = f.estimate(ud, td, precision="tf32x3", refine_iters=0)
    G, _, _ = f.gram(ud, td, precision="tf32x3")
    G = G.cpu().numpy()
    dinv = 1.0 / np.sqrt(np.real(np.diag(G)))
    ref = np.linalg.cond(G * dinv[:, None] * dinv[None, :])
    assert abs(st["cond_est"] - ref) <= 1e-6 * ref, (st["cond_est"], ref)


@pytest.mark.parametrize("P,Q,M", [(1, 0, 0), (7, 3, 1), (7, 7, 3), (9, 7, 6), (7, 7, 7)])
def test_estimate_solve_block_edges(P, Q, M):
    """K = 2, 13, 33, 64, 65: the triangular solves run in blocks of 32 rows, so
    these sizes put the last block at one row, a partial block, a full block
    and one past it; each estimate against numpy's lstsq on the same data, and
    the batched form on two problems against the single one."""
    u, t, _ = _ls_problem(P, Q, M, 30000, 5)
    f = dpd.DPD(P, Q, M)
    ud, td = torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda()
    h, _ = f.estimate(ud, td, precision="tf32x3", refine_iters=3)
    ref = oracle.ls(u, t, P, Q, M)
    e = np.linalg.norm(h.cpu().numpy().astype(np.complex128) - ref) / np.linalg.norm(ref)
    assert e <= 1e-4, (P, Q, M, e)
    hb, info = f.estimate_batched([ud, ud], [td, td], precision="tf32x3", refine_iters=3)
    assert info == [0, 0]
    eb = np.linalg.norm(hb.cpu().numpy().astype(np.complex128) - ref[None, :]) / np.linalg.norm(ref)
    assert eb <= 2e-4, (P, Q, M, eb)


def test_estimate_rejects_singular_gram():
    f = dpd.DPD(5, 5, 2)
    u = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    t = torch.ones(4096, dtype=torch.complex64, device="cuda")
    with pytest.raises(dpd.DPDError) as e:
        f.estimate(u, t, precision="tf32x3")
    assert e.value.code == 6


def test_estimate_batched_matches_single():
    P, Q, M = 7, 7, 3
    probs = [_ls_problem(P, Q, M, 20000 + 17 * i, 70 + i) for i in range(6)]
    f = dpd.DPD(P, Q, M)
    us = [torch.from_numpy(u).cuda() for u, _, _ in probs]
    ts = [torch.from_numpy(t).cuda() for _, t, _ in probs]
    hb, info = f.estimate_batched(us, ts, precision="tf32x3", refine_iters=2)
    assert info == [0] * len(probs)
    for i, (u, t, theta) in enumerate(probs):
        hs, _ = f.estimate(us[i], ts[i], precision="tf32x3", refine_iters=2)
        np.testing.assert_allclose(hb[i].cpu().numpy(), hs.cpu().numpy(), rtol=0, atol=1e-5)
        e = np.linalg.norm(hb[i].cpu().numpy() - theta) / np.linalg.norm(theta)
        assert e < 1e-4, (i, e)


def test_gram_without_host_readback_matches():
    """want_tt=False: same G and g, no host synchronisation inside the call."""
    P, Q, M, n = 9, 9, 4, 30011
    u, t, _ = _ls_problem(P, Q, M, n, seed=5)
    f = dpd.DPD(P, Q, M)
    ud, td = torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda()
    for prec in ("fp32", "tf32x3", "bf16x3"):
        G1, g1, tt1 = f.gram(ud, td, precision=prec)
        G2, g2, tt2 = f.gram(ud, td, precision=prec, want_tt=False)
        torch.cuda.synchronize()
        assert tt2 is None and tt1 > 0
        assert torch.equal(G1, G2) and torch.equal(g1, g2)
    f.close()


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16x3"])
def test_gram_uses_the_basis_of_eq2_whatever_the_estimate_basis(precision):
    """dpd_gram returns the Gram of the monomial basis of Eq. 2 also on a handle
    whose estimates run in the orthogonal basis (set and used first, so that
    its basis matrix exists on the device), against the FP64 oracle."""
    P, Q, M, n = 7, 5, 3, 6007
    u, t, _ = _ls_problem(P, Q, M, n, seed=9)
    f = dpd.DPD(P, Q, M)
    ud, td = torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda()
    f.estimate(ud, td, precision=precision, refine_iters=1, basis="orthogonal")
    G, g, tt = f.gram(ud, td, precision=precision)
    Gr, gr = oracle.gram(u, t, P, Q, M)
    d = np.sqrt(np.abs(np.diag(Gr)))
    err = np.abs(G.cpu().numpy() - Gr) / np.outer(d, d)
    assert err.max() <= GRAM_TOL[precision], err.max()
    f.close()


@pytest.mark.parametrize("basis", ["monomial", "orthogonal"])
def test_estimate_batched_refinement_paths_agree(basis):
    """The batch refined together (16-byte aligned inputs: one launch per
    kernel for all problems) and refined problem by problem (an input that is
    only 8-byte aligned selects that path) give the same coefficients, and both
    match the FP64 oracle's LS solution; problems of different lengths, one
    shorter than a tile."""
    P, Q, M = 9, 9, 4
    lens = [20000, 3001, 65536 + 7, 1500, 40000]
    probs = [_ls_problem(P, Q, M, n, 90 + i) for i, n in enumerate(lens)]
    f = dpd.DPD(P, Q, M)
    us = [torch.from_numpy(u).cuda() for u, _, _ in probs]
    ts = [torch.from_numpy(t).cuda() for _, t, _ in probs]
    h_tog, info = f.estimate_batched(us, ts, precision="tf32x3", refine_iters=2, basis=basis)
    assert info == [0] * len(probs)
    # the same first input at an 8-byte (not 16-byte) aligned address
    buf = torch.zeros(len(probs[0][0]) + 1, dtype=torch.complex64, device="cuda")
    buf[1:] = us[0]
    us_mis = [buf[1:]] + us[1:]
    h_one, info = f.estimate_batched(us_mis, ts, precision="tf32x3", refine_iters=2, basis=basis)
    assert info == [0] * len(probs)
    a, b = h_tog.cpu().numpy().astype(np.complex128), h_one.cpu().numpy().astype(np.complex128)
    # the two paths sum the gradient partials in different orders (one CTA per
    # problem against several): FP32 rounding, amplified by the refinement
    for i in range(len(probs)):
        assert np.linalg.norm(a[i] - b[i]) <= 1e-4 * np.linalg.norm(b[i]), (basis, i)
    for i, (u, t, _) in enumerate(probs):
        ref = oracle.ls(u, t, P, Q, M)
        e = np.linalg.norm(h_tog[i].cpu().numpy().astype(np.complex128) - ref) / np.linalg.norm(ref)
        assert e < 1e-3, (basis, i, e)


@pytest.mark.parametrize("aligned", [True, False])
@pytest.mark.parametrize("n", [1000, 2 * 3072 - 5, 3072 * 152 * 2 + 1237])
def test_estimate_residual_statistic_against_oracle(n, aligned):
    """stats["rel_residual"] = ||t - Psi h||^2 / ||t||^2 for the returned
    coefficients (Sec. 2.2's least-squares residual), with a target that the
    model does not fit exactly (complex Gaussian noise at 0.3 of the signal's
    RMS), against the same ratio from the FP64 oracle filter.  A 16-byte
    aligned input takes the filter pass that sums the squares itself (one
    partial per warp, 3072-sample tiles: n spans one partial tile, two CTAs
    and several tiles per CTA with a ragged end); an 8-byte aligned one the
    filter followed
    by a separate sum.  The ratio uses the FP64 coefficients on the device and
    their FP32 copy here: a difference of order 1e-7 relative to ||Psi h||."""
    P, Q, M = 11, 11, 7
    u, theta = synth.ls_problem(n, P, Q, M, seed=71)
    y = oracle.apply(u, theta, P, Q, M)
    rng = np.random.default_rng([71, 2])
    rms = np.sqrt(np.mean(np.abs(y) ** 2))
    t = (y + 0.3 * rms / np.sqrt(2) * (rng.standard_normal(n) + 1j * rng.standard_normal(n))).astype(np.complex64)
    f = dpd.DPD(P, Q, M)
    ud, td = torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda()
    if not aligned:
        bu = torch.zeros(n + 1, dtype=torch.complex64, device="cuda")
        bt = torch.zeros(n + 1, dtype=torch.complex64, device="cuda")
        bu[1:], bt[1:] = ud, td
        ud, td = bu[1:], bt[1:]
    h, st = f.estimate(ud, td, precision="tf32x3", refine_iters=1)
    hc = h.cpu().numpy().astype(np.complex128)
    e = t.astype(np.complex128) - oracle.apply(u, hc, P, Q, M)
    ref = np.sum(np.abs(e) ** 2) / np.sum(np.abs(t.astype(np.complex128)) ** 2)
    assert ref > 1e-3
    assert abs(st["rel_residual"] - ref) <= 1e-4 * ref, (st["rel_residual"], ref)
    f.close()


def test_estimate_batched_accepts_a_2d_batch():
    """Equal-length problems as two 2-D tensors (problems x samples) and as the
    lists of their rows reach the library at the same device addresses: the
    estimates agree bit for bit, each matches the FP64 oracle's LS solution
    (Sec. 2.2), and a t shorter than its u is refused."""
    P, Q, M, n = 5, 3, 4, 4000
    probs = [_ls_problem(P, Q, M, n, 200 + i) for i in range(4)]
    U = torch.stack([torch.from_numpy(u) for u, _, _ in probs]).cuda()
    T = torch.stack([torch.from_numpy(t) for _, t, _ in probs]).cuda()
    f = dpd.DPD(P, Q, M)
    h2, info2 = f.estimate_batched(U, T, precision="tf32x3", refine_iters=2)
    hl, infol = f.estimate_batched(list(U), list(T), precision="tf32x3", refine_iters=2)
    assert info2 == infol == [0] * len(probs)
    assert torch.equal(h2, hl)
    for i, (u, t, _) in enumerate(probs):
        ref = oracle.ls(u, t, P, Q, M)
        e = np.linalg.norm(h2[i].cpu().numpy().astype(np.complex128) - ref) / np.linalg.norm(ref)
        assert e <= 1e-4, (i, e)
    with pytest.raises(ValueError):
        f.estimate_batched([U[0]], [T[0][:-1]])
    f.close()
