"""The allocation-free coefficient-gradient entry point (dpd_grad_coeffs_noalloc).

It serves callers that may not allocate device memory, so it runs without a
handle and keeps its scratch in a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test.  Each check calls the entry point twice in a row (a large
problem, then a smaller one, so stale rows from the first call would show) and
compares with dpd_grad's coefficient gradient on the same inputs; one case is
also compared with the FP64 oracle's gradient directly, two calls of different
models are queued on one stream before a single synchronisation, and a warmed-up
call is checked to leave the device's free memory unchanged."""
import ctypes

import numpy as np
import pytest

import dpd_synth as synth
import oracle
from util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1612_09001_gb300 as dpd  # noqa: E402
from paper_1612_09001_gb300 import _lib  # noqa: E402


def _inputs(n, seed):
    x = torch.from_numpy(synth.clipped_gaussian(n, 0.4, key=(30, seed, 0))).cuda()
    g = np.random.default_rng([30, seed, 1])
    gy = torch.from_numpy((g.standard_normal(n) + 1j * g.standard_normal(n)).astype(np.complex64)).cuda()
    return x, gy


def _call(P, Q, M, x, gy, gh):
    """Queue one call on the current stream (no synchronisation)."""
    lib = _lib.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.dpd_grad_coeffs_noalloc(P, Q, M, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(gy.data_ptr()),
                                     x.numel(), ctypes.c_void_p(gh.data_ptr()), s)
    assert rc == 0, _lib.STATUS.get(rc, rc)


def _noalloc(P, Q, M, x, gy, K):
    gh = torch.full((K,), complex(9, 9), dtype=torch.complex64, device="cuda")
    _call(P, Q, M, x, gy, gh)
    torch.cuda.synchronize()
    return gh.cpu().numpy()


def _oracle_gh(P, Q, M, x, gy):
    """The FP64 oracle's coefficient gradient (gh does not depend on the
    coefficients, so any K values serve) and the element scale
    sum_n |Psi_nj| |gy_n| that an FP32 sum of its terms is measured against."""
    xs, gys = x.cpu().numpy(), gy.cpu().numpy()
    h = np.zeros(dpd.num_coeffs(P, Q, M), np.complex128)
    ref, _ = oracle.grad(xs, h, gys, P, Q, M, want_x=False)
    scale, _ = oracle.grad(np.abs(xs).astype(np.complex128), h, np.abs(gys).astype(np.complex128), P, Q, M,
                           want_x=False)
    return ref, np.abs(scale)


def _check_against_oracle(got, P, Q, M, x, gy, tol=1e-5):
    ref, scale = _oracle_gh(P, Q, M, x, gy)
    err = np.abs(got.astype(np.complex128) - ref)
    bad = np.nonzero(err > tol * scale + 1e-30)[0]
    assert bad.size == 0, (P, Q, M, bad[:5], err[bad[:5]], scale[bad[:5]])
    assert rel_err(got, ref) <= tol, (P, Q, M, rel_err(got, ref))


def _with_handle(P, Q, M, x, gy):
    f = dpd.DPD(P, Q, M)
    gh = torch.empty(f.K, dtype=torch.complex64, device="cuda")
    f.grad(x, gy, gh=gh)
    f.sync_status()
    f.close()
    return gh.cpu().numpy()


@pytest.mark.parametrize("P,Q,M", [(9, 9, 4), (11, 11, 7), (5, 3, 4), (1, 0, 0)])
def test_noalloc_matches_dpd_grad_twice(P, Q, M):
    K = dpd.num_coeffs(P, Q, M)
    for n, seed in ((1 << 20, 1), (3001, 2)):
        x, gy = _inputs(n, seed)
        got = _noalloc(P, Q, M, x, gy, K)
        ref = _with_handle(P, Q, M, x, gy)
        assert rel_err(got, ref) <= 1e-5, (P, Q, M, n, rel_err(got, ref))


def test_noalloc_rejects_bad_arguments():
    lib = _lib.load()
    x, gy = _inputs(100, 3)
    gh = torch.empty(51, dtype=torch.complex64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = lambda t, off=0: ctypes.c_void_p(t.data_ptr() + off)
    assert lib.dpd_grad_coeffs_noalloc(8, 9, 4, vp(x), vp(gy), 100, vp(gh), s) == 2     # even order
    assert lib.dpd_grad_coeffs_noalloc(9, 9, 8, vp(x), vp(gy), 100, vp(gh), s) == 2     # 9 taps
    assert lib.dpd_grad_coeffs_noalloc(-1, 9, 4, vp(x), vp(gy), 100, vp(gh), s) == 1    # negative order
    assert lib.dpd_grad_coeffs_noalloc(9, 9, 4, vp(x, 4), vp(gy), 100, vp(gh), s) == 1  # misaligned
    assert lib.dpd_grad_coeffs_noalloc(9, 9, 4, vp(x), vp(gy), 100, vp(x), s) == 1      # gh overlaps x
    empty = torch.empty(0, dtype=torch.complex64, device="cuda")
    gh.fill_(1)
    assert lib.dpd_grad_coeffs_noalloc(9, 9, 4, vp(empty), vp(empty), 0, vp(gh), s) == 0
    torch.cuda.synchronize()
    assert torch.all(gh == 0)


def test_noalloc_matches_oracle_twice():
    """Directly against the FP64 oracle, at the same element-wise bound as
    dpd_grad's own parity tests, on two calls in a row."""
    P, Q, M = 9, 9, 4
    K = dpd.num_coeffs(P, Q, M)
    for n, seed in ((1 << 18, 4), (4099, 5)):
        x, gy = _inputs(n, seed)
        _check_against_oracle(_noalloc(P, Q, M, x, gy, K), P, Q, M, x, gy)


def test_noalloc_two_models_queued_on_one_stream():
    """Calls on one stream run in order, so two calls with different models
    (different K, different partial rows) queued before one synchronisation
    each give their own result."""
    x1, gy1 = _inputs(1 << 19, 6)
    x2, gy2 = _inputs(70001, 7)
    m1, m2 = (11, 11, 7), (5, 3, 2)
    gh1 = torch.full((dpd.num_coeffs(*m1),), complex(9, 9), dtype=torch.complex64, device="cuda")
    gh2 = torch.full((dpd.num_coeffs(*m2),), complex(9, 9), dtype=torch.complex64, device="cuda")
    _call(*m1, x1, gy1, gh1)
    _call(*m2, x2, gy2, gh2)
    torch.cuda.synchronize()
    _check_against_oracle(gh1.cpu().numpy(), *m1, x1, gy1)
    _check_against_oracle(gh2.cpu().numpy(), *m2, x2, gy2)


def test_noalloc_call_leaves_free_memory_unchanged():
    """After a first call of the same model (which loads the kernels), a call
    changes the device's free memory by nothing."""
    P, Q, M = 7, 7, 3
    K = dpd.num_coeffs(P, Q, M)
    x, gy = _inputs(1 << 20, 8)
    gh = torch.empty(K, dtype=torch.complex64, device="cuda")
    _call(P, Q, M, x, gy, gh)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _call(P, Q, M, x, gy, gh)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    _check_against_oracle(gh.cpu().numpy(), P, Q, M, x, gy)
