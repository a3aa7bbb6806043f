"""The allocation-free coefficient-gradient entry point (dpd_grad_coeffs_noalloc).

It serves callers that may not allocate device memory, so it runs without a
handle and keeps its scratch in a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test.  Each check calls the entry point twice in a row (a large
problem, then a smaller one, so stale rows from the first call would show) and
compares with dpd_grad's coefficient gradient on the same inputs."""
import ctypes

import numpy as np
import pytest

import dpd_synth as synth
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


def _noalloc(P, Q, M, x, gy, K):
    lib = _lib.load()
    gh = torch.full((K,), complex(9, 9), dtype=torch.complex64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.dpd_grad_coeffs_noalloc(P, Q, M, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(gy.data_ptr()),
                                     x.numel(), ctypes.c_void_p(gh.data_ptr()), s)
    assert rc == 0, _lib.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    return gh.cpu().numpy()


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
    assert lib.dpd_grad_coeffs_noalloc(8, 9, 4, vp(x), vp(gy), 100, vp(gh), s) == 1     # even order
    assert lib.dpd_grad_coeffs_noalloc(9, 9, 8, vp(x), vp(gy), 100, vp(gh), s) == 1     # 9 taps
    assert lib.dpd_grad_coeffs_noalloc(9, 9, 4, vp(x, 4), vp(gy), 100, vp(gh), s) == 1  # misaligned
    assert lib.dpd_grad_coeffs_noalloc(9, 9, 4, vp(x), vp(gy), 100, vp(x), s) == 1      # gh overlaps x
    empty = torch.empty(0, dtype=torch.complex64, device="cuda")
    gh.fill_(1)
    assert lib.dpd_grad_coeffs_noalloc(9, 9, 4, vp(empty), vp(empty), 0, vp(gh), s) == 0
    torch.cuda.synchronize()
    assert torch.all(gh == 0)
