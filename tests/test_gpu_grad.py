"""GPU parity of dpd_grad (the hand-written adjoint) against the FP64 oracle's
gradient (itself pinned by central finite differences), plus the gradient
convention checked against torch's own CPU autograd of a plain float64
restatement of Eq. 1."""
import numpy as np
import pytest

import dpd_synth as synth
import oracle
from util import assert_parity, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1612_09001_gb300 as dpd  # noqa: E402
from paper_1612_09001_gb300.autograd import DPDFunction  # noqa: E402


def gpu_grad(x, h, gy, P, Q, M, want_h=True, want_x=True, launch=None):
    f = dpd.DPD(P, Q, M)
    if launch:
        f.set_adj_launch(*launch)
    f.set_coeffs(torch.from_numpy(h).cuda())
    xd = torch.from_numpy(x).cuda()
    gyd = torch.from_numpy(gy).cuda()
    gh = torch.full((f.K,), complex(5, 5), dtype=torch.complex64, device="cuda") if want_h else None
    gx = torch.full_like(xd, complex(5, 5)) if want_x else None
    f.grad(xd, gyd, gh=gh, gx=gx)
    f.sync_status()
    f.close()
    return (gh.cpu().numpy() if want_h else None), (gx.cpu().numpy() if want_x else None)


def check_gh(gh, x, h, gy, P, Q, M, tol=1e-5):
    """Element-wise: |gh - ref|_j <= tol * sum_n |Psi_{n,j}| |gy_n| (the size of the
    terms the FP32 sum adds), plus the plain normwise bound."""
    ref, _ = oracle.grad(x, h, gy, P, Q, M, want_x=False)
    scale, _ = oracle.grad(np.abs(x).astype(np.complex128), h, np.abs(gy).astype(np.complex128), P, Q, M,
                           want_x=False)
    scale = np.abs(scale)
    err = np.abs(gh.astype(np.complex128) - ref)
    bad = np.nonzero(err > tol * scale + 1e-30)[0]
    assert bad.size == 0, f"gh elements {bad[:5]} err {err[bad[:5]]} scale {scale[bad[:5]]}"
    assert rel_err(gh, ref) <= tol, rel_err(gh, ref)


def make(P, Q, M, n, seed):
    x = synth.clipped_gaussian(n, 0.4, key=(20, seed, 0))
    h = synth.coeffs(P, Q, M, key=(20, seed, 1), f_std=0.3, g_std=0.2)
    g = np.random.default_rng([20, seed, 2])
    gy = (g.standard_normal(n) + 1j * g.standard_normal(n)).astype(np.complex64)
    return x, h, gy


MODELS = [(5, 3, 4), (7, 7, 3), (9, 9, 4), (11, 11, 7), (1, 0, 0), (1, 1, 2), (3, 0, 2), (0, 5, 2), (3, 9, 1),
          (7, 0, 3), (11, 1, 5)]


@pytest.mark.parametrize("P,Q,M", MODELS)
def test_grad_parity(P, Q, M):
    x, h, gy = make(P, Q, M, 50021, P * 100 + Q * 10 + M)
    gh, gx = gpu_grad(x, h, gy, P, Q, M)
    _, gx_ref = oracle.grad(x, h, gy, P, Q, M, want_h=False)
    assert_parity(gx, gx_ref, what=f"gx P={P} Q={Q} M={M}")
    check_gh(gh, x, h, gy, P, Q, M)


@pytest.mark.parametrize("n", [1, 2, 5, 1023, 1024, 1025, 4097, 300001])
@pytest.mark.parametrize("launch", [None, (1, 1), (3, 4), (37, 2), (600, 1), (5, 3), (150, 5)])
def test_grad_sizes_and_tap_schedules(n, launch):
    P, Q, M = 7, 5, 6
    x, h, gy = make(P, Q, M, n, n)
    gh, gx = gpu_grad(x, h, gy, P, Q, M, launch=launch)
    _, gx_ref = oracle.grad(x, h, gy, P, Q, M, want_h=False)
    assert_parity(gx, gx_ref, what=f"gx n={n}")
    check_gh(gh, x, h, gy, P, Q, M)


@pytest.mark.parametrize("n", [1, 9, 1031, 2 * 1024 + 9, 20011])
@pytest.mark.parametrize("shift", [(0, 0, 1), (1, 0, 0), (0, 1, 0), (1, 1, 1)])
def test_grad_alignment_paths(n, shift):
    """16-byte aligned x and gy take the staged (bulk-copy ring) kernels, any
    other 8-byte alignment the plain-load kernels; gx may be 8-byte aligned in
    both.  Sizes straddle the 1024-sample tile and its 8-sample look-ahead."""
    P, Q, M = 9, 7, 5
    x, h, gy = make(P, Q, M, n, 7 * n + sum(shift))
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(torch.from_numpy(h).cuda())

    def placed(a, off):
        buf = torch.zeros(len(a) + 1, dtype=torch.complex64, device="cuda")
        v = buf[off:off + len(a)]
        v.copy_(torch.from_numpy(a).cuda())
        return v

    xd, gyd = placed(x, shift[0]), placed(gy, shift[1])
    gx = placed(np.full(n, 5 + 5j, np.complex64), shift[2])
    gh = torch.full((f.K,), complex(5, 5), dtype=torch.complex64, device="cuda")
    f.grad(xd, gyd, gh=gh, gx=gx)
    f.sync_status()
    _, gx_ref = oracle.grad(x, h, gy, P, Q, M, want_h=False)
    assert_parity(gx.cpu().numpy(), gx_ref, what=f"gx n={n} shift={shift}")
    check_gh(gh.cpu().numpy(), x, h, gy, P, Q, M)


@pytest.mark.parametrize("P,Q,M", [(9, 9, 4), (7, 0, 3), (1, 1, 0), (11, 11, 7), (3, 5, 2)])
@pytest.mark.parametrize("n", [4099, 70001])
def test_grad_host_coefficients_param_bank(P, Q, M, n):
    """Coefficients set from host memory: the input gradient takes them from the
    kernel parameter bank (device-set ones from shared memory); both against
    the oracle."""
    x, h, gy = make(P, Q, M, n, 31 * P + M + n)
    xd, gyd = torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda()
    _, gx_ref = oracle.grad(x, h, gy, P, Q, M, want_h=False)
    for src in (h, torch.from_numpy(h).cuda()):
        f = dpd.DPD(P, Q, M)
        f.set_coeffs(src)
        gx = torch.empty_like(xd)
        gh = torch.empty(f.K, dtype=torch.complex64, device="cuda")
        f.grad(xd, gyd, gh=gh, gx=gx)
        f.sync_status()
        f.close()
        assert_parity(gx.cpu().numpy(), gx_ref, what=f"gx P={P} Q={Q} M={M} host={not torch.is_tensor(src)}")
        check_gh(gh.cpu().numpy(), x, h, gy, P, Q, M)


@pytest.mark.parametrize("P,Q,M", [(9, 9, 4), (7, 7, 3)])
def test_grad_full_size_2p24(P, Q, M):
    """Both gradients on the 2^24-sample OFDM signal with an OFDM output
    gradient and host-set coefficients: the adjoint benchmark's workload and
    launch path."""
    n = 1 << 24
    x = synth.ofdm2(n, key=(0, 0))
    gy = synth.ofdm2(n, key=(0, 1))
    h = synth.coeffs(P, Q, M, key=(0, 1))
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(h)
    xd, gyd = torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda()
    gx = torch.empty_like(xd)
    gh = torch.empty(f.K, dtype=torch.complex64, device="cuda")
    f.grad(xd, gyd, gh=gh, gx=gx)
    f.sync_status()
    f.close()
    _, gx_ref = oracle.grad(x, h, gy, P, Q, M, want_h=False)
    assert_parity(gx.cpu().numpy(), gx_ref, what=f"gx 2^24 P={P} M={M}")
    check_gh(gh.cpu().numpy(), x, h, gy, P, Q, M)


def test_adj_launch_limits():
    f = dpd.DPD(5, 5, 2)
    for bad in [(0, 2), (1, 0), (1, 6), (10 ** 6, 2)]:
        with pytest.raises(dpd.DPDError):
            f.set_adj_launch(*bad)
    f.set_adj_launch(1, 5)
    f.close()


def test_grad_only_h_or_only_x_and_no_coeffs_for_h():
    P, Q, M = 5, 5, 2
    x, h, gy = make(P, Q, M, 7777, 1)
    gh, _ = gpu_grad(x, h, gy, P, Q, M, want_x=False)
    check_gh(gh, x, h, gy, P, Q, M)
    _, gx = gpu_grad(x, h, gy, P, Q, M, want_h=False)
    assert_parity(gx, oracle.grad(x, h, gy, P, Q, M, want_h=False)[1])
    # the coefficient gradient does not depend on h, so it needs no coefficients
    f = dpd.DPD(P, Q, M)
    ghd = torch.empty(f.K, dtype=torch.complex64, device="cuda")
    f.grad(torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda(), gh=ghd)
    f.sync_status()
    check_gh(ghd.cpu().numpy(), x, h, gy, P, Q, M)
    with pytest.raises(dpd.DPDError):
        f.grad(torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda(),
               gx=torch.empty(len(x), dtype=torch.complex64, device="cuda"))


def test_grad_empty_zeroes_gh():
    f = dpd.DPD(3, 3, 1)
    gh = torch.full((f.K,), 3 + 3j, dtype=torch.complex64, device="cuda")
    e = torch.empty(0, dtype=torch.complex64, device="cuda")
    f.grad(e, e, gh=gh)
    f.sync_status()
    assert torch.all(gh == 0)


def test_grad_deterministic():
    P, Q, M = 9, 9, 4
    x, h, gy = make(P, Q, M, 1 << 20, 99)
    a, ax = gpu_grad(x, h, gy, P, Q, M)
    b, bx = gpu_grad(x, h, gy, P, Q, M)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    assert np.array_equal(ax.view(np.uint64), bx.view(np.uint64))


def _torch_dpd(x, h, P, Q, M):
    """Eq. 1 in plain torch float64 ops (for autograd's own derivative)."""
    L = M + 1
    n = x.shape[0]
    bp = (P + 1) // 2 if P else 0
    bq = (Q + 1) // 2 if Q else 0
    y = torch.zeros(n, dtype=x.dtype) + h[-1]
    r = (x.real ** 2 + x.imag ** 2)
    for b in range(bp):
        psi = r ** b * x
        for k in range(L):
            y = y + torch.cat([torch.zeros(k, dtype=x.dtype), h[b * L + k] * psi[: n - k]])
    for b in range(bq):
        psi = r ** b * torch.conj(x)
        for k in range(L):
            y = y + torch.cat([torch.zeros(k, dtype=x.dtype), h[(bp + b) * L + k] * psi[: n - k]])
    return y


@pytest.mark.parametrize("P,Q,M", [(5, 3, 2), (7, 7, 3), (1, 0, 0)])
def test_autograd_function_matches_torch_autograd(P, Q, M):
    n = 3000
    x, h, _ = make(P, Q, M, n, 7)
    t = synth.ofdm2(n, key=(21, 0))
    # loss = sum |y - t|^2 (a real loss, as in direct learning)
    xc = torch.from_numpy(x.astype(np.complex128)).requires_grad_(True)
    hc = torch.from_numpy(h.astype(np.complex128)).requires_grad_(True)
    yc = _torch_dpd(xc, hc, P, Q, M)
    (yc - torch.from_numpy(t.astype(np.complex128))).abs().pow(2).sum().backward()

    f = dpd.DPD(P, Q, M)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    hd = torch.from_numpy(h).cuda().requires_grad_(True)
    yd = DPDFunction.apply(xd, hd, f)
    (yd - torch.from_numpy(t).cuda()).abs().pow(2).sum().backward()
    f.sync_status()
    assert rel_err(yd.detach().cpu().numpy(), yc.detach().numpy()) < 1e-5
    assert rel_err(xd.grad.cpu().numpy(), xc.grad.numpy()) < 1e-5
    assert rel_err(hd.grad.cpu().numpy(), hc.grad.numpy()) < 1e-5


def test_device_set_coefficients_use_the_same_tables():
    """Coefficients set from device memory: the tables are copied back behind
    the set; gradients before the copy has landed (tables read on the device)
    and after (tables passed by value) are bitwise equal, and equal to those of
    the same coefficients set from host memory."""
    P, Q, M = 9, 9, 4
    n = 100003
    x = torch.from_numpy(synth.ofdm2(n, key=(95, 0))).cuda()
    gy = torch.from_numpy(synth.ofdm2(n, key=(95, 1))).cuda()
    h = synth.coeffs(P, Q, M, key=(95, 2)).astype(np.complex64)
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(torch.from_numpy(h).cuda())
    gh0 = torch.empty(f.K, dtype=torch.complex64, device="cuda")
    gx0 = torch.empty_like(x)
    f.grad(x, gy, gh=gh0, gx=gx0)          # queued right behind the set
    torch.cuda.synchronize()
    gh1 = torch.empty_like(gh0)
    gx1 = torch.empty_like(x)
    f.grad(x, gy, gh=gh1, gx=gx1)          # the copy back has landed
    f.sync_status()
    g = dpd.DPD(P, Q, M)
    g.set_coeffs(h)                        # host memory
    gh2 = torch.empty_like(gh0)
    gx2 = torch.empty_like(x)
    g.grad(x, gy, gh=gh2, gx=gx2)
    g.sync_status()
    for a, b in ((gx0, gx1), (gx1, gx2), (gh0, gh1), (gh1, gh2)):
        assert torch.equal(a, b)
    f.close()
    g.close()
