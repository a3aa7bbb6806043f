"""GPU parity of dpd_apply (Eq. 1 / Algorithm 1) against the FP64 oracle.

Every case runs the CUDA path through the C ABI (paper_1612_09001_gb300.DPD)
and the oracle on the same seeded complex64 inputs, and compares element by
element (normwise relative error and max element error <= 1e-5)."""
import ctypes

import numpy as np
import pytest

import dpd_synth as synth
import oracle
from util import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1612_09001_gb300 as dpd  # noqa: E402
from paper_1612_09001_gb300 import _lib  # noqa: E402


def run_gpu(x, h, P, Q, M, launch=None, offset=0, out_offset=0, host_coeffs=False):
    f = dpd.DPD(P, Q, M)
    if launch:
        f.set_fwd_launch(**launch)
    f.set_coeffs(h if host_coeffs else torch.from_numpy(h).cuda())
    n = len(x)
    xb = torch.zeros(n + offset + 2, dtype=torch.complex64, device="cuda")
    xb[offset: offset + n] = torch.from_numpy(x).cuda()
    yb = torch.full((n + out_offset + 2,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    xv = xb[offset: offset + n]
    yv = yb[out_offset: out_offset + n]
    f.apply(xv, out=yv)
    f.sync_status()
    yb = yb.cpu().numpy()
    # guard elements around the output must be untouched
    assert np.all(yb[:out_offset] == np.complex64(7 - 7j))
    assert np.all(yb[out_offset + n:] == np.complex64(7 - 7j))
    f.close()
    return yb[out_offset: out_offset + n]


def test_config0_clipped_gaussian_p5_m2():
    x = synth.clipped_gaussian(1 << 16, 0.3, key=(0, 0))
    h = synth.coeffs(5, 5, 2, key=(0, 1))
    assert_parity(run_gpu(x, h, 5, 5, 2), oracle.apply(x, h, 5, 5, 2), what="config 0")


def test_table2_p5_q3_l5_ragged():
    x = synth.ofdm2(100003, key=(1, 0))
    h = synth.coeffs(5, 3, 4, key=(1, 1))
    assert_parity(run_gpu(x, h, 5, 3, 4), oracle.apply(x, h, 5, 3, 4), what="table 2")


@pytest.mark.parametrize("launch", [None, dict(mode=3, V=8, warps=12, stages=3, group=0),
                                    dict(mode=3, V=8, warps=12, stages=4, group=4),
                                    dict(mode=3, V=8, warps=16, stages=3, group=2),
                                    dict(mode=3, V=6, warps=16, stages=4, group=4),
                                    dict(mode=3, V=6, warps=12, stages=3, group=0)],
                         ids=["default", "one_group", "w12g4", "w16g2", "v6w16g4", "v6w12"])
def test_config1_full_size_ofdm_p9_m4(launch):
    """Full 2^24-sample OFDM workload, coefficients from host memory as the
    benchmark installs them, at the default shape (16 consumer warps in groups
    of 4) and at other shapes the autotuner chooses from (parameter-bank packed
    FMAs, V 8)."""
    n = 1 << 24
    x = synth.ofdm2(n, key=(0, 0))
    h = synth.coeffs(9, 9, 4, key=(0, 1))
    y = run_gpu(x, h, 9, 9, 4, launch=launch, host_coeffs=True)
    assert_parity(y, oracle.apply(x, h, 9, 9, 4), what="config 1")


MODELS = [(P, Q, M) for P in (0, 1, 3, 5, 7, 9, 11) for Q in (0, 1, 3, 5, 7, 9, 11)
          for M in (0, 3, 7) if P + Q > 0]


@pytest.mark.parametrize("P,Q,M", MODELS)
def test_model_sweep(P, Q, M):
    n = 3001 + 17 * M
    x = synth.clipped_gaussian(n, 0.5, key=(2, P, Q, M))
    h = synth.coeffs(P, Q, M, key=(2, P, Q, M, 1), f_std=0.3, g_std=0.3)
    assert_parity(run_gpu(x, h, P, Q, M), oracle.apply(x, h, P, Q, M), what=f"P={P} Q={Q} M={M}")


@pytest.mark.parametrize("M", range(8))
def test_every_memory_depth(M):
    x = synth.clipped_gaussian(5000, 0.4, key=(3, M))
    h = synth.coeffs(7, 5, M, key=(3, M, 1), f_std=0.3, g_std=0.3)
    assert_parity(run_gpu(x, h, 7, 5, M), oracle.apply(x, h, 7, 5, M), what=f"M={M}")


LAUNCHES = [
    dict(V=4, warps=8, stages=4, ctas_per_sm=0, use_tma=1),
    dict(V=2, warps=8, stages=4, ctas_per_sm=0, use_tma=1),
    dict(V=4, warps=1, stages=2, ctas_per_sm=1, use_tma=1),
    dict(V=2, warps=16, stages=8, ctas_per_sm=0, use_tma=1),
    dict(V=4, warps=4, stages=3, ctas_per_sm=2, use_tma=1),
    dict(V=4, warps=8, stages=4, ctas_per_sm=0, use_tma=0),
    dict(V=2, warps=8, stages=4, ctas_per_sm=0, use_tma=0),
    dict(V=8, warps=12, stages=4, ctas_per_sm=0, use_tma=1, group=4),
    dict(V=8, warps=12, stages=3, ctas_per_sm=0, use_tma=1, group=1),
    dict(V=4, warps=16, stages=3, ctas_per_sm=0, use_tma=1, group=4),
    dict(V=2, warps=16, stages=8, ctas_per_sm=0, use_tma=1, group=2),
    dict(V=8, warps=6, stages=2, ctas_per_sm=3, use_tma=1, group=3),
    dict(V=6, warps=16, stages=4, ctas_per_sm=0, use_tma=1, group=4, mode=3),
    dict(V=6, warps=5, stages=3, ctas_per_sm=2, use_tma=1, mode=3),
]


@pytest.mark.parametrize("launch", LAUNCHES,
                         ids=lambda d: "V{V}w{warps}s{stages}c{ctas_per_sm}t{use_tma}g{g}".format(g=d.get("group", 0), **d))
@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 9, 255, 256, 257, 1023, 1024, 1025, 2047, 4100, 70001])
def test_sizes_and_launch_shapes(launch, n):
    P, Q, M = 9, 9, 4
    x = synth.clipped_gaussian(n, 0.5, key=(4, n))
    h = synth.coeffs(P, Q, M, key=(4, 1), f_std=0.3, g_std=0.3)
    assert_parity(run_gpu(x, h, P, Q, M, launch=launch), oracle.apply(x, h, P, Q, M), what=f"n={n} {launch}")


@pytest.mark.parametrize("P,Q,M", [(9, 9, 4), (5, 5, 2), (7, 7, 3), (11, 11, 7), (9, 3, 4)])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("V", [4, 8])
@pytest.mark.parametrize("use_tma", [1, 0])
@pytest.mark.parametrize("host_coeffs", [True, False])
def test_compute_modes(P, Q, M, mode, V, use_tma, host_coeffs):
    """Parameter-bank / shared-memory coefficients and scalar / packed FMAs."""
    for n in (1, 1000, 65537):
        x = synth.clipped_gaussian(n, 0.5, key=(8, n, M))
        h = synth.coeffs(P, Q, M, key=(8, 1), f_std=0.3, g_std=0.3)
        launch = dict(mode=mode, V=V, warps=8, stages=4, ctas_per_sm=0, use_tma=use_tma)
        y = run_gpu(x, h, P, Q, M, launch=launch, host_coeffs=host_coeffs)
        assert_parity(y, oracle.apply(x, h, P, Q, M), what=f"n={n} {launch}")


@pytest.mark.parametrize("P,Q,M", [(9, 9, 4), (5, 5, 2), (7, 7, 3), (11, 11, 7)])
@pytest.mark.parametrize("warps,group,stages", [(16, 4, 4), (12, 3, 3), (12, 2, 4), (16, 8, 4), (16, 2, 3)])
def test_grouped_shapes(P, Q, M, warps, group, stages):
    """The grouped ring at the shapes the library builds with compile-time
    tile arithmetic (16/4/4, 12/3/3, 12/2/4, 16/8/4 for the benchmarked models) and a
    runtime one (16/2/3), with parameter-bank coefficients (mode 3), on sizes
    that end inside a group's sub-tile, on a group boundary and past one."""
    h = synth.coeffs(P, Q, M, key=(9, 1), f_std=0.3, g_std=0.3)
    S = warps * 32 * 8
    for n in (1, 77, S // 2 + 3, S, S + 8 * 32 * group + 1, 5 * S - 1, (1 << 20) + 3):
        x = synth.clipped_gaussian(n, 0.5, key=(9, n, P))
        launch = dict(mode=3, V=8, warps=warps, stages=stages, ctas_per_sm=0, use_tma=1, group=group)
        y = run_gpu(x, h, P, Q, M, launch=launch, host_coeffs=True)
        assert_parity(y, oracle.apply(x, h, P, Q, M), what=f"n={n} {launch}")


@pytest.mark.parametrize("P,Q,M", [(1, 1, 0), (3, 1, 1), (5, 5, 2), (7, 7, 3), (9, 9, 4), (11, 3, 5), (11, 11, 7), (0, 7, 6)])
def test_six_samples_per_thread(P, Q, M):
    """V = 6 (packed FMAs, parameter-bank or shared-memory coefficients):
    every order and tap count, sizes that end inside a thread's six samples."""
    h = synth.coeffs(P, Q, M, key=(10, 1), f_std=0.3, g_std=0.3)
    for n in (1, 5, 6, 7, 191, 193, 3 * 1024 + 5, 100003):
        x = synth.clipped_gaussian(n, 0.5, key=(10, n, P, M))
        for host in (True, False):
            launch = dict(mode=3, V=6, warps=8, stages=3, ctas_per_sm=0, use_tma=1, group=2)
            y = run_gpu(x, h, P, Q, M, launch=launch, host_coeffs=host)
            assert_parity(y, oracle.apply(x, h, P, Q, M), what=f"n={n} host={host} {launch}")


@pytest.mark.parametrize("offset,out_offset", [(1, 0), (0, 1), (1, 1), (3, 2)])
def test_eight_byte_aligned_buffers(offset, out_offset):
    x = synth.clipped_gaussian(9999, 0.4, key=(5, offset))
    h = synth.coeffs(5, 5, 2, key=(5, 1))
    y = run_gpu(x, h, 5, 5, 2, offset=offset, out_offset=out_offset)
    assert_parity(y, oracle.apply(x, h, 5, 5, 2), what=f"offsets {offset},{out_offset}")


def test_identity_is_bitwise():
    x = synth.clipped_gaussian(123457, 0.3, key=(6, 0))
    for P, Q, M in [(5, 5, 2), (9, 9, 4), (11, 11, 7), (1, 0, 0)]:
        h = np.zeros(dpd.num_coeffs(P, Q, M), np.complex64)
        h[0] = 1
        y = run_gpu(x, h, P, Q, M)
        assert np.array_equal(y.view(np.uint64), x.view(np.uint64)), (P, Q, M)


def test_empty_input_launches_nothing():
    f = dpd.DPD(5, 5, 2)
    f.set_coeffs(synth.coeffs(5, 5, 2))
    torch.cuda.synchronize()
    before = dpd.kernel_launches()
    x = torch.empty(0, dtype=torch.complex64, device="cuda")
    y = f.apply(x)
    assert y.numel() == 0 and dpd.kernel_launches() == before
    f.sync_status()


def test_host_side_errors_with_device():
    lib = _lib.load()
    f = dpd.DPD(5, 5, 2)
    x = torch.zeros(100, dtype=torch.complex64, device="cuda")
    y = torch.zeros(100, dtype=torch.complex64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # before coefficients are set
    assert lib.dpd_apply(f.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 100, s) == 3
    f.set_coeffs(synth.coeffs(5, 5, 2))
    # overlapping and in-place ranges
    assert lib.dpd_apply(f.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 100, s) == 1
    assert lib.dpd_apply(f.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr() + 8 * 50), 100, s) == 1
    # misaligned (4-byte) pointer, negative length, wrong coefficient count
    assert lib.dpd_apply(f.handle, ctypes.c_void_p(x.data_ptr() + 4), ctypes.c_void_p(y.data_ptr()), 10, s) == 1
    assert lib.dpd_apply(f.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), -1, s) == 1
    h = torch.zeros(18, dtype=torch.complex64)
    assert lib.dpd_set_coeffs(f.handle, ctypes.c_void_p(h.data_ptr()), 18, 0, s) == 1
    assert lib.dpd_set_fwd_launch(f.handle, 0, 3, 8, 4, 0, 1, 0) == 1
    assert lib.dpd_set_fwd_launch(f.handle, 0, 4, 8, 9, 0, 1, 0) == 1
    assert lib.dpd_set_fwd_launch(f.handle, 4, 4, 8, 4, 0, 1, 0) == 1
    assert lib.dpd_set_fwd_launch(f.handle, 3, 8, 12, 4, 0, 1, 5) == 1    # group does not divide warps
    assert lib.dpd_set_fwd_launch(f.handle, 3, 8, 17, 4, 0, 1, 0) == 1    # more than 16 warps
    assert lib.dpd_set_fwd_launch(f.handle, 3, 8, 16, 8, 0, 1, 1) == 2    # rings larger than shared memory
    f.sync_status()


def test_device_coefficients_and_graph_replay():
    P, Q, M = 7, 7, 3
    n = 200000
    x = synth.clipped_gaussian(n, 0.3, key=(7, 0))
    h1 = synth.coeffs(P, Q, M, key=(7, 1))
    h2 = synth.coeffs(P, Q, M, key=(7, 2), f_std=0.1)
    f = dpd.DPD(P, Q, M)
    hd = torch.from_numpy(h1).cuda()
    f.set_coeffs(hd)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        f.apply(xd, out=yd)        # warm up outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        f.set_coeffs(hd)
        f.apply(xd, out=yd)
    g.replay()
    torch.cuda.synchronize()
    assert_parity(yd.cpu().numpy(), oracle.apply(x, h1, P, Q, M), what="graph h1")
    hd.copy_(torch.from_numpy(h2).cuda())   # the graph re-reads the device coefficients
    g.replay()
    torch.cuda.synchronize()
    assert_parity(yd.cpu().numpy(), oracle.apply(x, h2, P, Q, M), what="graph h2")
    f.sync_status()


@pytest.mark.parametrize("zero_copy", [False, True])
@pytest.mark.parametrize("P,Q,M,n", [(9, 9, 4, 300007), (5, 3, 4, 2 * (1 << 21) + 12345), (11, 11, 7, (1 << 21) + 1),
                                     (7, 0, 3, 5)])
def test_apply_host(P, Q, M, n, zero_copy):
    """Host buffers: chunked copy / compute pipeline (chunks of 2^21 samples with
    history), or zero copy (the kernel reads and writes pinned host memory)."""
    x = synth.ofdm2(n, key=(9, P, n % 97))
    h = synth.coeffs(P, Q, M, key=(9, 1))
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(h)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.full((n,), complex(7, 7), dtype=torch.complex64).pin_memory()
    f.apply_host(xh, out=yh, zero_copy=zero_copy)
    f.sync_status()
    ref = oracle.apply(x, h, P, Q, M)
    assert_parity(yh.numpy(), ref, what=f"host path zero_copy={zero_copy}")
    # device memory is refused by the host entry point
    lib = _lib.load()
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.dpd_apply_host(f.handle, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), n,
                              int(zero_copy), s) == 1
    assert lib.dpd_apply_host(f.handle, ctypes.c_void_p(xh.data_ptr()), ctypes.c_void_p(yh.data_ptr()), n, 7, s) == 1
    # ordinary pageable memory: copies work anywhere; zero copy where the GPU can access it, else refused
    xp = torch.from_numpy(x.copy())
    yp = torch.empty_like(xp)
    try:
        f.apply_host(xp, out=yp, zero_copy=zero_copy)
        f.sync_status()
        assert_parity(yp.numpy(), ref, what="host path pageable")
    except dpd.DPDError as e:
        assert zero_copy and e.code == 1
    f.close()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 9, 2047, 2048, 2049, 2056, 4095, 4097, 100003])
@pytest.mark.parametrize("P,Q,M,device_coeffs", [(9, 9, 4, False), (9, 9, 4, True), (11, 11, 7, False),
                                                 (3, 1, 0, True), (5, 5, 2, False)])
def test_zero_copy_tiles_and_tails(n, P, Q, M, device_coeffs):
    """Zero copy on 16-byte aligned pinned buffers (the staged kernel): ragged
    tile tails, odd lengths, tiles shorter than the history, both coefficient
    sources."""
    x = synth.ofdm2(n, key=(31, P, n % 89))
    h = synth.coeffs(P, Q, M, key=(31, 2))
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(torch.from_numpy(h).cuda() if device_coeffs else h)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.full((n + 2,), complex(7, -7), dtype=torch.complex64).pin_memory()
    f.apply_host(xh, out=yh[:n], zero_copy=True)
    f.sync_status()
    f.close()
    y = yh.numpy()
    assert np.all(y[n:] == np.complex64(7 - 7j))   # nothing written past the end
    assert_parity(y[:n], oracle.apply(x, h, P, Q, M), what=f"zero copy n={n}")


@pytest.mark.parametrize("xo,yo", [(1, 0), (0, 1), (1, 1)])
def test_zero_copy_eight_byte_aligned(xo, yo):
    """8-byte aligned host buffers take the plain-load path."""
    n = 50001
    x = synth.ofdm2(n, key=(32, xo, yo))
    h = synth.coeffs(7, 7, 3, key=(32, 1))
    f = dpd.DPD(7, 7, 3)
    f.set_coeffs(h)
    xb = torch.zeros(n + 1, dtype=torch.complex64).pin_memory()
    xb[xo: xo + n] = torch.from_numpy(x)
    yb = torch.zeros(n + 1, dtype=torch.complex64).pin_memory()
    f.apply_host(xb[xo: xo + n], out=yb[yo: yo + n], zero_copy=True)
    f.sync_status()
    f.close()
    assert_parity(yb[yo: yo + n].numpy(), oracle.apply(x, h, 7, 7, 3), what="zero copy 8-byte aligned")
