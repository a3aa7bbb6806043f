"""GPU parity of dpd_apply_stream: a continuous sample stream filtered block
by block (history carried across calls) must equal Eq. 1 applied once to the
concatenated stream, computed by the FP64 oracle."""
import numpy as np
import pytest

import dpd_synth as synth
import oracle
from util import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1612_09001_gb300 as dpd  # noqa: E402


def blocks_of(n, seed, cuts):
    """Split [0, n) into blocks: fixed awkward sizes first, then seeded random ones."""
    rng = np.random.default_rng(seed)
    sizes = list(cuts)
    while sum(sizes) < n:
        sizes.append(int(rng.integers(1, 70000)))
    sizes[-1] -= sum(sizes) - n
    return [s for s in sizes if s >= 0]


def stream_apply(f, x, sizes, offset=0, launch=None):
    if launch:
        f.set_fwd_launch(**launch)
    out = np.empty_like(x)
    pos = 0
    for s in sizes:
        xb = torch.zeros(s + offset, dtype=torch.complex64, device="cuda")
        xb[offset:] = torch.from_numpy(x[pos: pos + s]).cuda()
        y = f.apply_stream(xb[offset:])
        out[pos: pos + s] = y.cpu().numpy()
        pos += s
    f.sync_status()
    return out


@pytest.mark.parametrize("P,Q,M", [(9, 9, 4), (5, 3, 4), (11, 11, 7), (7, 7, 0), (3, 0, 2)])
@pytest.mark.parametrize("offset", [0, 1])
def test_stream_equals_one_pass(P, Q, M, offset):
    n = 400003
    x = synth.ofdm2(n, key=(20, P))
    h = synth.coeffs(P, Q, M, key=(20, M))
    sizes = blocks_of(n, seed=P + 10 * M, cuts=[0, 1, 2, 3, 0, 5, 7, 8, 9, 1, 257, 4100])
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(torch.from_numpy(h).cuda())
    y = stream_apply(f, x, sizes, offset)
    f.close()
    assert_parity(y, oracle.apply(x, h, P, Q, M), what="stream P=%d Q=%d M=%d" % (P, Q, M))


@pytest.mark.parametrize("launch", [dict(use_tma=0), dict(mode=0), dict(V=4, warps=4, stages=2)])
def test_stream_launch_shapes(launch):
    n = 200001
    x = synth.ofdm2(n, key=(21, 0))
    h = synth.coeffs(9, 9, 4, key=(21, 1))
    f = dpd.DPD(9, 9, 4)
    f.set_coeffs(h)
    y = stream_apply(f, x, blocks_of(n, 3, [4, 1, 1, 1, 1, 1, 1, 1, 9999]), launch=launch)
    f.close()
    assert_parity(y, oracle.apply(x, h, 9, 9, 4), what="stream launch %s" % launch)


def test_reset_restarts_from_zero_history():
    n = 50000
    x = synth.ofdm2(n, key=(22, 0))
    h = synth.coeffs(7, 7, 3, key=(22, 1))
    f = dpd.DPD(7, 7, 3)
    f.set_coeffs(h)
    xd = torch.from_numpy(x).cuda()
    f.apply_stream(xd[:12345])
    f.reset_stream()
    y = f.apply_stream(xd).cpu().numpy()
    # after a reset the stream starts over, so the first block equals dpd_apply
    assert np.array_equal(y, f.apply(xd).cpu().numpy())
    f.sync_status()
    f.close()
    assert_parity(y, oracle.apply(x, h, 7, 7, 3), what="after reset")


def test_empty_block_keeps_history():
    x = synth.ofdm2(1000, key=(23, 0))
    h = synth.coeffs(5, 5, 4, key=(23, 1))
    f = dpd.DPD(5, 5, 4)
    f.set_coeffs(h)
    xd = torch.from_numpy(x).cuda()
    a = f.apply_stream(xd[:500])
    f.apply_stream(xd[500:500])
    b = f.apply_stream(xd[500:])
    f.sync_status()
    f.close()
    y = torch.cat([a, b]).cpu().numpy()
    assert_parity(y, oracle.apply(x, h, 5, 5, 4), what="empty block")


def test_stream_graph_replay():
    """A captured apply_stream advances the history on every replay."""
    blk, reps = 8192, 6
    x = synth.ofdm2(blk * reps, key=(24, 0))
    h = synth.coeffs(9, 9, 4, key=(24, 1))
    f = dpd.DPD(9, 9, 4)
    f.set_coeffs(torch.from_numpy(h).cuda())
    xin = torch.empty(blk, dtype=torch.complex64, device="cuda")
    yout = torch.empty(blk, dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        f.apply_stream(xin, out=yout, stream=s)   # first call outside capture
    torch.cuda.synchronize()
    f.reset_stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        f.apply_stream(xin, out=yout, stream=s)
    out = []
    for r in range(reps):
        xin.copy_(torch.from_numpy(x[r * blk:(r + 1) * blk]).cuda())
        g.replay()
        out.append(yout.cpu().numpy().copy())
    f.sync_status()
    f.close()
    assert_parity(np.concatenate(out), oracle.apply(x, h, 9, 9, 4), what="stream graph replay")
