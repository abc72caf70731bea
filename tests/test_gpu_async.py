"""GPU: the asynchronous forms (sz3g_compress_async / sz3g_decompress_async).
They enqueue without synchronising or allocating, report the stream length
and status on the device, and can be captured into a CUDA graph; replays of a
captured compress on new data in the same buffer must give the oracle's
stream for that data, byte for byte."""
import struct

import numpy as np
import pytest

import oracle as O
from paper_2111_02925_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_02925_gb300 import build as B  # noqa: E402
from paper_2111_02925_gb300 import sz3g as G  # noqa: E402

B.build()
G.load()
DEV = "cuda"


def _bufs(shape, eb, interp=G.CUBIC, mode=G.REL):
    p = G.make_params(shape, eb, eb_mode=mode, interp=interp)
    cap = G.sz3g_compress_bound(p)
    xd = torch.empty(int(np.prod(shape)), dtype=torch.float32, device=DEV)
    out = torch.zeros(cap, dtype=torch.uint8, device=DEV)
    res = torch.zeros(2, dtype=torch.int64, device=DEV)  # [0]: bytes, [1]: status (int32 in the low half)
    ws = G.workspace(p, False, DEV)
    return p, cap, xd, out, res, ws


def _enqueue_compress(p, cap, xd, out, res, ws, stream):
    return G.sz3g_compress_async(p, xd.data_ptr(), out.data_ptr(), cap, res.data_ptr(), res.data_ptr() + 8,
                                 ws.data_ptr(), ws.numel(), stream)


def _result(res):
    r = res.cpu().numpy()
    status = np.array([int(r[1]) & 0xFFFFFFFF], np.uint32).view(np.int32)[0]
    return int(r[0]), int(status)


def _oracle_stream(x, eb, interp=O.CUBIC, mode=O.REL):
    return O.compress(O.make_params(x.shape, eb, eb_mode=mode, interp=interp), x)


def test_async_compress_and_decompress_match_oracle():
    x = S.grf((36, 40, 44), 3).astype(np.float32)
    p, cap, xd, out, res, ws = _bufs(x.shape, 1e-3)
    xd.copy_(torch.from_numpy(x.reshape(-1)))
    st = torch.cuda.current_stream()
    assert _enqueue_compress(p, cap, xd, out, res, ws, st.cuda_stream) == G.OK
    torch.cuda.synchronize()
    nb, status = _result(res)
    so = _oracle_stream(x, 1e-3)
    assert status == G.OK and nb == len(so)
    s = out[:nb].cpu().numpy().tobytes()
    assert s == so
    # decompress from the host copy of the header
    head = np.frombuffer(s[:G.HEADER_BYTES], np.uint8).copy()
    y = torch.empty(x.size, dtype=torch.float32, device=DEV)
    wsd = G.workspace(p, True, DEV)
    stat = torch.full((1,), 7, dtype=torch.int32, device=DEV)
    rc = G.sz3g_decompress_async(head.ctypes.data, out.data_ptr(), nb, y.data_ptr(), y.numel() * 4,
                                 stat.data_ptr(), wsd.data_ptr(), wsd.numel(), st.cuda_stream)
    assert rc == G.OK
    torch.cuda.synchronize()
    assert int(stat.item()) == G.OK
    want = O.decompress(so).reshape(-1)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), want.view(np.uint32))


def test_captured_compress_replays_on_new_data():
    shape = (40, 36, 48)
    p, cap, xd, out, res, ws = _bufs(shape, 1e-3)
    xd.copy_(torch.from_numpy(S.grf(shape, 10).astype(np.float32).reshape(-1)))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm the kernels' attributes outside the capture
        assert _enqueue_compress(p, cap, xd, out, res, ws, side.cuda_stream) == G.OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        rc = _enqueue_compress(p, cap, xd, out, res, ws, torch.cuda.current_stream().cuda_stream)
    assert rc == G.OK
    for seed in (11, 12, 13):
        x = S.grf(shape, seed).astype(np.float32)
        xd.copy_(torch.from_numpy(x.reshape(-1)))
        out.zero_()
        res.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        nb, status = _result(res)
        so = _oracle_stream(x, 1e-3)
        assert status == G.OK and nb == len(so)
        assert out[:nb].cpu().numpy().tobytes() == so


def test_captured_decompress_replays():
    x = S.grf((30, 34, 40), 21).astype(np.float32)
    so = _oracle_stream(x, 1e-3)
    p = G.make_params(x.shape, 1e-3, eb_mode=G.REL, interp=G.CUBIC)
    d = torch.from_numpy(np.frombuffer(so, np.uint8).copy()).to(DEV)
    head = np.frombuffer(so[:G.HEADER_BYTES], np.uint8).copy()
    y = torch.empty(x.size, dtype=torch.float32, device=DEV)
    wsd = G.workspace(p, True, DEV)
    stat = torch.zeros(1, dtype=torch.int32, device=DEV)

    def enq(stream):
        return G.sz3g_decompress_async(head.ctypes.data, d.data_ptr(), d.numel(), y.data_ptr(), y.numel() * 4,
                                       stat.data_ptr(), wsd.data_ptr(), wsd.numel(), stream)

    assert enq(torch.cuda.current_stream().cuda_stream) == G.OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        assert enq(torch.cuda.current_stream().cuda_stream) == G.OK
    want = O.decompress(so).reshape(-1).view(np.uint32)
    for _ in range(2):
        y.fill_(float("nan"))
        stat.fill_(99)
        g.replay()
        torch.cuda.synchronize()
        assert int(stat.item()) == G.OK
        assert np.array_equal(y.cpu().numpy().view(np.uint32), want)


def test_async_reports_errors_on_the_device():
    st = torch.cuda.current_stream().cuda_stream
    # REL bound on a constant field
    p, cap, xd, out, res, ws = _bufs((16, 18, 20), 1e-3)
    xd.fill_(2.5)
    assert _enqueue_compress(p, cap, xd, out, res, ws, st) == G.OK
    torch.cuda.synchronize()
    assert _result(res) == (0, G.E_ZERO_RANGE_REL)
    # a non-finite input
    xd.copy_(torch.from_numpy(S.grf((16, 18, 20), 4).astype(np.float32).reshape(-1)))
    xd[100] = float("inf")
    assert _enqueue_compress(p, cap, xd, out, res, ws, st) == G.OK
    torch.cuda.synchronize()
    assert _result(res) == (0, G.E_NONFINITE)
    # an output buffer too small for the stream
    xd[100] = 0.0
    rc = G.sz3g_compress_async(p, xd.data_ptr(), out.data_ptr(), 1024, res.data_ptr(), res.data_ptr() + 8,
                               ws.data_ptr(), ws.numel(), st)
    assert rc == G.OK
    torch.cuda.synchronize()
    assert _result(res) == (0, G.E_CAPACITY)
    # host-side checks: no workspace, a short workspace
    assert G.sz3g_compress_async(p, xd.data_ptr(), out.data_ptr(), cap, res.data_ptr(), res.data_ptr() + 8,
                                 0, 0, st) == G.E_INVAL
    assert G.sz3g_compress_async(p, xd.data_ptr(), out.data_ptr(), cap, res.data_ptr(), res.data_ptr() + 8,
                                 ws.data_ptr(), 256, st) == G.E_CAPACITY
    # a code length past the limit: found by the decoder's table build
    x = S.grf((20, 20, 20), 5).astype(np.float32)
    s = bytearray(_oracle_stream(x, 1e-3))
    n_unpred = struct.unpack_from("<Q", s, 88)[0]
    s[288 + ((n_unpred * 4 + 7) & ~7) + 2] = 30
    d = torch.from_numpy(np.frombuffer(bytes(s), np.uint8).copy()).to(DEV)
    head = np.frombuffer(bytes(s[:G.HEADER_BYTES]), np.uint8).copy()
    pd = G.make_params(x.shape, 1e-3, eb_mode=G.REL, interp=G.CUBIC)
    wsd = G.workspace(pd, True, DEV)
    y = torch.empty(x.size, dtype=torch.float32, device=DEV)
    stat = torch.zeros(1, dtype=torch.int32, device=DEV)
    rc = G.sz3g_decompress_async(head.ctypes.data, d.data_ptr(), d.numel(), y.data_ptr(), y.numel() * 4,
                                 stat.data_ptr(), wsd.data_ptr(), wsd.numel(), st)
    assert rc == G.OK
    torch.cuda.synchronize()
    assert int(stat.item()) == G.E_CORRUPT
    # a damaged magic is a host-side error
    head[0] ^= 0xFF
    assert G.sz3g_decompress_async(head.ctypes.data, d.data_ptr(), d.numel(), y.data_ptr(), y.numel() * 4,
                                   stat.data_ptr(), wsd.data_ptr(), wsd.numel(), st) == G.E_CORRUPT
