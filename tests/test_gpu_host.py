"""GPU: the end-to-end forms on host buffers (sz3g_compress_host /
sz3g_decompress_host).  Their streams and fields must equal the oracle's byte
for byte, from pinned and from pageable host memory, across changes of shape
(the staging set grows), from two threads at once (one of them stages through
pool memory), after sz3g_trim, and after a call that failed."""
import threading

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


def _host_roundtrip(x, eb, interp, pinned=True, stream=0):
    p = G.make_params(x.shape, eb, dtype=G.F64 if x.dtype == np.float64 else G.F32, eb_mode=G.REL, interp=interp)
    cap = G.sz3g_compress_bound(p)
    hx = torch.from_numpy(np.ascontiguousarray(x).reshape(-1))
    hs = torch.zeros(cap, dtype=torch.uint8)
    hy = torch.empty(x.size, dtype=hx.dtype)
    if pinned:
        hx, hs, hy = hx.pin_memory(), hs.pin_memory(), hy.pin_memory()
    rc, nb = G.sz3g_compress_host(p, hx.data_ptr(), hs.data_ptr(), cap, stream)
    assert rc == G.OK, G.load().sz3g_strerror(rc)
    rc = G.sz3g_decompress_host(hs.data_ptr(), nb, hy.data_ptr(), hy.numel() * hy.element_size(), stream)
    assert rc == G.OK, G.load().sz3g_strerror(rc)
    return hs[:nb].numpy().tobytes(), hy.numpy().copy()


def _oracle(x, eb, interp):
    op = O.make_params(x.shape, eb, dtype=O.F64 if x.dtype == np.float64 else O.F32, eb_mode=O.REL, interp=interp)
    s = O.compress(op, x)
    return s, O.decompress(s).reshape(-1)


def _same_field(a, b):
    bits = np.uint32 if a.dtype == np.float32 else np.uint64
    return np.array_equal(a.view(bits), b.reshape(-1).view(bits))


@pytest.mark.parametrize("pinned", [True, False])
def test_host_forms_match_oracle_across_shapes(pinned):
    cases = [
        (S.grf((33, 47, 70), 5).astype(np.float32), 1e-3, G.CUBIC),
        (S.grf((70, 66, 90), 6).astype(np.float32), 1e-4, G.LINEAR),   # staging grows
        (S.grf((21, 18, 30), 7).astype(np.float64), 1e-3, G.CUBIC),    # smaller again, another type
        (S.grf((33, 47, 70), 5).astype(np.float32), 1e-3, G.CUBIC),    # same shape as the first
        (S.grf((48, 50, 64), 8).astype(np.float32), 1e-3, G.CUBIC),    # 16-byte rows
        (S.grf((36, 44), 9).astype(np.float32), 1e-3, G.LINEAR),     # 2-D
    ]
    for x, eb, interp in cases:
        s, y = _host_roundtrip(x, eb, interp, pinned=pinned)
        so, yo = _oracle(x, eb, interp)
        assert s == so
        assert _same_field(y, yo)


def test_host_forms_from_two_threads():
    xs = [S.grf((40, 44, 52), 11 + t).astype(np.float32) for t in range(2)]
    want = [_oracle(x, 1e-3, G.CUBIC) for x in xs]
    got = [None, None]
    errors = []

    def run(t):
        try:
            st = torch.cuda.Stream()
            for _ in range(3):
                got[t] = _host_roundtrip(xs[t], 1e-3, G.CUBIC, stream=st.cuda_stream)
        except Exception as e:  # surfaced below
            errors.append(e)

    th = [threading.Thread(target=run, args=(t,)) for t in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for t in range(2):
        assert got[t][0] == want[t][0]
        assert _same_field(got[t][1], want[t][1])


def test_host_decompress_into_pinned_output_at_any_offset():
    # outputs that start at any 4-byte offset of a page-locked buffer
    x = S.grf((40, 52, 64), 13).astype(np.float32)
    so, yo = _oracle(x, 1e-3, G.CUBIC)
    hs = torch.from_numpy(np.frombuffer(so, np.uint8).copy()).pin_memory()
    big = torch.full((x.size + 16,), np.nan, dtype=torch.float32).pin_memory()
    for off in (0, 1, 4, 3):
        y = big[off:off + x.size]
        rc = G.sz3g_decompress_host(hs.data_ptr(), hs.numel(), y.data_ptr(), x.size * 4, 0)
        assert rc == G.OK
        assert _same_field(y.numpy().copy(), yo)


def test_host_forms_after_trim_and_after_errors():
    x = S.grf((30, 36, 40), 21).astype(np.float32)
    so, yo = _oracle(x, 1e-3, G.CUBIC)
    p = G.make_params(x.shape, 1e-3, eb_mode=G.REL, interp=G.CUBIC)
    hx = torch.from_numpy(x.reshape(-1)).pin_memory()
    hs = torch.zeros(G.sz3g_compress_bound(p), dtype=torch.uint8).pin_memory()
    # output buffer smaller than the stream
    rc, _ = G.sz3g_compress_host(p, hx.data_ptr(), hs.data_ptr(), 64, 0)
    assert rc == G.E_CAPACITY
    # a stream whose header is damaged
    bad = torch.from_numpy(np.frombuffer(so, np.uint8).copy())
    bad[0] ^= 0xFF
    hy = torch.empty(x.size, dtype=torch.float32)
    assert G.sz3g_decompress_host(bad.data_ptr(), bad.numel(), hy.data_ptr(), hy.numel() * 4, 0) == G.E_CORRUPT
    # an output buffer too small for the field
    good = torch.from_numpy(np.frombuffer(so, np.uint8).copy())
    assert G.sz3g_decompress_host(good.data_ptr(), good.numel(), hy.data_ptr(), 16, 0) == G.E_CAPACITY
    # a REL bound on a constant field
    z = np.zeros((8, 9, 10), np.float32)
    pz = G.make_params(z.shape, 1e-3, eb_mode=G.REL)
    hz = torch.from_numpy(z.reshape(-1))
    hzs = torch.zeros(G.sz3g_compress_bound(pz), dtype=torch.uint8)
    assert G.sz3g_compress_host(pz, hz.data_ptr(), hzs.data_ptr(), hzs.numel(), 0)[0] == G.E_ZERO_RANGE_REL
    # the next calls work, before and after the kept memory is freed
    for trim in (False, True):
        if trim:
            G.sz3g_trim()
        s, y = _host_roundtrip(x, 1e-3, G.CUBIC)
        assert s == so and _same_field(y, yo)
