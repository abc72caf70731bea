"""The checking build: every kernel index check compiled in.

The library built with -DSZ3G_CHECK guards the kernels' computed global
and shared-memory writes (codes, reconstructions, the even-k plane, code
rows staged from global memory, payload words, unpredictable values, zero
counts) with range checks; a failed check raises a flag, the call reports
SZ3G_E_CHECK and the access is skipped.  Running the parity cases, the
batch forms, the Huffman stage entry points and the 512^3 headline field on
that build shows that no index leaves its buffer, with every result still
byte-identical to the oracle (or, at 512^3, to the ordinary build).  It
stands in for a memory checker, which is not available here.  The file
runs last in the GPU suite and loads the ordinary library again at the end.
"""
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

DEV = "cuda"

CASES = [
    # name, field maker, dtype, eb_mode, eb, interp, order, radius, chunk
    ("bumps64_lin", lambda: S.gaussian_bumps(64, 1), O.F32, O.ABS, 3.1e-3, O.LINEAR, (0, 1, 2), 32768, 4096),
    ("grf_ragged_cubic", lambda: S.grf((37, 50, 29), 2), O.F32, O.REL, 1e-3, O.CUBIC, (0, 1, 2), 32768, 4096),
    ("grf_order201", lambda: S.grf((33, 17, 65), 3), O.F32, O.REL, 1e-2, O.CUBIC, (2, 0, 1), 32768, 512),
    ("grf_tight_unpred", lambda: S.grf((24, 24, 24), 4), O.F32, O.REL, 1e-5, O.LINEAR, (1, 2, 0), 64, 256),
    ("latlon_cubic", lambda: S.latlon(181, 363, 5), O.F64, O.ABS, 1e-5, O.CUBIC, (1, 0), 32768, 4096),
    ("grf1d", lambda: S.grf((5000,), 6), O.F32, O.REL, 1e-3, O.CUBIC, (0,), 32768, 1024),
    ("grf4d", lambda: S.grf((7, 9, 6, 10), 7), O.F32, O.REL, 1e-3, O.LINEAR, (3, 1, 0, 2), 32768, 256),
    ("grf3d_f64_cubic", lambda: S.grf((40, 48, 80), 12).astype(np.float64), O.F64, O.REL, 1e-4, O.CUBIC,
     (0, 1, 2), 32768, 4096),
    # 2-D FP32: code rows by per-row copies (rows of 100 odd-k codes) and,
    # on the power-of-two grid, by tensor copies
    ("grf2d_f32_cubic", lambda: S.grf((136, 200), 13), O.F32, O.REL, 1e-3, O.CUBIC, (0, 1), 32768, 4096),
    ("grf2d_f32_pow2_lin", lambda: S.grf((128, 256), 14), O.F32, O.REL, 1e-3, O.LINEAR, (0, 1), 32768, 4096),
    ("tiny_2x1x3", lambda: np.arange(6, dtype=np.float32).reshape(2, 1, 3), O.F32, O.ABS, 0.1, O.CUBIC,
     (0, 1, 2), 32768, 8),
    ("all_unpred", lambda: S.grf((12, 13, 14), 9), O.F32, O.REL, 1e-7, O.LINEAR, (0, 1, 2), 2, 8),
    ("grf_130_cubic", lambda: S.grf((130, 66, 140), 10), O.F32, O.REL, 1e-4, O.CUBIC, (0, 1, 2), 32768, 4096),
]


def _compress(gp, x):
    t = torch.float32 if gp.dtype == G.F32 else torch.float64
    xd = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(DEV).to(t)
    cap = G.sz3g_compress_bound(gp)
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    rc, nb = G.sz3g_compress(gp, xd.data_ptr(), out.data_ptr(), cap, stream=G._stream_handle())
    return rc, out[:nb].cpu().numpy().tobytes() if rc == G.OK else b""


def _decompress(s, n, dtype):
    sd = torch.from_numpy(np.frombuffer(s, np.uint8).copy()).to(DEV)
    t = torch.float32 if dtype == G.F32 else torch.float64
    y = torch.empty(max(n, 1), dtype=t, device=DEV)
    rc = G.sz3g_decompress(sd.data_ptr(), len(s), y.data_ptr(), n * y.element_size(), stream=G._stream_handle())
    return rc, y[:n].cpu().numpy()


@pytest.fixture(scope="module")
def checked():
    """The checking build loaded in place of the ordinary library; the 512^3
    headline stream of the ordinary build is taken first for comparison."""
    B.build()
    G.load(B.LIB, reload=True)
    x = S.grf((512, 512, 512), 2)
    gp = G.make_params(x.shape, 1e-3, eb_mode=G.REL, interp=G.CUBIC)
    rc, ref = _compress(gp, x)
    assert rc == G.OK
    rc, yref = _decompress(ref, x.size, G.F32)
    assert rc == G.OK
    G.load(B.build(check=True), reload=True)
    yield {"x": x, "gp": gp, "ref": ref, "yref": yref.view(np.uint32)}
    G.load(B.LIB, reload=True)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_checked_build_round_trip_matches_oracle(checked, case):
    _, make, dt, mode, eb, interp, order, radius, chunk = case
    x = make()
    x = x.astype(np.float64 if dt == O.F64 else np.float32)
    kw = dict(dtype=dt, eb_mode=mode, interp=interp, order=order, radius=radius, chunk=chunk)
    rc, s = _compress(G.make_params(x.shape, eb, **kw), x)
    assert rc == G.OK, G.strerror(rc)
    assert s == O.compress(O.make_params(x.shape, eb, **kw), x)
    rc, y = _decompress(s, x.size, dt)
    assert rc == G.OK, G.strerror(rc)
    w = np.uint64 if dt == O.F64 else np.uint32
    assert np.array_equal(y.view(w), O.decompress(s).reshape(-1).view(w))


def test_checked_build_headline_field(checked):
    rc, s = _compress(checked["gp"], checked["x"])
    assert rc == G.OK, G.strerror(rc)
    assert s == checked["ref"]
    rc, y = _decompress(s, checked["x"].size, G.F32)
    assert rc == G.OK, G.strerror(rc)
    assert np.array_equal(y.view(np.uint32), checked["yref"])


@pytest.mark.parametrize("queue", [False, True])
def test_checked_build_batch(checked, queue):
    shapes = [(40, 36, 44), (33, 50, 29), (64, 20, 30), (17, 65, 9)]
    xs = [S.grf(sh, 900 + i).astype(np.float32) for i, sh in enumerate(shapes)]
    ebs = [1e-3, 3e-4, 2e-3, 1e-2]
    params = [G.make_params(x.shape, eb, eb_mode=G.REL, interp=i % 2) for i, (x, eb) in enumerate(zip(xs, ebs))]
    ref = [O.compress(O.make_params(x.shape, eb, eb_mode=O.REL, interp=i % 2), x)
           for i, (x, eb) in enumerate(zip(xs, ebs))]
    ins = [torch.from_numpy(x.reshape(-1)).to(DEV) for x in xs]
    caps = [G.sz3g_compress_bound(p) for p in params]
    outs = [torch.zeros(c, dtype=torch.uint8, device=DEV) for c in caps]
    b = G.Batch(params, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], caps)
    try:
        b.set_queue(queue)
        b.configure(2, 0)
        b.run(G._stream_handle())
        rc, nbytes, st = b.results()
    finally:
        b.close()
    assert rc == G.OK and all(v == G.OK for v in st), [G.strerror(v) for v in st]
    assert [o[:n].cpu().numpy().tobytes() for o, n in zip(outs, nbytes)] == ref


@pytest.mark.parametrize("nsym,spread,chunk", [(65536, 300.0, 4096), (1024, 20.0, 1000), (8, 0.3, 512)])
def test_checked_build_huffman_stages(checked, nsym, spread, chunk):
    rng = np.random.default_rng(nsym)
    n = 200_003
    c = nsym // 2 if nsym > 2 else 0
    codes = np.clip(np.round(rng.laplace(c, spread, n)), 0, nsym - 1).astype(np.uint16)
    hist = O.histogram(codes)
    ln = O.huffman_lengths(hist[:nsym])
    hd = torch.from_numpy(hist.astype(np.uint32).view(np.int32)).to(DEV)
    glen = torch.empty(nsym, dtype=torch.uint8, device=DEV)
    gcode = torch.empty(nsym, dtype=torch.int32, device=DEV)
    assert G.sz3g_huffman_build(hd.data_ptr(), nsym, glen.data_ptr(), gcode.data_ptr(), G._stream_handle()) == G.OK
    assert np.array_equal(glen.cpu().numpy(), ln)
    cd = torch.from_numpy(codes.view(np.int16).copy()).to(DEV)
    nch = (n + chunk - 1) // chunk
    nsb = (chunk + 511) // 512
    cap = n + 64
    words = torch.zeros(cap, dtype=torch.int32, device=DEV)
    cw = torch.zeros(nch, dtype=torch.int32, device=DEV)
    sub = torch.zeros(max(nch * (nsb - 1), 1), dtype=torch.int16, device=DEV)
    rc, nw = G.sz3g_huffman_encode(cd.data_ptr(), n, glen.data_ptr(), gcode.data_ptr(), nsym, chunk,
                                   words.data_ptr(), cap, cw.data_ptr(), sub.data_ptr() if nsb > 1 else 0,
                                   stream=G._stream_handle())
    assert rc == G.OK, G.strerror(rc)
    back = torch.empty(n + 64, dtype=torch.int16, device=DEV)
    for sb in ([sub.data_ptr()] if nsb > 1 else []) + [0]:  # with the sub-block table, then whole chunks
        back.zero_()
        rc = G.sz3g_huffman_decode(words.data_ptr(), nw, cw.data_ptr(), sb, chunk, glen.data_ptr(), nsym,
                                   back.data_ptr(), n, stream=G._stream_handle())
        assert rc == G.OK, G.strerror(rc)
        assert np.array_equal(back[:n].cpu().numpy().view(np.uint16), codes)
