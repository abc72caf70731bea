"""GPU: batches (many fields per graph launch) against one call per field and
against the oracle.  A batch runs the same kernels as the single-field calls,
so its streams and reconstructions must be byte-identical to theirs, under
every branch count and CTA cap, and after the autotuner has picked one."""
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


def _mix(count, seed, scale):
    """The uneven batch mix (log-uniform axes, REL bounds, mixed kinds),
    axes scaled down by `scale` so the oracle finishes quickly."""
    out = []
    for dims, eb, interp in S.batch_shapes(count, seed):
        d = tuple(max(2, int(round(a / scale))) for a in dims)
        out.append((d, eb, interp))
    return out


def _fields(mix, seed):
    return [S.grf(d, seed + i).astype(np.float32) for i, (d, _, _) in enumerate(mix)]


def _single(params, xs):
    streams = []
    for p, x in zip(params, xs):
        xd = torch.from_numpy(x.reshape(-1)).to(DEV)
        cap = G.sz3g_compress_bound(p)
        out = torch.empty(cap, dtype=torch.uint8, device=DEV)
        rc, nb = G.sz3g_compress(p, xd.data_ptr(), out.data_ptr(), cap, stream=G._stream_handle())
        assert rc == 0
        streams.append(out[:nb].cpu().numpy().tobytes())
    return streams


def _batch_compress(params, xs, configs):
    ins = [torch.from_numpy(x.reshape(-1)).to(DEV) for x in xs]
    caps = [G.sz3g_compress_bound(p) for p in params]
    outs = [torch.zeros(c, dtype=torch.uint8, device=DEV) for c in caps]
    b = G.Batch(params, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], caps)
    results = []
    try:
        for cfg in configs:
            if cfg == "tune":
                br, cap = b.tune(G._stream_handle())
                assert br >= 1 and cap >= 0
            elif cfg is not None:
                b.configure(*cfg)
            for o in outs:
                o.zero_()
            b.run(G._stream_handle())
            rc, nbytes, st = b.results()
            assert rc == 0 and all(s == 0 for s in st)
            results.append([o[:n].cpu().numpy().tobytes() for o, n in zip(outs, nbytes)])
        br, cap, nodes = b.info()
        assert nodes > len(params)  # every field's launches are graph nodes
    finally:
        b.close()
    return results


def test_batch_compress_matches_single_calls_and_oracle():
    mix = _mix(12, 4, 4.0)
    xs = _fields(mix, 400)
    params = [G.make_params(x.shape, eb, eb_mode=G.REL, interp=it) for x, (_, eb, it) in zip(xs, mix)]
    ref = _single(params, xs)
    runs = _batch_compress(params, xs, [None, (1, 0), (3, 0), (12, 16), (5, 1), "tune"])
    for r in runs:
        assert r == ref
    # two of the fields also against the oracle
    for i in (0, 7):
        op = O.make_params(xs[i].shape, mix[i][1], eb_mode=O.REL, interp=mix[i][2])
        assert O.compress(op, xs[i]) == ref[i]


def test_batch_decompress_matches_single_calls():
    mix = _mix(10, 5, 4.0)
    xs = _fields(mix, 500)
    params = [G.make_params(x.shape, eb, eb_mode=G.REL, interp=it) for x, (_, eb, it) in zip(xs, mix)]
    streams = _single(params, xs)
    sd = [torch.from_numpy(np.frombuffer(s, np.uint8).copy()).to(DEV) for s in streams]
    outs = [torch.full((x.size,), float("nan"), dtype=torch.float32, device=DEV) for x in xs]
    b = G.Batch(None, [t.data_ptr() for t in sd], [t.data_ptr() for t in outs], [x.size * 4 for x in xs],
                in_bytes=[len(s) for s in streams], decompress=True)
    try:
        for cfg in (None, (2, 0), (10, 8)):
            if cfg is not None:
                b.configure(*cfg)
            b.run(G._stream_handle())
            rc, _, st = b.results()
            assert rc == 0 and all(s == 0 for s in st)
            for s, o in zip(streams, outs):
                ref = O.decompress(s)
                got = o.cpu().numpy()
                assert np.array_equal(got.view(np.uint32), ref.reshape(-1).view(np.uint32))
    finally:
        b.close()


def test_batch_reports_per_field_errors():
    xs = [S.grf((20, 24, 28), 1), np.zeros((16, 16, 16), np.float32)]  # REL on a constant field
    params = [G.make_params(x.shape, 1e-3, eb_mode=G.REL, interp=G.CUBIC) for x in xs]
    ins = [torch.from_numpy(x.reshape(-1)).to(DEV) for x in xs]
    caps = [G.sz3g_compress_bound(p) for p in params]
    outs = [torch.zeros(c, dtype=torch.uint8, device=DEV) for c in caps]
    b = G.Batch(params, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], caps)
    try:
        b.run(G._stream_handle())
        rc, _, st = b.results()
        assert st[0] == 0 and st[1] == G.E_ZERO_RANGE_REL and rc == G.E_ZERO_RANGE_REL
    finally:
        b.close()
