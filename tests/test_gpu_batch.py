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
            elif isinstance(cfg, str) and cfg.startswith("queue"):
                b.set_queue(True)
                b.configure(int(cfg[5:]), 0)
                on, levels = b.queue_info()
                assert on and levels > 0
            elif cfg is not None:
                b.set_queue(False)
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
    runs = _batch_compress(params, xs, [None, (1, 0), (3, 0), (12, 16), (5, 1), "queue1", "queue5", "tune"])
    for r in runs:
        assert r == ref
    # every field also against the oracle
    for i in range(len(xs)):
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
        for cfg in (None, (2, 0), (10, 8), "queue3", "queue1"):
            if isinstance(cfg, str):
                b.set_queue(True)
                b.configure(int(cfg[5:]), 0)
                assert b.queue_info()[0]
            elif cfg is not None:
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


def test_level_queue_mixed_types_and_ranks():
    """The cross-field level queue over fields of both element types, ranks 1
    to 4 (rank 4 keeps its own launches), both interpolations and uneven
    bounds: streams byte-identical to one call per field, and back."""
    rng = np.random.default_rng(9)
    shapes = [(37, 29, 41), (64, 48, 40), (90, 70), (257,), (5, 6, 7, 8), (33, 17, 65), (128, 3, 50), (19, 160)]
    xs, params = [], []
    for i, sh in enumerate(shapes):
        x = S.grf(sh, 900 + i)
        dt = O.F64 if i % 3 == 1 else O.F32
        xs.append(x.astype(np.float64 if dt == O.F64 else np.float32))
        params.append(G.make_params(sh, float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-2)))),
                                    dtype=G.F64 if dt == O.F64 else G.F32, eb_mode=G.REL, interp=i % 2))
    ref = _single(params, xs)
    ins = [torch.from_numpy(x.reshape(-1)).to(DEV) for x in xs]
    caps = [G.sz3g_compress_bound(p) for p in params]
    outs = [torch.zeros(c, dtype=torch.uint8, device=DEV) for c in caps]
    b = G.Batch(params, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], caps)
    try:
        for br in (1, 3, 8):
            b.set_queue(True)
            b.configure(br, 0)
            on, levels = b.queue_info()
            assert on and levels > 0
            for o in outs:
                o.zero_()
            b.run(G._stream_handle())
            rc, nbytes, st = b.results()
            assert rc == 0 and all(v == 0 for v in st)
            assert [o[:n].cpu().numpy().tobytes() for o, n in zip(outs, nbytes)] == ref
    finally:
        b.close()
    sd = [torch.from_numpy(np.frombuffer(r, np.uint8).copy()).to(DEV) for r in ref]
    back = [torch.full((x.size,), float("nan"), dtype=torch.float64 if x.dtype == np.float64 else torch.float32,
                       device=DEV) for x in xs]
    bd = G.Batch(None, [t.data_ptr() for t in sd], [t.data_ptr() for t in back], [x.nbytes for x in xs],
                 in_bytes=[len(r) for r in ref], decompress=True)
    try:
        bd.set_queue(True)
        bd.configure(4, 0)
        bd.run(G._stream_handle())
        rc, _, st = bd.results()
        assert rc == 0 and all(v == 0 for v in st)
        for r, o, x in zip(ref, back, xs):
            want = O.decompress(r).reshape(-1)
            got = o.cpu().numpy()
            assert got.dtype == want.dtype and np.array_equal(got.view(np.uint8), want.view(np.uint8))
    finally:
        bd.close()
