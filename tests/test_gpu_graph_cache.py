"""GPU: calls with a caller-owned workspace replay a cached graph of the
pipeline.  Replays must give the same bytes as the oracle, a change of
parameters on the same buffers must not replay the old pipeline, and the
replayed launches must still be counted."""
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


def test_graph_cache_replays_match_oracle():
    x = S.grf((40, 52, 36), 31).astype(np.float32)
    xd = torch.from_numpy(x.reshape(-1)).to(DEV)
    sh = G._stream_handle()
    G.sz3g_graph_cache(True)
    results = []
    for eb, interp in ((1e-3, G.CUBIC), (1e-3, G.CUBIC), (1e-4, G.LINEAR), (1e-3, G.CUBIC), (1e-4, G.LINEAR)):
        p = G.make_params(x.shape, eb, eb_mode=G.REL, interp=interp)
        wsc = G.workspace(p, False, DEV)
        wsd = G.workspace(p, True, DEV)
        cap = max(G.sz3g_compress_bound(G.make_params(x.shape, e, eb_mode=G.REL)) for e in (1e-3, 1e-4))
        if not results:
            out = torch.zeros(cap, dtype=torch.uint8, device=DEV)
            y = torch.empty_like(xd)
            ws_c = torch.zeros(max(wsc.numel(), 1 << 24), dtype=torch.uint8, device=DEV)
            ws_d = torch.zeros(max(wsd.numel(), 1 << 24), dtype=torch.uint8, device=DEV)
        n0 = G.sz3g_launch_count()
        rc, nb = G.sz3g_compress(p, xd.data_ptr(), out.data_ptr(), cap, ws_c.data_ptr(), ws_c.numel(), sh)
        assert rc == 0
        rc = G.sz3g_decompress(out.data_ptr(), nb, y.data_ptr(), y.numel() * 4, ws_d.data_ptr(), ws_d.numel(), sh)
        assert rc == 0
        launches = G.sz3g_launch_count() - n0
        s = out[:nb].cpu().numpy().tobytes()
        op = O.make_params(x.shape, eb, eb_mode=O.REL, interp=interp)
        assert s == O.compress(op, x)
        assert np.array_equal(y.cpu().numpy().view(np.uint32), O.decompress(s).reshape(-1).view(np.uint32))
        results.append((eb, interp, launches))
    # a replay counts the same launches as the capture it replays
    assert results[0][2] > 0 and results[1][2] == results[0][2] == results[3][2]
    assert results[2][2] == results[4][2] > 0
    G.sz3g_graph_cache(False)
    p = G.make_params(x.shape, 1e-3, eb_mode=G.REL, interp=G.CUBIC)
    rc, nb = G.sz3g_compress(p, xd.data_ptr(), out.data_ptr(), cap, ws_c.data_ptr(), ws_c.numel(), sh)
    assert rc == 0 and out[:nb].cpu().numpy().tobytes() == O.compress(O.make_params(x.shape, 1e-3, eb_mode=O.REL,
                                                                                   interp=O.CUBIC), x)
    G.sz3g_graph_cache(True)


def test_graph_cache_reports_errors_of_replays():
    # a REL bound on a constant field fails the same way on every replay
    x = np.zeros((24, 20, 28), np.float32)
    xd = torch.from_numpy(x.reshape(-1)).to(DEV)
    p = G.make_params(x.shape, 1e-3, eb_mode=G.REL)
    cap = G.sz3g_compress_bound(p)
    out = torch.zeros(cap, dtype=torch.uint8, device=DEV)
    ws = G.workspace(p, False, DEV)
    G.sz3g_graph_cache(True)
    for _ in range(3):
        rc, _ = G.sz3g_compress(p, xd.data_ptr(), out.data_ptr(), cap, ws.data_ptr(), ws.numel(), G._stream_handle())
        assert rc == G.E_ZERO_RANGE_REL
