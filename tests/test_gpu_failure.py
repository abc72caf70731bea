"""GPU failure handling, every failure injected on the host.

No test here faults, traps or hangs the GPU.  A dependency of the batch's
level queue is made unreachable and a chunk of the one-pass encoder is kept
from publishing its look-back state, with the wait limits shortened: the
bounded waits give up, the call reports SZ3G_E_TIMEOUT, and the next normal
call is byte-identical to the oracle.  A refused workspace allocation gives
SZ3G_E_NOMEM and keeps no device memory.  Every parity case also runs twice
and must give the same bytes both times (a stand-in for a race detector:
results that depend on scheduling would differ between runs).
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

B.build()
G.load()
DEV = "cuda"
SHORT_WAIT = 4000  # polls of about 100 ns (queue) or 32 ns (look-back) before a wait gives up


@pytest.fixture(autouse=True)
def _reset_injection():
    assert G.sz3g_debug_inject(G.DEBUG_RESET) == G.OK
    yield
    assert G.sz3g_debug_inject(G.DEBUG_RESET) == G.OK
    G.sz3g_graph_cache(True)


def _compress(gp, x):
    xd = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(DEV)
    cap = G.sz3g_compress_bound(gp)
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    rc, nb = G.sz3g_compress(gp, xd.data_ptr(), out.data_ptr(), cap, stream=G._stream_handle())
    return rc, out[:nb].cpu().numpy().tobytes() if rc == G.OK else b""


def test_unknown_injection_is_refused():
    assert G.sz3g_debug_inject(99, 0) == G.E_INVAL
    assert G.sz3g_debug_inject(G.DEBUG_WAIT_LIMIT, -1) == G.E_INVAL


def test_level_queue_wait_times_out_then_recovers():
    shapes = [(40, 36, 44), (33, 50, 29), (64, 20, 30)]
    xs = [S.grf(sh, 700 + i).astype(np.float32) for i, sh in enumerate(shapes)]
    ebs = [1e-3, 3e-4, 2e-3]
    params = [G.make_params(x.shape, eb, eb_mode=G.REL, interp=i % 2) for i, (x, eb) in enumerate(zip(xs, ebs))]
    ref = [O.compress(O.make_params(x.shape, eb, eb_mode=O.REL, interp=i % 2), x)
           for i, (x, eb) in enumerate(zip(xs, ebs))]
    ins = [torch.from_numpy(x.reshape(-1)).to(DEV) for x in xs]
    caps = [G.sz3g_compress_bound(p) for p in params]
    outs = [torch.zeros(c, dtype=torch.uint8, device=DEV) for c in caps]

    def run(stall):
        if stall:
            assert G.sz3g_debug_inject(G.DEBUG_WAIT_LIMIT, SHORT_WAIT) == G.OK
            assert G.sz3g_debug_inject(G.DEBUG_QUEUE_STALL, 0) == G.OK
        b = G.Batch(params, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], caps)
        try:
            b.set_queue(True)
            b.configure(2, 0)
            assert b.queue_info()[0]
            b.run(G._stream_handle())
            rc, nbytes, st = b.results()
        finally:
            b.close()
            G.sz3g_debug_inject(G.DEBUG_RESET)
        return rc, nbytes, st

    rc, _, st = run(True)
    assert rc == G.E_TIMEOUT and G.E_TIMEOUT in st
    rc, nbytes, st = run(False)
    assert rc == G.OK and all(v == G.OK for v in st)
    assert [o[:n].cpu().numpy().tobytes() for o, n in zip(outs, nbytes)] == ref


def test_encoder_lookback_times_out_then_recovers():
    # 48^3 codes in 4096-code chunks: 27 chunks, the one-pass encoder
    x = S.grf((48, 48, 48), 11).astype(np.float32)
    gp = G.make_params(x.shape, 1e-3, eb_mode=G.REL, interp=G.CUBIC)
    op = O.make_params(x.shape, 1e-3, eb_mode=O.REL, interp=O.CUBIC)
    G.sz3g_graph_cache(False)
    assert G.sz3g_debug_inject(G.DEBUG_WAIT_LIMIT, SHORT_WAIT) == G.OK
    assert G.sz3g_debug_inject(G.DEBUG_SILENT_CHUNK, 5) == G.OK
    rc, _ = _compress(gp, x)
    assert rc == G.E_TIMEOUT
    assert G.sz3g_debug_inject(G.DEBUG_RESET) == G.OK
    rc, s = _compress(gp, x)
    assert rc == G.OK and s == O.compress(op, x)


def test_refused_allocation_reports_nomem_and_keeps_nothing():
    x = S.grf((40, 44, 36), 12).astype(np.float32)
    gp = G.make_params(x.shape, 1e-3, eb_mode=G.REL, interp=G.LINEAR)
    op = O.make_params(x.shape, 1e-3, eb_mode=O.REL, interp=O.LINEAR)
    rc, s = _compress(gp, x)  # warm the library's pool
    assert rc == G.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert G.sz3g_debug_inject(G.DEBUG_ALLOC_FAIL, 1) == G.OK
    rc, _ = _compress(gp, x)
    assert rc == G.E_NOMEM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0
    # decompress without a workspace is refused the same way
    assert G.sz3g_debug_inject(G.DEBUG_ALLOC_FAIL, 1) == G.OK
    sd = torch.from_numpy(np.frombuffer(s, np.uint8).copy()).to(DEV)
    y = torch.empty(x.size, dtype=torch.float32, device=DEV)
    assert G.sz3g_decompress(sd.data_ptr(), len(s), y.data_ptr(), x.nbytes, stream=G._stream_handle()) == G.E_NOMEM
    # the next calls succeed and match the oracle
    rc, s2 = _compress(gp, x)
    assert rc == G.OK and s2 == O.compress(op, x)
    assert G.sz3g_decompress(sd.data_ptr(), len(s), y.data_ptr(), x.nbytes, stream=G._stream_handle()) == G.OK
    assert np.array_equal(y.cpu().numpy().view(np.uint32), O.decompress(s).reshape(-1).view(np.uint32))


CASES = [
    ("bumps48_lin", lambda: S.gaussian_bumps(48, 1), O.F32, O.ABS, 3e-3, O.LINEAR, (0, 1, 2), 32768, 4096),
    ("grf_ragged_cubic", lambda: S.grf((37, 50, 29), 2), O.F32, O.REL, 1e-3, O.CUBIC, (0, 1, 2), 32768, 4096),
    ("grf_order201", lambda: S.grf((33, 17, 65), 3), O.F32, O.REL, 1e-2, O.CUBIC, (2, 0, 1), 32768, 512),
    ("grf_tight_unpred", lambda: S.grf((24, 24, 24), 4), O.F32, O.REL, 1e-5, O.LINEAR, (1, 2, 0), 64, 256),
    ("latlon_cubic", lambda: S.latlon(181, 363, 5), O.F64, O.ABS, 1e-5, O.CUBIC, (1, 0), 32768, 4096),
    ("grf4d", lambda: S.grf((7, 9, 6, 10), 7), O.F32, O.REL, 1e-3, O.LINEAR, (3, 1, 0, 2), 32768, 256),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_two_runs_give_the_same_bytes(case):
    _, make, dt, mode, eb, interp, order, radius, chunk = case
    x = make()
    x = x.astype(np.float64 if dt == O.F64 else np.float32)
    kw = dict(dtype=dt, eb_mode=mode, interp=interp, order=order, radius=radius, chunk=chunk)
    gp = G.make_params(x.shape, eb, **kw)
    first = _compress(gp, x)
    second = _compress(gp, x)
    assert first[0] == second[0] == G.OK and first[1] == second[1]
    assert first[1] == O.compress(O.make_params(x.shape, eb, **kw), x)
    sd = torch.from_numpy(np.frombuffer(first[1], np.uint8).copy()).to(DEV)
    t = torch.float64 if dt == O.F64 else torch.float32
    outs = []
    for _ in range(2):
        y = torch.full((x.size,), float("nan"), dtype=t, device=DEV)
        assert G.sz3g_decompress(sd.data_ptr(), len(first[1]), y.data_ptr(), x.size * y.element_size(),
                                 stream=G._stream_handle()) == G.OK
        outs.append(y.cpu().numpy().view(np.uint8).copy())
    assert np.array_equal(outs[0], outs[1])
