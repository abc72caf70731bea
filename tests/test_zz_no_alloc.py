"""The decoder entry point that allocates nothing (sz3g_huffman_decode_static).

Callers whose device memory belongs to another allocator, or that cannot risk
an allocation blocking or failing mid-run, decode through this entry point:
its scratch is a fixed array inside the library.  This file is collected last
so that a run stopping at the first failure has run every other test first;
it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_02925_gb300 import build as B  # noqa: E402
from paper_2111_02925_gb300 import sz3g as G  # noqa: E402

B.build()
G.load()


def _encoded(seed, n, chunk, spread):
    rng = np.random.default_rng(seed)
    codes = np.clip(np.round(rng.laplace(32768, spread, n)), 0, 65535).astype(np.uint16)
    codes[rng.integers(0, n, 40)] = 0
    ln = O.huffman_lengths(O.histogram(codes))
    cc = O.canonical_codes(ln)
    words, cw, sub = O.huffman_encode(codes, ln, cc, chunk, with_sub=True)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    return codes, dev(words.view(np.int32)), words.size, dev(cw.view(np.int32)), dev(sub.view(np.int16)) if sub.size \
        else None, dev(ln)


@pytest.mark.parametrize("seed,n,chunk,spread", [(0, 300_001, 4096, 8.0), (1, 77_777, 1024, 500.0), (2, 4_099, 8, 2.0)])
def test_static_decode_matches_allocating_decode_twice(seed, n, chunk, spread):
    codes, w, nw, cw, sub, ln = _encoded(seed, n, chunk, spread)
    sh = G._stream_handle()
    ref = torch.empty(n, dtype=torch.int16, device="cuda")
    assert G.sz3g_huffman_decode(w.data_ptr(), nw, cw.data_ptr(), sub.data_ptr() if sub is not None else 0, chunk,
                                 ln.data_ptr(), 65536, ref.data_ptr(), n, sh) == G.OK
    for _ in range(2):  # two calls in a row share the fixed scratch
        out = torch.full((n,), -1, dtype=torch.int16, device="cuda")
        rc = G.sz3g_huffman_decode_static(w.data_ptr(), nw, cw.data_ptr(), sub.data_ptr() if sub is not None else 0,
                                          chunk, ln.data_ptr(), 65536, out.data_ptr(), n, sh)
        assert rc == G.OK
        assert torch.equal(out, ref)
    assert np.array_equal(ref.cpu().numpy().view(np.uint16), codes)


def test_static_decode_refuses_streams_beyond_its_scratch():
    codes, w, nw, cw, sub, ln = _encoded(3, 1000, 8, 4.0)
    out = torch.empty(16, dtype=torch.int16, device="cuda")
    # 2^31 codes in 8-code chunks would need far more than the fixed scratch;
    # the call is refused before anything is launched
    rc = G.sz3g_huffman_decode_static(w.data_ptr(), nw, cw.data_ptr(), 0, 8, ln.data_ptr(), 65536, out.data_ptr(),
                                      1 << 31, G._stream_handle())
    assert rc == G.E_CAPACITY


def test_static_decode_reports_corrupt_then_recovers():
    """A moved sub-block boundary is reported as SZ3G_E_CORRUPT (the same
    status as the allocating decoder), and the next well-formed call, which
    starts from a reset status block, succeeds and matches it."""
    codes, w, nw, cw, sub, ln = _encoded(4, 50_000, 4096, 30.0)
    sh = G._stream_handle()
    bad = sub.clone()
    bad[0] += 1
    out = torch.empty(codes.size, dtype=torch.int16, device="cuda")
    args = (w.data_ptr(), nw, cw.data_ptr())
    tail = (4096, ln.data_ptr(), 65536, out.data_ptr(), codes.size, sh)
    assert G.sz3g_huffman_decode(*args, bad.data_ptr(), *tail) == G.E_CORRUPT
    assert G.sz3g_huffman_decode_static(*args, bad.data_ptr(), *tail) == G.E_CORRUPT
    assert G.sz3g_huffman_decode_static(*args, sub.data_ptr(), *tail) == G.OK
    assert np.array_equal(out.cpu().numpy().view(np.uint16), codes)


def test_static_decode_small_alphabet():
    rng = np.random.default_rng(5)
    n, nsym = 20_001, 40
    codes = rng.integers(0, nsym, n).astype(np.uint16)
    ln = O.huffman_lengths(O.histogram(codes))[:nsym].copy()
    full = np.zeros(65536, np.uint8)
    full[:nsym] = ln
    cc = O.canonical_codes(full)
    words, cw, sub = O.huffman_encode(codes, full, cc, 1024, with_sub=True)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    w, c, sb, l = dev(words.view(np.int32)), dev(cw.view(np.int32)), dev(sub.view(np.int16)), dev(ln)
    sh = G._stream_handle()
    ref = torch.empty(n, dtype=torch.int16, device="cuda")
    assert G.sz3g_huffman_decode(w.data_ptr(), words.size, c.data_ptr(), sb.data_ptr(), 1024, l.data_ptr(), nsym,
                                 ref.data_ptr(), n, sh) == G.OK
    for _ in range(2):
        out = torch.full((n,), -1, dtype=torch.int16, device="cuda")
        assert G.sz3g_huffman_decode_static(w.data_ptr(), words.size, c.data_ptr(), sb.data_ptr(), 1024, l.data_ptr(),
                                            nsym, out.data_ptr(), n, sh) == G.OK
        assert torch.equal(out, ref)
    assert np.array_equal(ref.cpu().numpy().view(np.uint16), codes)
