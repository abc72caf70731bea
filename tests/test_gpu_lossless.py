"""GPU: the lossless stage against the oracle -- the same bytes for every
input, round trips, and corrupt streams rejected."""
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


def _dev(b: bytes):
    t = torch.zeros(max(len(b), 1) + 16, dtype=torch.uint8, device=DEV)
    if b:
        t[: len(b)] = torch.from_numpy(np.frombuffer(b, np.uint8).copy()).to(DEV)
    return t


def gpu_lz(data: bytes) -> bytes:
    src = _dev(data)
    cap = G.sz3g_lossless_bound(len(data))
    out = torch.zeros(cap + 16, dtype=torch.uint8, device=DEV)
    rc, nb = G.sz3g_lossless_compress(src.data_ptr(), len(data), out.data_ptr(), cap, G._stream_handle())
    assert rc == G.OK
    return out[:nb].cpu().numpy().tobytes()


def gpu_unlz(stream: bytes, cap: int):
    src = _dev(stream)
    out = torch.full((max(cap, 1) + 16,), 0xAB, dtype=torch.uint8, device=DEV)
    rc, n = G.sz3g_lossless_decompress(src.data_ptr(), len(stream), out.data_ptr(), cap, G._stream_handle())
    return rc, (out[:n].cpu().numpy().tobytes() if rc == G.OK else b"")


def _inputs():
    rng = np.random.default_rng(11)
    x = S.latlon(180, 360, seed=3).astype(np.float64)
    op = O.make_params(x.shape, 1e-6 * (float(x.max()) - float(x.min())), dtype=O.F64, eb_mode=O.ABS,
                       interp=O.CUBIC)
    return [
        b"", b"q", b"abcd", b"abcabcabcabc", bytes(32768), bytes(32769), bytes(100003),
        rng.integers(0, 256, 70001, dtype=np.uint8).tobytes(),
        b"the quick brown fox jumps over the lazy dog " * 2000,
        rng.integers(0, 3, 65536 + 77, dtype=np.uint8).tobytes(),
        np.repeat(rng.integers(0, 256, 9000, dtype=np.uint8), rng.integers(1, 60, 9000)).tobytes(),
        bytes(rng.integers(0, 256, 13, dtype=np.uint8)) * 9000,
        O.compress(op, x),  # a stream of the compressor itself
    ]


@pytest.mark.parametrize("case", range(13))
def test_lossless_matches_oracle_and_round_trips(case):
    data = _inputs()[case]
    s = gpu_lz(data)
    assert s == O.lz_compress(data)
    rc, back = gpu_unlz(s, len(data))
    assert rc == G.OK and back == data


def test_lossless_rejects_corrupt_streams():
    d = b"abcabcabcabc" * 3000
    s = bytearray(O.lz_compress(d))
    assert gpu_unlz(bytes(s), len(d))[0] == G.OK
    assert gpu_unlz(bytes(s), len(d) - 1)[0] == G.E_CAPACITY
    bad = bytearray(s)
    bad[0] = ord("X")
    assert gpu_unlz(bytes(bad), len(d))[0] == G.E_CORRUPT
    k = (24 + 4 * 2 + 7) & ~7
    for off in (b"\x00\x00", b"\x10\x00"):  # the first match's distance: zero, then past the output
        bad = bytearray(s)
        bad[k + 4:k + 6] = off
        assert gpu_unlz(bytes(bad), len(d))[0] == G.E_CORRUPT
    size = struct.unpack_from("<I", s, 24)[0]
    bad = bytearray(s)
    struct.pack_into("<I", bad, 24, size - 2)  # a truncated payload
    assert gpu_unlz(bytes(bad), len(d))[0] == G.E_CORRUPT
    bad = bytearray(s)
    struct.pack_into("<I", bad, 24, 0x80000000 | 100)  # a raw block of the wrong length
    assert gpu_unlz(bytes(bad), len(d))[0] == G.E_CORRUPT
    assert gpu_unlz(bytes(s[:20]), len(d))[0] == G.E_CORRUPT
