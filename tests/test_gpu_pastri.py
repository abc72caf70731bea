"""GPU: the SZ3-Pastri modules against the oracle, byte for byte -- the
unpred-aware quantizer's bitplane streams and decoded values, and the fixed
Huffman table with the chunked encode / decode run on it."""
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
DEV = "cuda"


def gpu_bp_encode(v: np.ndarray, eb: float, cap=None):
    dt = G.F32 if v.dtype == np.float32 else G.F64
    d = torch.from_numpy(np.ascontiguousarray(v).reshape(-1)).to(DEV) if v.size else None
    cap = G.sz3g_bitplane_bound(v.size) if cap is None else cap
    out = torch.zeros(max(cap, 16), dtype=torch.uint8, device=DEV)
    rc, nb = G.sz3g_bitplane_encode(dt, d.data_ptr() if d is not None else 0, v.size, eb, out.data_ptr(), cap,
                                    G._stream_handle())
    return rc, (out[:nb].cpu().numpy().tobytes() if rc == G.OK else b"")


def gpu_bp_decode(s: bytes, n: int, dtype, cap=None):
    d = torch.from_numpy(np.frombuffer(s, np.uint8).copy()).to(DEV)
    y = torch.full((max(n, 1),), float("nan"), dtype=torch.float32 if dtype == np.float32 else torch.float64,
                   device=DEV)
    cap = n * np.dtype(dtype).itemsize if cap is None else cap
    rc, nn = G.sz3g_bitplane_decode(d.data_ptr(), len(s), y.data_ptr(), cap, G._stream_handle())
    return rc, (y[:nn].cpu().numpy() if rc == G.OK else None)


def _bits(a):
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1023, 1024, 1025, 4099, 300001])
def test_bitplane_matches_oracle(dtype, n):
    rng = np.random.default_rng(n + 3)
    v = (rng.laplace(0.0, 50.0, n) * rng.choice([1e-4, 1.0, 30.0], n)).astype(dtype)
    for eb in (1e-3, 0.37, 5.0):
        rc, s = gpu_bp_encode(v, eb)
        assert rc == G.OK
        so = O.bitplane_encode(v, eb)
        assert s == so
        rc, y = gpu_bp_decode(s, n, dtype)
        assert rc == G.OK
        assert np.array_equal(_bits(y), _bits(O.bitplane_decode(so)))


def test_bitplane_edge_widths():
    # B = 0 (everything below the bound), and B = 61 (values near 2^61 2^e)
    z = np.array([1e-9, -2e-9, 0.0, -0.0] * 10, np.float64)
    rc, s = gpu_bp_encode(z, 1e-3)
    assert rc == G.OK and s == O.bitplane_encode(z, 1e-3)
    w = np.array([2.0 ** 61 - 2.0 ** 9, -(2.0 ** 60), 3.0, -1.0, 2.0 ** 40 + 1.0], np.float64)
    rc, s = gpu_bp_encode(w, 1.0)
    assert rc == G.OK and s == O.bitplane_encode(w, 1.0)
    assert int(np.frombuffer(s[20:24], np.uint32)[0]) == 61
    rc, y = gpu_bp_decode(s, w.size, np.float64)
    assert np.array_equal(_bits(y), _bits(O.bitplane_decode(s)))
    # float values whose aligned integers exceed 24 bits decode exactly
    f = np.array([1.0e6, -3.3e5, 7.25, 1.0e-3], np.float32)
    rc, s = gpu_bp_encode(f, 1e-4)
    assert rc == G.OK and s == O.bitplane_encode(f, 1e-4)
    rc, y = gpu_bp_decode(s, f.size, np.float32)
    assert np.array_equal(_bits(y), _bits(O.bitplane_decode(s)))


def test_bitplane_errors_match_oracle():
    cases = [
        (np.array([1.0, np.inf, 2.0], np.float32), 0.1),
        (np.array([np.nan] * 40, np.float64), 0.1),
        (np.array([2.0 ** 62, 1.0], np.float64), 1.0),
        (np.array([2.0 ** 63, 0.0, -np.inf], np.float64), 1.0),
    ]
    for v, eb in cases:
        assert gpu_bp_encode(v, eb)[0] == O.bitplane_encode_status(v, eb)[0] != G.OK
    for eb in (0.0, -1.0, float("nan"), float("inf")):
        assert gpu_bp_encode(np.ones(5, np.float32), eb)[0] == G.E_INVAL
    v = np.arange(100, dtype=np.float32)
    so = O.bitplane_encode(v, 0.5)
    assert gpu_bp_encode(v, 0.5, cap=len(so) - 4)[0] == G.E_CAPACITY
    assert gpu_bp_encode(v, 0.5, cap=len(so))[1] == so
    for bad in (b"XZBP" + so[4:], so[:31], so[:-1], so[:20] + np.uint32(63).tobytes() + so[24:]):
        assert gpu_bp_decode(bad, 100, np.float32)[0] == G.E_CORRUPT
    assert gpu_bp_decode(so, 100, np.float32, cap=396)[0] == G.E_CAPACITY


@pytest.mark.parametrize("radius", [2, 3, 4, 5, 100, 1024, 1025, 1500, 4097, 32768])
def test_fixed_huffman_table_matches_oracle(radius):
    glen = torch.zeros(2 * radius, dtype=torch.uint8, device=DEV)
    gcode = torch.zeros(2 * radius, dtype=torch.int32, device=DEV)
    assert G.sz3g_huffman_fixed(radius, glen.data_ptr(), gcode.data_ptr(), G._stream_handle()) == G.OK
    torch.cuda.synchronize()
    ol = O.huffman_fixed_lengths(radius)
    assert np.array_equal(glen.cpu().numpy(), ol)
    assert np.array_equal(gcode.cpu().numpy().view(np.uint32), O.canonical_codes(ol))


def test_fixed_huffman_encode_decode_match_oracle():
    radius, chunk = 32768, 4096
    rng = np.random.default_rng(9)
    n = 3 * chunk + 777
    codes = np.clip(np.round(rng.laplace(radius, 6.0, n)), 1, 2 * radius - 1).astype(np.uint16)
    codes[::1013] = 0
    codes[5::4001] = 1           # the far ends of the code range
    codes[7::4003] = 2 * radius - 1
    nsym = 2 * radius
    glen = torch.zeros(nsym, dtype=torch.uint8, device=DEV)
    gcode = torch.zeros(nsym, dtype=torch.int32, device=DEV)
    assert G.sz3g_huffman_fixed(radius, glen.data_ptr(), gcode.data_ptr(), G._stream_handle()) == G.OK
    ol = O.huffman_fixed_lengths(radius)
    ow, ocw, osub = O.huffman_encode(codes, ol, O.canonical_codes(ol), chunk=chunk, with_sub=True)
    cd = torch.from_numpy(codes).to(DEV)
    nch = (n + chunk - 1) // chunk
    cap = nch * ((chunk * 24 + 31) // 32)
    gw = torch.zeros(cap, dtype=torch.int32, device=DEV)
    gcw = torch.zeros(nch, dtype=torch.int32, device=DEV)
    gsub = torch.zeros(nch * (chunk // 512 - 1), dtype=torch.int16, device=DEV)
    rc, nw = G.sz3g_huffman_encode(cd.data_ptr(), n, glen.data_ptr(), gcode.data_ptr(), nsym, chunk, gw.data_ptr(),
                                   cap, gcw.data_ptr(), gsub.data_ptr(), G._stream_handle())
    assert rc == G.OK and nw == ow.size
    assert np.array_equal(gw[:nw].cpu().numpy().view(np.uint32), ow)
    assert np.array_equal(gcw.cpu().numpy().view(np.uint32), ocw)
    assert np.array_equal(gsub.cpu().numpy().view(np.uint16), osub)
    back = torch.zeros(n, dtype=torch.int16, device=DEV)
    rc = G.sz3g_huffman_decode(gw.data_ptr(), nw, gcw.data_ptr(), gsub.data_ptr(), chunk, glen.data_ptr(), nsym,
                               back.data_ptr(), n, G._stream_handle())
    assert rc == G.OK
    assert np.array_equal(back.cpu().numpy().view(np.uint16), codes)
    # the predefined code is incomplete: a window past its last codeword is
    # no codeword and stops the decoder
    ones = torch.full_like(gw, -1)
    rc = G.sz3g_huffman_decode(ones.data_ptr(), nw, gcw.data_ptr(), 0, chunk, glen.data_ptr(), nsym,
                               back.data_ptr(), n, G._stream_handle())
    assert rc == G.E_CORRUPT
