"""Pins of the oracle's stream layout and its validation (SZ3 paper Alg. 1
lines 5-9: save the predictor (nothing: constant coefficients), the
quantizer's unpredictable values, the Huffman codes and the encoder's tree).

The header and section offsets are read back here with `struct`, byte by
byte, from the written layout; corrupted and truncated streams must give an
error status, never a crash.
"""
import struct

import numpy as np
import pytest

import oracle as O
from paper_2111_02925_gb300 import synthetic as S


def _pad8(x):
    return (x + 7) & ~7


def parse(stream: bytes):
    h = {}
    assert stream[:4] == b"SZ3G"
    (h["version"],) = struct.unpack_from("<H", stream, 4)
    h["dtype"], h["ndim"] = stream[6], stream[7]
    h["dims"] = list(struct.unpack_from("<4Q", stream, 8))
    h["eb_mode"], h["interp"], h["per_level"], h["L"] = stream[40:44]
    (h["radius"],) = struct.unpack_from("<I", stream, 44)
    h["eb"], h["eb_abs"] = struct.unpack_from("<2d", stream, 48)
    (h["ebT_bits"],) = struct.unpack_from("<Q", stream, 64)
    h["chunk"], h["n_used"] = struct.unpack_from("<2I", stream, 72)
    h["n_codes"], h["n_unpred"], h["n_chunks"], h["n_words"] = struct.unpack_from("<4Q", stream, 80)
    esz = 4 if h["dtype"] == 0 else 8
    off = 288
    h["off_unpred"] = off
    off += _pad8(h["n_unpred"] * esz)
    h["off_table"] = off
    off += _pad8(h["n_used"] * 3)
    h["off_chunks"] = off
    off += _pad8(h["n_chunks"] * 4)
    h["n_sub"] = h["n_chunks"] * ((h["chunk"] + 511) // 512 - 1)
    h["off_sub"] = off
    off += _pad8(h["n_sub"] * 2)
    h["off_payload"] = off
    off += _pad8(h["n_words"] * 4)
    h["end"] = off
    return h


@pytest.mark.parametrize("dtype", [O.F32, O.F64])
def test_header_and_sections(dtype):
    t = np.float32 if dtype == O.F32 else np.float64
    x = S.grf((30, 20, 17), 1).astype(t)
    x[3, 4, 5] = 50.0  # beyond radius * 2 eb: a certain unpredictable
    p = O.make_params(x.shape, 1e-3, dtype=dtype, eb_mode=O.REL, interp=O.CUBIC, order=(2, 0, 1), chunk=2048,
                      radius=64)
    s = O.compress(p, x)
    h = parse(s)
    assert h["version"] == 1 and h["dtype"] == dtype and h["ndim"] == 3
    assert h["dims"] == [30, 20, 17, 1]
    assert (h["eb_mode"], h["interp"], h["per_level"], h["L"]) == (O.REL, O.CUBIC, 0, 5)
    assert h["radius"] == 64 and h["chunk"] == 2048 and h["eb"] == 1e-3
    assert list(s[272:275]) == [2, 0, 1]
    codes, unpred, recon, ebT = O.quantize(p, x)
    assert h["n_codes"] == x.size and h["n_unpred"] == unpred.size and unpred.size >= 1
    assert h["n_chunks"] == (x.size + 2047) // 2048
    assert h["end"] == len(s)
    ebT_bits = np.array([ebT], t).view(np.uint32 if dtype == O.F32 else np.uint64)[0]
    assert h["ebT_bits"] == int(ebT_bits)
    assert h["eb_abs"] == 1e-3 * (float(x.max()) - float(x.min()))
    got_unpred = np.frombuffer(s, t, count=h["n_unpred"], offset=h["off_unpred"])
    assert np.array_equal(got_unpred, unpred)
    # code-length table: (u16 symbol, u8 length), increasing symbols
    tab = [struct.unpack_from("<HB", s, h["off_table"] + 3 * i) for i in range(h["n_used"])]
    hist = O.histogram(codes)
    ln = O.huffman_lengths(hist)
    assert [a for a, _ in tab] == np.flatnonzero(hist).tolist()
    assert [b for _, b in tab] == ln[np.flatnonzero(hist)].tolist()
    cw = np.frombuffer(s, np.uint32, count=h["n_chunks"], offset=h["off_chunks"])
    words = np.frombuffer(s, np.uint32, count=h["n_words"], offset=h["off_payload"])
    assert int(cw.sum()) == h["n_words"]
    assert np.array_equal(O.huffman_decode(words, cw, ln, x.size, 2048), codes)
    # sub-block table: bit lengths of 512-code sub-blocks 0..2 of every chunk
    sub = np.frombuffer(s, np.uint16, count=h["n_sub"], offset=h["off_sub"]).reshape(h["n_chunks"], 3)
    for j in range(h["n_chunks"]):
        for b in range(3):
            blk = codes[j * 2048 + b * 512: min(j * 2048 + (b + 1) * 512, x.size)]
            assert sub[j, b] == int(np.sum(ln[blk].astype(np.int64)))
    # padding bytes are zero
    assert s[275:288] == bytes(13)
    rp, n = O.read_header(s)
    assert n == x.size and rp.eb_mode == O.REL and list(rp.dims) == [30, 20, 17, 1]


def test_per_level_fields():
    x = S.grf((16, 16, 16), 2)
    lo = {1: (2, 1, 0), 2: (0, 1, 2), 3: (1, 2, 0), 4: (2, 0, 1)}
    li = {1: O.CUBIC, 2: O.LINEAR, 3: O.CUBIC, 4: O.LINEAR}
    p = O.make_params(x.shape, 1e-3, eb_mode=O.REL, level_interp=li, level_order=lo)
    s = O.compress(p, x)
    assert s[42] == 1 and s[43] == 4
    assert list(s[112:112 + 6]) == [0, O.CUBIC, O.LINEAR, O.CUBIC, O.LINEAR, 0]
    for l in range(1, 5):
        assert list(s[144 + 4 * l:144 + 4 * l + 3]) == list(lo[l])
    y = O.decompress(s)
    assert np.array_equal(y, O.quantize(p, x)[2])


def test_corrupt_and_truncated_streams_are_rejected():
    x = S.grf((20, 20, 20), 5)
    p = O.make_params(x.shape, 1e-3, eb_mode=O.REL, chunk=1024)
    s = bytearray(O.compress(p, x))
    out = np.zeros(x.size, np.float32)
    assert O.decompress_status(bytes(s), out) == O.OK
    assert O.decompress_status(bytes(s), np.zeros(x.size - 1, np.float32)) == O.E_CAPACITY
    for cut in (0, 10, 287, 288, len(s) // 2, len(s) - 1):
        assert O.decompress_status(bytes(s[:cut]), out) == O.E_CORRUPT
    h = parse(bytes(s))

    def flip(off, val):
        b = bytearray(s)
        b[off] = val
        return bytes(b)

    assert O.decompress_status(flip(0, ord("X")), out) == O.E_CORRUPT  # magic
    assert O.decompress_status(flip(4, 2), out) == O.E_CORRUPT  # version
    assert O.decompress_status(flip(6, 7), out) == O.E_CORRUPT  # dtype
    assert O.decompress_status(flip(43, 9), out) == O.E_CORRUPT  # level count
    b = bytearray(s)
    struct.pack_into("<I", b, h["off_chunks"], struct.unpack_from("<I", s, h["off_chunks"])[0] + 1)
    assert O.decompress_status(bytes(b), out) == O.E_CORRUPT  # chunk words no longer sum
    b = bytearray(s)
    b[h["off_table"] + 2] = 30  # a length above the limit
    assert O.decompress_status(bytes(b), out) == O.E_CORRUPT
    b = bytearray(s)
    struct.pack_into("<H", b, h["off_sub"], struct.unpack_from("<H", s, h["off_sub"])[0] + 1)
    assert O.decompress_status(bytes(b), out) == O.E_CORRUPT  # sub-block boundary moved
    b = bytearray(s)
    struct.pack_into("<Q", b, 64, 0)  # eb_T = 0
    assert O.decompress_status(bytes(b), out) == O.E_CORRUPT
    # flipping payload bits either still decodes (and stays within the alphabet)
    # or is reported; it never crashes
    rng = np.random.default_rng(0)
    for _ in range(30):
        b = bytearray(s)
        i = int(rng.integers(h["off_payload"], h["end"]))
        b[i] ^= 1 << int(rng.integers(8))
        assert O.decompress_status(bytes(b), out) in (O.OK, O.E_CORRUPT)
