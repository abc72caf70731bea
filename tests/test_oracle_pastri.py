"""Pins of the oracle's SZ3-Pastri modules (no GPU): the unpred-aware
quantizer (Sec. 4.2, values aligned to the bound's exponent and stored by
bitplane) and the fixed Huffman code (Sec. 3.2 Encoder, a predefined tree).

Each check is independent of the oracle's own arithmetic: hand-worked
fixtures, the bound 2^e <= eb < 2^(e+1), numpy's own truncation and bit
unpacking, Kraft sums and prefix-freedom by enumeration."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _words(stream: bytes) -> np.ndarray:
    return np.frombuffer(stream[O.BP_HEADER:], np.uint32)


def _header(stream: bytes):
    magic = stream[:4]
    dtype, = np.frombuffer(stream[4:8], np.uint32)
    n, = np.frombuffer(stream[8:16], np.uint64)
    e, = np.frombuffer(stream[16:20], np.int32)
    B, = np.frombuffer(stream[20:24], np.uint32)
    W, = np.frombuffer(stream[24:32], np.uint64)
    return magic, int(dtype), int(n), int(e), int(B), int(W)


def _unpack(stream: bytes):
    """Signed integers from the planes, by numpy bit unpacking."""
    magic, dtype, n, e, B, W = _header(stream)
    w = _words(stream).reshape(1 + B, W) if W else np.zeros((1 + B, 0), np.uint32)
    bits = np.unpackbits(w.view(np.uint8).reshape(1 + B, W, 4), axis=2, bitorder="little").reshape(1 + B, W * 32)
    bits = bits[:, :n].astype(np.uint64)
    mag = np.zeros(n, np.uint64)
    for p in range(1, 1 + B):  # plane p holds bit B - p
        mag |= bits[p] << np.uint64(B - p)
    sign = bits[0].astype(bool)
    return sign, mag, bits


def test_bitplane_hand_worked_example():
    g = json.load(open(os.path.join(GOLD, "bitplane_small.json")))
    v = np.array(g["values"], np.float32)
    s = O.bitplane_encode(v, g["eb"])
    magic, dtype, n, e, B, W = _header(s)
    assert (magic, dtype, n, e, B, W) == (b"SZBP", O.F32, v.size, g["e"], g["B"], 1)
    assert _words(s).tolist() == g["words"]
    assert O.bitplane_decode(s).tolist() == g["decoded"]


@pytest.mark.parametrize("eb", [0.5, 1.0, 0.7, 1e-3, 3.0, 2.0 ** -30, 1e-310, 1e300, 12345.678])
def test_bitplane_exponent_brackets_the_bound(eb):
    e = O.bitplane_exponent(eb)
    assert math.ldexp(1.0, e) <= eb < math.ldexp(1.0, e + 1)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1000, 4099])
def test_bitplane_values_bound_and_planes(dtype, n):
    rng = np.random.default_rng(n + 7)
    v = (rng.laplace(0.0, 40.0, n) * rng.choice([1e-3, 1.0, 1e3], n)).astype(dtype)
    eb = 0.013
    s = O.bitplane_encode(v, eb)
    magic, dt, nn, e, B, W = _header(s)
    assert nn == n and W == (n + 31) // 32
    assert len(s) == O.BP_HEADER + 4 * W * (1 + B)
    q = np.trunc(v.astype(np.float64) / 2.0 ** e)
    assert B == (int(np.abs(q).max()).bit_length() if n else 0)
    sign, mag, bits = _unpack(s)
    assert np.array_equal(mag, np.abs(q).astype(np.uint64))
    assert np.array_equal(sign, q < 0)
    # bits past n are zero in every plane
    w = _words(s).reshape(1 + B, W) if W else np.zeros((1 + B, 0), np.uint32)
    full = np.unpackbits(w.view(np.uint8).reshape(1 + B, W, 4), axis=2, bitorder="little").reshape(1 + B, -1)
    assert not full[:, n:].any()
    y = O.bitplane_decode(s)
    assert y.dtype == dtype and y.size == n
    assert np.array_equal(y.astype(np.float64), q * 2.0 ** e)
    assert np.all(np.abs(y.astype(np.float64) - v.astype(np.float64)) < 2.0 ** e)
    assert 2.0 ** e <= eb


def test_bitplane_all_zero_and_tiny_values_have_no_planes():
    v = np.array([0.0, -0.0, 1e-9, -3e-4], np.float64)
    s = O.bitplane_encode(v, 1e-3)
    assert _header(s)[4] == 0 and len(s) == O.BP_HEADER + 4
    assert _words(s).tolist() == [0]
    assert O.bitplane_decode(s).tolist() == [0.0, 0.0, 0.0, 0.0]


def test_bitplane_errors():
    rc, _ = O.bitplane_encode_status(np.array([1.0, np.inf], np.float32), 0.1)
    assert rc == O.E_NONFINITE
    rc, _ = O.bitplane_encode_status(np.array([1.0, np.nan], np.float64), 0.1)
    assert rc == O.E_NONFINITE
    # an aligned integer of 62 bits or more
    rc, _ = O.bitplane_encode_status(np.array([2.0 ** 62], np.float64), 1.0)
    assert rc == O.E_INVAL
    # a non-finite value anywhere is reported before a too-wide one
    rc, _ = O.bitplane_encode_status(np.array([2.0 ** 63, 0.0, np.inf], np.float64), 1.0)
    assert rc == O.E_NONFINITE
    rc, _ = O.bitplane_encode_status(np.array([2.0 ** 61], np.float64), 1.0)
    assert rc == O.OK
    for eb in (0.0, -1.0, float("nan"), float("inf")):
        assert O.bitplane_encode_status(np.ones(3, np.float32), eb)[0] == O.E_INVAL
    s = O.bitplane_encode(np.arange(40, dtype=np.float32), 0.25)
    for bad in (b"XZBP" + s[4:], s[:31], s[:-1]):
        assert O.bitplane_decode_status(bad, 40, np.float32)[0] == O.E_CORRUPT
    assert O.bitplane_decode_status(s, 39, np.float32)[0] == O.E_CAPACITY


def test_fixed_huffman_hand_worked_code():
    g = json.load(open(os.path.join(GOLD, "fixed_huffman_r4.json")))
    lengths = O.huffman_fixed_lengths(g["radius"])
    assert lengths.tolist() == g["lengths"]
    assert O.canonical_codes(lengths).tolist() == g["codes"]


@pytest.mark.parametrize("radius", [2, 3, 5, 100, 1024, 1025, 2048, 5000, 32768])
def test_fixed_huffman_lengths_kraft_and_classes(radius):
    lengths = O.huffman_fixed_lengths(radius)
    assert lengths.size == 2 * radius and lengths.min() >= 1 and lengths.max() <= O.LMAX
    assert sum(2.0 ** -int(l) for l in lengths) <= 1.0
    # lengths by enumeration of the distance classes
    want = np.zeros(2 * radius, np.int64)
    want[0] = 24
    for s in range(1, 2 * radius):
        k = abs(s - radius)
        c = k.bit_length()
        want[s] = 1 if k == 0 else (2 * c + 2 if c <= 10 else 24)
    assert np.array_equal(lengths.astype(np.int64), want)


def test_fixed_huffman_prefix_free_and_round_trip():
    radius = 1200
    lengths = O.huffman_fixed_lengths(radius)
    canon = O.canonical_codes(lengths)
    words = sorted(format(int(c), f"0{int(l)}b") for c, l in zip(canon, lengths))
    assert len(set(words)) == len(words)
    assert all(not b.startswith(a) for a, b in zip(words, words[1:]))
    rng = np.random.default_rng(5)
    codes = np.clip(np.round(rng.laplace(radius, 3.0, 20000)), 0, 2 * radius - 1).astype(np.uint16)
    codes[::997] = 0
    w, cw = O.huffman_encode(codes, lengths, canon, chunk=1024)[:2]
    back = O.huffman_decode(w, cw, lengths, codes.size, chunk=1024)
    assert np.array_equal(back, codes)
    # the predefined code costs its lengths, nothing for a stored table
    assert int(cw.sum()) * 32 >= int(lengths[codes].astype(np.int64).sum())
