"""The lossless stage's oracle (oracle/szlz.c) against a hand-worked parse, a
closed form, the stream layout, round trips and a strict decoder."""
import json
import os
import struct

import numpy as np

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _payload(stream, b=0):
    n, nb = struct.unpack_from("<QI", stream, 8)
    sizes = struct.unpack_from(f"<{nb}I", stream, 24)
    k = (24 + 4 * nb + 7) & ~7
    for i in range(b):
        k += ((sizes[i] & 0x7FFFFFFF) + 3) & ~3
    return sizes[b], stream[k:k + (sizes[b] & 0x7FFFFFFF)]


def test_hand_worked_parse():
    g = json.load(open(os.path.join(HERE, "golden", "lz_abc.json")))
    s = O.lz_compress(g["input_ascii"].encode())
    size, pay = _payload(s)
    assert size == g["payload_len"] and pay.hex() == g["payload_hex"]
    assert O.lz_decompress(s) == g["input_ascii"].encode()


def test_zero_block_closed_form():
    # position 0 has no candidate; position 1's is 0: one literal, then a match
    # at distance 1 of the remaining 32767 bytes (length - 4 - 15 = 32748 =
    # 128 x 255 + 108 in extension bytes), then the empty final sequence
    s = O.lz_compress(bytes(32768))
    size, pay = _payload(s)
    want = bytes([0x1F, 0x00, 0x01, 0x00] + [255] * 128 + [108, 0x00])
    assert size == len(want) and pay == want


def test_layout_and_raw_blocks():
    rng = np.random.default_rng(5)
    data = rng.integers(0, 256, 3 * 32768 + 1000, dtype=np.uint8).tobytes()
    s = O.lz_compress(data)
    assert s[:4] == b"SZLZ"
    bs, n, nb = struct.unpack_from("<IQI", s, 4)
    assert (bs, n, nb) == (32768, len(data), 4)
    sizes = struct.unpack_from("<4I", s, 24)
    # random bytes do not compress: every block stored raw with its length
    assert [v & 0x7FFFFFFF for v in sizes] == [32768, 32768, 32768, 1000]
    assert all(v & 0x80000000 for v in sizes)
    assert len(s) == ((24 + 16 + 7) & ~7) + 3 * 32768 + 1000


def test_round_trips():
    rng = np.random.default_rng(6)
    cases = [b"", b"x", b"xyzw", b"aaaaaaa", bytes(32767), bytes(32768), bytes(32769), bytes(100003),
             (b"the quick brown fox " * 3000), rng.integers(0, 3, 70001, dtype=np.uint8).tobytes(),
             bytes(rng.integers(0, 256, 20, dtype=np.uint8)) * 4000,
             np.repeat(rng.integers(0, 256, 5000, dtype=np.uint8), rng.integers(1, 40, 5000)).tobytes()]
    for d in cases:
        s = O.lz_compress(d)
        assert O.lz_decompress(s) == d
        # coded blocks never exceed the raw size
        assert len(s) <= ((24 + 4 * ((len(d) + 32767) // 32768) + 7) & ~7) + len(d) + 3 * ((len(d) + 32767) // 32768)


def test_decoder_rejects_corrupt_streams():
    d = b"abcabcabcabc" * 100
    s = bytearray(O.lz_compress(d))
    assert O.lz_decompress_status(bytes(s), len(d))[0] == O.OK
    assert O.lz_decompress_status(bytes(s), len(d) - 1)[0] == O.E_CAPACITY
    bad = bytearray(s)
    bad[0] = ord("X")
    assert O.lz_decompress_status(bytes(bad), len(d))[0] == O.E_CORRUPT
    size, pay = _payload(bytes(s))
    k = (24 + 4 + 7) & ~7
    # the first match's distance (after token and 3 literals) set to 0, then past the output
    for off in (b"\x00\x00", b"\x10\x00"):
        bad = bytearray(s)
        bad[k + 4:k + 6] = off
        assert O.lz_decompress_status(bytes(bad), len(d))[0] == O.E_CORRUPT
    # truncated payload
    bad = bytearray(s)
    struct.pack_into("<I", bad, 24, size - 2)
    assert O.lz_decompress_status(bytes(bad), len(d))[0] == O.E_CORRUPT
