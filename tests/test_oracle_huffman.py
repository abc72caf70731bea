"""Pins of the oracle's Huffman stage (SZ3 paper Sec. 3.2 Encoder: a Huffman
tree built greedily from the symbol frequencies, a codebook generated from the
tree, the codes encoded with it; decode reverses it).

Independent checks: a hand-built example, the Kraft equality of a full binary
tree, the total bit count of a textbook heap-based Huffman (any optimal prefix
code has the same total), exhaustive minimality over all prefix-code length
vectors for up to 6 symbols, and encode/decode round trips with per-chunk word
counts recomputed here from the lengths.
"""
import heapq
import itertools
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def textbook_total(freqs):
    """Total bits of a Huffman code built with a binary heap."""
    f = [int(v) for v in freqs if v > 0]
    if len(f) == 1:
        return f[0]
    h = list(f)
    heapq.heapify(h)
    total = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        total += a + b
        heapq.heappush(h, a + b)
    return total


def test_golden_four_symbols():
    g = json.load(open(os.path.join(GOLD, "huffman_4sym.json")))
    freq = np.zeros(32, np.uint64)
    freq[g["symbols"]] = g["freq"]
    ln = O.huffman_lengths(freq)
    assert ln[g["symbols"]].tolist() == g["lengths"]
    assert int(ln.sum()) == sum(g["lengths"])
    cc = O.canonical_codes(ln)
    assert cc[g["symbols"]].tolist() == g["codes"]
    words, cw = O.huffman_encode(np.array(g["stream"], np.uint16), ln, cc, chunk=8)
    assert words.tolist() == g["words"] and cw.tolist() == [1]


def test_golden_tie_rule():
    g = json.load(open(os.path.join(GOLD, "huffman_tie.json")))
    ln = O.huffman_lengths(np.array(g["freq"], np.uint64))
    assert ln.tolist() == g["lengths"]
    assert O.canonical_codes(ln).tolist() == g["codes"]


def _kraft(ln):
    return sum(Fr(1, 2 ** int(l)) for l in ln if l > 0)


@pytest.mark.parametrize("seed", range(8))
def test_kraft_and_optimal_total(seed):
    rng = np.random.default_rng(seed)
    nsym = int(rng.integers(2, 3000))
    freq = np.zeros(65536, np.uint64)
    kind = seed % 3
    syms = rng.choice(65536, nsym, replace=False)
    if kind == 0:
        f = rng.integers(1, 1000, nsym)
    elif kind == 1:  # geometric, like quantization codes around the radius
        f = np.maximum(1, (1e6 * 0.7 ** np.arange(nsym)).astype(np.int64))
    else:  # many ties
        f = rng.integers(1, 4, nsym)
    freq[syms] = f
    ln = O.huffman_lengths(freq)
    assert np.all((ln > 0) == (freq > 0))
    assert _kraft(ln) == 1
    unlimited = O.huffman_lengths(freq, 32)
    if unlimited.max() <= O.LMAX:  # the limit did not bite: an optimal code
        assert np.array_equal(ln, unlimited)
        total = int(np.sum(ln.astype(np.int64) * freq.astype(np.int64)))
        assert total == textbook_total(freq)
    else:
        assert ln.max() <= O.LMAX


def test_exhaustive_minimality_small_alphabets():
    rng = np.random.default_rng(2)
    for trial in range(60):
        k = int(rng.integers(2, 7))
        f = rng.integers(1, 50, k)
        freq = np.zeros(k, np.uint64)
        freq[:] = f
        ln = O.huffman_lengths(freq)
        got = int(np.sum(ln.astype(np.int64) * f))
        best = None
        for lens in itertools.product(range(1, k), repeat=k):
            if sum(Fr(1, 2 ** l) for l in lens) <= 1:
                t = sum(a * b for a, b in zip(lens, f))
                best = t if best is None else min(best, t)
        assert got == best


def test_single_symbol_gets_length_one():
    freq = np.zeros(65536, np.uint64)
    freq[32768] = 12345
    ln = O.huffman_lengths(freq)
    assert ln[32768] == 1 and int(ln.sum()) == 1
    cc = O.canonical_codes(ln)
    assert cc[32768] == 0
    codes = np.full(10000, 32768, np.uint16)
    w, cw = O.huffman_encode(codes, ln, cc, chunk=4096)
    assert cw.tolist() == [128, 128, 57]  # 4096 bits = 128 words; 1808 bits -> 57 words
    assert np.all(w == 0)
    assert np.array_equal(O.huffman_decode(w, cw, ln, codes.size, 4096), codes)


def test_length_limit():
    # Fibonacci weights force a degenerate tree of depth nsym-1 > 24
    fib = [1, 1]
    while len(fib) < 30:
        fib.append(fib[-1] + fib[-2])
    freq = np.zeros(64, np.uint64)
    freq[:30] = fib
    ln24 = O.huffman_lengths(freq, 32)
    assert ln24.max() > 24  # without a limit the tree is that deep
    ln = O.huffman_lengths(freq)
    assert ln.max() <= O.LMAX and _kraft(ln) == 1
    assert np.all((ln > 0) == (freq > 0))


def test_canonical_code_properties():
    rng = np.random.default_rng(4)
    freq = np.zeros(65536, np.uint64)
    syms = rng.choice(65536, 500, replace=False)
    freq[syms] = rng.integers(1, 10 ** 6, 500)
    ln = O.huffman_lengths(freq)
    cc = O.canonical_codes(ln)
    used = np.flatnonzero(ln)
    order = sorted(used, key=lambda s: (ln[s], s))
    bits = [format(int(cc[s]), f"0{int(ln[s])}b") for s in order]
    # prefix-free
    for a, b in zip(bits, bits[1:]):
        assert not b.startswith(a)
    srt = sorted(bits)
    for a, b in zip(srt, srt[1:]):
        assert not b.startswith(a)
    # canonical: increasing as left-aligned binary fractions, first is all zeros
    vals = [Fr(int(b, 2), 2 ** len(b)) for b in bits]
    assert vals[0] == 0 and all(x < y for x, y in zip(vals, vals[1:]))
    # consecutive: next = (prev + 1) << (growth in length)
    for (s0, s1) in zip(order, order[1:]):
        assert int(cc[s1]) == (int(cc[s0]) + 1) << int(ln[s1] - ln[s0])


@pytest.mark.parametrize("chunk", [8, 16, 4096, 1000 * 8, 520])
def test_encode_decode_round_trip(chunk):
    rng = np.random.default_rng(chunk)
    n = 50_000 + 13
    codes = np.clip(np.round(rng.laplace(32768, 6, n)), 0, 65535).astype(np.uint16)
    codes[rng.integers(0, n, 50)] = 0
    hist = O.histogram(codes)
    assert int(hist.sum()) == n and hist[32768] == np.sum(codes == 32768)
    ln = O.huffman_lengths(hist)
    cc = O.canonical_codes(ln)
    words, cw, sub = O.huffman_encode(codes, ln, cc, chunk, with_sub=True)
    nch = (n + chunk - 1) // chunk
    assert cw.size == nch
    nsb = O.sub_blocks(chunk)
    assert sub.size == nch * nsb
    for j in range(0, nch, max(1, nch // 7)):
        for b in range(nsb):
            blk = codes[j * chunk + b * 512: min(j * chunk + min((b + 1) * 512, chunk), n)]
            assert sub[j * nsb + b] == int(np.sum(ln[blk].astype(np.int64)))
    # per-chunk word counts from the lengths alone
    for j in range(nch):
        bits = int(np.sum(ln[codes[j * chunk:(j + 1) * chunk]].astype(np.int64)))
        assert cw[j] == (bits + 31) // 32
    assert words.size == int(cw.sum())
    back = O.huffman_decode(words, cw, ln, n, chunk, sub_bits=sub)
    assert np.array_equal(back, codes)
    if sub.size:
        bad = sub.copy()
        bad[0] ^= 1
        with pytest.raises(O.OracleError):
            O.huffman_decode(words, cw, ln, n, chunk, sub_bits=bad)
