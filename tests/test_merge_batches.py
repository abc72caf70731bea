"""The batched form of the two-queue Huffman merge, checked on the host.

The codebook kernels do not run the greedy merge of Sec. 3.2 (Encoder) one
node at a time; they build the same tree in batches.  In the merged
consumption order S (leaves and internal nodes by weight, a leaf before an
internal node of equal weight, internal nodes in creation order) internal
node j has S[2j], S[2j+1] as children and sits at position
P(j) = j + #(leaves not heavier than it).  Once node j0 exists, the items of
S before P(j0) are those leaves and the internal nodes below j0, so nodes
j0+1 .. (P-2)/2 can all be built at once from the segment that merges the
leaves and internal nodes not yet consumed; the next node takes node j0 and
its neighbour in S.  This file restates that schedule in plain Python (one
loop where the GPU has one thread per node) with the length-limit halving
rounds, and compares the code lengths with the oracle's serial merge on
many alphabets, including chain-shaped trees that need one batch per node
and deep trees that need the halving rounds.
"""
from bisect import bisect_right

import numpy as np
import pytest

import oracle as O


def _batched_tree(w):
    """Parents of the two-queue merge over the sorted leaf weights w, built
    batch by batch; returns (parent, number of batches)."""
    K = len(w)
    W = [0] * (K - 1)
    parent = [-1] * (2 * K - 1)
    j0, a, m, w0 = 0, 2, 0, w[0] + w[1]
    W[0] = w0
    parent[0] = parent[1] = K
    batches = 0
    while j0 + 2 < K:  # node K - 2 is the root
        batches += 1
        P = j0 + bisect_right(w, w0, a, K)
        cL, j1 = P - j0, (P - 2) // 2
        for t in range(j1 - j0):  # nodes j0+1 .. j1, independent of each other
            d = 2 * t
            lo, hi = max(0, d - (j0 - m)), min(d, cL - a)  # leaves among the first d items of the segment
            while lo < hi:
                i = (lo + hi) // 2
                if w[a + i] <= W[m + d - i - 1]:
                    lo = i + 1
                else:
                    hi = i
            x, y, ids, tot = a + lo, m + d - lo, [], 0
            for _ in range(2):
                leaf = x < cL and (y >= j0 or w[x] <= W[y])
                ids.append(x if leaf else K + y)
                tot += w[x] if leaf else W[y]
                x, y = x + leaf, y + (not leaf)
            W[j0 + 1 + t] = tot
            parent[ids[0]] = parent[ids[1]] = K + j0 + 1 + t
        jn = j1 + 1
        if P & 1:  # the segment's last item, then node j0
            last_leaf = j0 == m or (cL > a and w[cL - 1] > W[j0 - 1])
            i0 = cL - 1 if last_leaf else K + j0 - 1
            wn = (w[cL - 1] if last_leaf else W[j0 - 1]) + w0
            ids = (i0, K + j0)
            a, m = cL, j0 + 1
        else:  # node j0, then the next front
            leaf = cL < K and (j1 == j0 or w[cL] <= W[j0 + 1])
            ids = (K + j0, cL if leaf else K + j0 + 1)
            wn = w0 + (w[cL] if leaf else W[j0 + 1])
            a, m = cL + leaf, j0 + 1 + (not leaf)
        W[jn] = wn
        parent[ids[0]] = parent[ids[1]] = K + jn
        j0, w0 = jn, wn
    return parent, batches


def _batched_lengths(freq, lmax=O.LMAX):
    """Code lengths by symbol: leaves sorted by (weight, symbol), the batched
    merge, depths; weights halved (at least 1) while a code is too long."""
    f = np.asarray(freq, np.uint64)
    used = np.flatnonzero(f)
    out = np.zeros(f.size, np.uint8)
    if used.size == 1:
        out[used[0]] = 1
        return out, 0
    wt = f[used].astype(np.int64)
    total = 0
    while True:
        order = np.lexsort((used, wt))  # by weight, then symbol
        parent, nb = _batched_tree([int(v) for v in wt[order]])
        total += nb
        K, root = used.size, 2 * used.size - 2
        depth = np.zeros(K, np.int64)
        for i in range(K):
            v, dd = i, 0
            while v != root:
                v, dd = parent[v], dd + 1
            depth[i] = dd
        if depth.max() <= lmax:
            out[used[order]] = depth
            return out, total
        wt = np.maximum(wt >> 1, 1)


def _fib(n):
    a, b, r = 1, 1, []
    for _ in range(n):
        r.append(a)
        a, b = b, a + b
    return r


@pytest.mark.parametrize("seed", range(40))
def test_batched_merge_equals_serial_merge(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(2, 700))
    kind = seed % 5
    if kind == 0:
        f = rng.integers(1, 11, K)
    elif kind == 1:
        f = np.ones(K, np.int64)
    elif kind == 2:
        f = np.exp(rng.uniform(0, 18, K)).astype(np.int64) + 1
    elif kind == 3:  # a quantization-code histogram: Laplacian around the middle
        c = np.arange(K) - K // 2
        f = (1e7 * np.exp(-np.abs(c) / (1.0 + K / 30.0))).astype(np.int64) + rng.integers(0, 2, K)
    else:
        f = rng.integers(1, 100000, K)
    hist = np.zeros(K + int(rng.integers(0, 50)), np.uint64)
    pos = np.sort(rng.choice(hist.size, K, replace=False))
    hist[pos] = np.maximum(f, 0)
    hist[pos[hist[pos] == 0]] = 1
    got, _ = _batched_lengths(hist)
    assert np.array_equal(got, O.huffman_lengths(hist))


def test_chain_tree_one_batch_per_node():
    f = np.array(_fib(20), np.uint64)
    got, nb = _batched_lengths(f)
    assert np.array_equal(got, O.huffman_lengths(f))
    assert got.max() == 19 and nb == 18


def test_deep_tree_takes_the_halving_rounds():
    f = np.array(_fib(40), np.uint64)
    got, _ = _batched_lengths(f)
    want = O.huffman_lengths(f)
    assert want.max() <= O.LMAX and np.array_equal(got, want)


@pytest.mark.parametrize("f", [[5], [3, 9], [1, 1, 1], [2, 1, 1], [7, 7, 1, 1, 1, 1]])
def test_tiny_alphabets(f):
    h = np.array(f, np.uint64)
    assert np.array_equal(_batched_lengths(h)[0], O.huffman_lengths(h))
