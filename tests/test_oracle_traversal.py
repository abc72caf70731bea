"""Pins of the oracle's traversal (the multilevel interpolation schedule).

SZ3 paper Alg. 1 (predict and quantize every point once, in one pass) and
Sec. 6.2 (SZ3-Interp: multilevel interpolation).  The order is checked
against an independent characterisation, not the oracle's odometer walk:

* a point p != 0 first appears at the level l whose stride s = 2^(l-1) is the
  largest power of two dividing every coordinate;
* its pass is the latest axis in that level's order on which p/s is odd;
* the stream is sorted by (level descending, pass ascending, row-major index).

Then, by brute force over every shape in {1..8}^3, the neighbours at +-s and
+-3s on the pass axis (the predictor's inputs) all come earlier, and every
point appears exactly once.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def keys(dims, order_of_level):
    """(level, pass, row-major) key of every point, computed from coordinates."""
    dims = list(dims)
    nd = len(dims)
    L = 0
    while (1 << L) < max(dims):
        L += 1
    coords = np.stack(np.meshgrid(*[np.arange(n) for n in dims], indexing="ij"), -1).reshape(-1, nd)
    N = coords.shape[0]
    tz = np.full((N, nd), 99, np.int64)
    for a in range(nd):
        c = coords[:, a]
        nz = c != 0
        tz[nz, a] = np.array([(int(v) & -int(v)).bit_length() - 1 for v in c[nz]], np.int64)
    v = tz.min(1)
    level = np.where(v == 99, L + 1, v + 1)  # anchor sorts first
    s = np.where(v == 99, 1, 1 << np.minimum(v, 62))
    pas = np.full(N, -1, np.int64)
    axis = np.full(N, -1, np.int64)
    for idx in range(N):
        if level[idx] == L + 1:
            continue
        o = order_of_level(int(level[idx]))
        for k in range(nd):
            a = o[k]
            if (coords[idx, a] // s[idx]) % 2 == 1:
                pas[idx] = k
                axis[idx] = a
    return coords, level, pas, axis, s, L


def expected_traversal(dims, order_of_level):
    coords, level, pas, axis, s, L = keys(dims, order_of_level)
    N = coords.shape[0]
    rowmajor = np.arange(N)
    order = np.lexsort((rowmajor, pas, -level))
    return order, coords, level, pas, axis, s


def test_golden_3x3():
    g = json.load(open(os.path.join(GOLD, "traversal_3x3.json")))
    p = O.make_params(g["dims"], 1.0, order=g["order"])
    assert O.traversal(p).tolist() == g["traversal"]


def test_golden_1d():
    g = json.load(open(os.path.join(GOLD, "interp_1d_worked.json")))
    p = O.make_params(g["dims"], g["eb"])
    assert O.traversal(p).tolist() == g["traversal"]


def _check_shape(dims, order):
    p = O.make_params(dims, 1.0, order=order)
    got = O.traversal(p).astype(np.int64)
    exp, coords, level, pas, axis, s = expected_traversal(dims, lambda l: order)
    N = len(exp)
    assert got[0] == 0
    assert np.array_equal(np.sort(got), np.arange(N))  # a permutation: every point once
    assert np.array_equal(got, exp)
    # causality: predictor inputs precede the point
    pos = np.empty(N, np.int64)
    pos[got] = np.arange(N)
    strides = np.cumprod([1] + list(dims[::-1]))[:-1][::-1]
    for idx in range(1, N):
        a, st = axis[idx], s[idx]
        i = coords[idx, a]
        for off in (-3 * st, -st, st, 3 * st):
            j = i + off
            if 0 <= j < dims[a]:
                nb = idx + off * strides[a]
                assert pos[nb] < pos[idx]


def test_partition_and_causality_all_shapes_up_to_8():
    orders3 = list(itertools.permutations(range(3)))
    rng = np.random.default_rng(0)
    for dims in itertools.product(range(1, 9), repeat=3):
        # every shape with the default order, and one other seeded order
        _check_shape(dims, (0, 1, 2))
        _check_shape(dims, orders3[rng.integers(len(orders3))])


@pytest.mark.parametrize("dims", [(1,), (2,), (7,), (8,), (9,), (33,), (5, 1), (1, 6), (6, 7), (16, 3),
                                  (3, 4, 5, 2), (2, 3, 2, 5)])
def test_partition_other_ranks(dims):
    for order in itertools.permutations(range(len(dims))):
        _check_shape(dims, order)


def test_per_level_orders():
    dims = (6, 5, 7)
    rng = np.random.default_rng(3)
    perms = list(itertools.permutations(range(3)))
    lo = {l: perms[rng.integers(6)] for l in range(1, 4)}
    p = O.make_params(dims, 1.0, level_order=lo)
    got = O.traversal(p).astype(np.int64)
    exp, *_ = expected_traversal(dims, lambda l: lo[l])
    assert np.array_equal(got, exp)


def test_level_count():
    for n, L in [(1, 0), (2, 1), (3, 2), (4, 2), (5, 3), (512, 9), (513, 10), (1800, 11), (3600, 12)]:
        assert O.shape(O.make_params([n], 1.0))[1] == L
    assert O.shape(O.make_params([3, 1800, 7], 1.0)) == (3 * 1800 * 7, 11)
