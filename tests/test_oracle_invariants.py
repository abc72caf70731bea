"""Invariant pins of the oracle's predict/quantize/recover path.

What the SZ3 paper fixes and these tests check:
* the error bound holds at every point (Sec. 1 and Sec. 3.2: error-bounded
  compression; the quantizer is the only lossy module) -- checked in exact
  rational / extended arithmetic, not with the oracle's own comparison;
* recover() reverses quantize() (Sec. 3.2): decompress(compress(x)) equals the
  reconstruction the compressor predicted from, bit for bit;
* interpolation uses constant coefficients (Sec. 6.2), so it is exact on data
  the interpolant reproduces: a constant field gives all-zero quantization
  indices; linear interpolation on an affine field and cubic interpolation on
  a quadratic one give indices within one bin of zero, except at the copy
  fallback, which cannot reproduce a slope.
"""
import itertools
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O
from paper_2111_02925_gb300 import synthetic as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")
R = 32768


def _point_info(dims, order):
    """Pass axis, stride, coordinate and neighbour availability of every code
    position, derived from coordinates (independent of the oracle)."""
    from test_oracle_traversal import expected_traversal

    exp, coords, level, pas, axis, s = expected_traversal(dims, lambda l: order)
    info = []
    for pos, idx in enumerate(exp):
        if pos == 0:
            info.append(None)
            continue
        a, st = axis[idx], s[idx]
        i, n = coords[idx, a], dims[a]
        info.append(dict(i=i, n=n, s=st, has_b=i + st < n, has_c=i >= 3 * st, has_d=i + 3 * st < n))
    return info


def test_golden_worked_example():
    g = json.load(open(os.path.join(GOLD, "interp_1d_worked.json")))
    p = O.make_params(g["dims"], g["eb"])
    x = np.array(g["x"], np.float32)
    codes, unpred, recon, ebT = O.quantize(p, x)
    assert (codes.astype(int) - R).tolist() == g["q"]
    assert recon.tolist() == g["recon"]
    assert unpred.size == 0


@pytest.mark.parametrize("dtype", [O.F32, O.F64])
@pytest.mark.parametrize("interp", [O.LINEAR, O.CUBIC])
def test_constant_field_gives_zero_indices(dtype, interp):
    t = np.float32 if dtype == O.F32 else np.float64
    for dims, c in [((17, 9, 12), 3.25), ((40, 33), -7.0), ((100,), 0.0), ((5, 6, 7, 3), 1e3)]:
        x = np.full(dims, c, t)
        p = O.make_params(dims, 1e-2, dtype=dtype, interp=interp)
        codes, unpred, recon, ebT = O.quantize(p, x)
        assert np.all(codes[1:] == R)
        assert unpred.size == (1 if codes[0] == 0 else 0)
        assert np.max(np.abs(recon.astype(np.float64) - c)) <= float(ebT)
        # the anchor has prediction 0; when it is unpredictable it is stored raw
        if codes[0] == 0:
            assert unpred[0] == x.ravel()[0]


@pytest.mark.parametrize("interp", [O.LINEAR, O.CUBIC])
@pytest.mark.parametrize("dims,order", [((33, 20, 17), (0, 1, 2)), ((64, 64), (1, 0)), ((129,), (0,)),
                                        ((12, 9, 30), (2, 0, 1))])
def test_affine_field_gives_near_zero_indices(interp, dims, order):
    rng = np.random.default_rng(11)
    coef = rng.uniform(-1, 1, len(dims))
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims], indexing="ij")
    x = (0.5 + sum(c * g for c, g in zip(coef, grids))).astype(np.float32)
    eb = 1e-2
    p = O.make_params(dims, eb, interp=interp, order=order)
    codes, unpred, recon, ebT = O.quantize(p, x)
    info = _point_info(dims, order)
    off = 0
    checked = 0
    for pos in range(1, len(codes)):
        f = info[pos]
        copy_fallback = (not f["has_b"]) and (not f["has_c"])
        if copy_fallback:
            continue
        checked += 1
        if abs(int(codes[pos]) - R) > 1:
            off += 1
    assert off == 0
    assert checked > 0.9 * (len(codes) - 1)
    nonzero = np.mean(codes[1:] != R)
    assert nonzero < 0.5  # most errors land in the zero bin


@pytest.mark.parametrize("dims", [(41, 23, 19), (70, 50)])
def test_cubic_on_quadratic_data(dims):
    rng = np.random.default_rng(5)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims], indexing="ij")
    x = sum(rng.uniform(-1, 1) * g + rng.uniform(-2e-3, 2e-3) * g * g for g in grids)
    x = x.astype(np.float64)
    order = tuple(range(len(dims)))
    p = O.make_params(dims, 1e-3, dtype=O.F64, interp=O.CUBIC, order=order)
    codes, unpred, recon, ebT = O.quantize(p, x)
    info = _point_info(dims, order)
    checked = 0
    for pos in range(1, len(codes)):
        f = info[pos]
        cubic_rule = (f["has_c"] and f["has_d"]) or (not f["has_c"] and f["has_d"]) or (f["has_c"] and f["has_b"])
        if not cubic_rule:
            continue
        checked += 1
        assert abs(int(codes[pos]) - R) <= 1
    assert checked > 0.8 * (len(codes) - 1)


def _max_err_exact(x, recon):
    if x.dtype == np.float32:
        return np.max(np.abs(x.ravel().astype(np.float64) - recon.astype(np.float64)))  # exact for nearby floats
    return max(abs(Fr(float(a)) - Fr(float(b))) for a, b in zip(x.ravel()[:20000], recon[:20000]))


CASES = [
    ("bumps32", lambda: S.gaussian_bumps(32, 1), O.F32, O.ABS, 1e-3 * 2.0),
    ("grf3d", lambda: S.grf((24, 40, 33), 2), O.F32, O.REL, 1e-3),
    ("grf3d_tight", lambda: S.grf((20, 21, 22), 9), O.F32, O.REL, 1e-6),
    ("latlon", lambda: S.latlon(90, 180, 3), O.F64, O.ABS, 1e-6 * 10),
    ("grf2d64", lambda: S.grf((65, 47), 4).astype(np.float64), O.F64, O.REL, 1e-4),
    ("grf4d", lambda: S.grf((6, 9, 5, 11), 6), O.F32, O.REL, 1e-3),
    ("grf1d", lambda: S.grf((1000,), 6), O.F32, O.REL, 1e-2),
]


@pytest.mark.parametrize("name,make,dtype,mode,eb", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("interp", [O.LINEAR, O.CUBIC])
def test_error_bound_and_round_trip(name, make, dtype, mode, eb, interp):
    x = make()
    t = np.float32 if dtype == O.F32 else np.float64
    x = x.astype(t)
    p = O.make_params(x.shape, eb, dtype=dtype, eb_mode=mode, interp=interp)
    codes, unpred, recon, ebT = O.quantize(p, x)
    eb_abs = eb * (float(x.max()) - float(x.min())) if mode == O.REL else eb
    assert float(ebT) <= eb_abs
    assert float(np.nextafter(t(ebT), t(np.inf))) > eb_abs or float(ebT) == eb_abs
    if dtype == O.F32:
        assert _max_err_exact(x, recon) <= float(ebT)
    else:
        assert _max_err_exact(x, recon) <= Fr(float(ebT))
    # unpredictables are stored raw, in traversal order
    trav = O.traversal(p)
    zero = codes == 0
    assert np.array_equal(unpred, x.ravel()[trav[zero]])
    assert np.array_equal(recon[trav[zero]], x.ravel()[trav[zero]])
    # recover() reverses quantize(): bitwise
    back = O.recover(p, ebT, codes, unpred)
    assert np.array_equal(back.view(np.uint8), recon.view(np.uint8))
    # and through the stream
    s = O.compress(p, x)
    y = O.decompress(s)
    assert np.array_equal(y.view(np.uint8), recon.view(np.uint8))


def test_small_radius_forces_unpredictables():
    x = S.grf((20, 20, 20), 3)
    for r in (2, 3, 8):
        p = O.make_params(x.shape, 1e-4, eb_mode=O.REL, radius=r, interp=O.CUBIC)
        codes, unpred, recon, ebT = O.quantize(p, x)
        assert codes.max() < 2 * r
        assert unpred.size > 0.5 * x.size
        y = O.decompress(O.compress(p, x))
        assert np.array_equal(y, recon)
        assert np.max(np.abs(y.astype(np.float64) - x.ravel())) <= float(ebT)


def test_brute_force_all_shapes_up_to_8():
    """Every shape in {1..8}^3, both interpolations, two orders: bound and round trip."""
    rng = np.random.default_rng(1)
    orders = list(itertools.permutations(range(3)))
    for dims in itertools.product(range(1, 9), repeat=3):
        x = rng.standard_normal(dims).astype(np.float32).cumsum(axis=2)
        for interp in (O.LINEAR, O.CUBIC):
            order = orders[rng.integers(6)]
            p = O.make_params(dims, 0.05, interp=interp, order=order)
            codes, unpred, recon, ebT = O.quantize(p, x)
            assert np.max(np.abs(recon.astype(np.float64) - x.ravel())) <= float(ebT)
            y = O.decompress(O.compress(p, x))
            assert np.array_equal(y, recon)


def test_error_bound_rounding_toward_zero():
    # REL: eb_abs = eb * (max - min) in double, then rounded toward 0 into T
    x = np.array([0.0, 0.1, 0.3], np.float32)
    p = O.make_params([3], 1e-3, eb_mode=O.REL)
    eb_abs, ebT = O.error_bound(p, x)
    assert eb_abs == 1e-3 * (float(np.float32(0.3)) - 0.0)
    assert float(ebT) <= eb_abs < float(np.nextafter(ebT, np.float32(1)))


def test_error_statuses():
    x = np.zeros((4, 4), np.float32)
    assert O.compress_status(O.make_params(x.shape, 1e-3, eb_mode=O.REL), x) == O.E_ZERO_RANGE_REL
    y = x.copy()
    y[1, 2] = np.nan
    assert O.compress_status(O.make_params(x.shape, 1e-3), y) == O.E_NONFINITE
    y[1, 2] = np.inf
    assert O.compress_status(O.make_params(x.shape, 1e-3, eb_mode=O.REL), y) == O.E_NONFINITE
    assert O.compress_status(O.make_params(x.shape, 0.0), x) == O.E_INVAL
    assert O.compress_status(O.make_params(x.shape, -1.0), x) == O.E_INVAL
    assert O.compress_status(O.make_params(x.shape, 1e-3, order=(0, 0)), x) == O.E_INVAL
    assert O.compress_status(O.make_params(x.shape, 1e-3, radius=1), x) == O.E_INVAL
    assert O.compress_status(O.make_params(x.shape, 1e-3, radius=32769), x) == O.E_INVAL
    assert O.compress_status(O.make_params(x.shape, 1e-3, chunk=100), x) == O.E_INVAL
    assert O.compress_status(O.make_params(x.shape, 1e-60), x) == O.E_INVAL  # eb_T underflows in FP32
