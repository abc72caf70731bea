"""Pins of the oracle's linear-scaling quantizer against its closed form.

SZ3 paper Sec. 3.2 (Quantizer): equal consecutive bins of width 2*eb, the
prediction error is replaced by the index of the bin that contains it, values
whose error falls outside the countable range are unpredictable and stored
separately; recover() reverses quantize().

The expected bin is computed here with exact rational arithmetic
(fractions.Fraction), not with the oracle's floating-point steps.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O


def exact_bin(d: Fr, eb: Fr) -> int:
    """h with |d| in [(2h-1) eb, (2h+1) eb), i.e. |d|/(2eb) rounded half up."""
    a = abs(d) / (2 * eb)
    h = int(a + Fr(1, 2))  # floor(a + 1/2)
    return h


@pytest.mark.parametrize("dtype", [O.F32, O.F64])
@pytest.mark.parametrize("eb", [0.5, 1e-3, 3.7e-5])
def test_bin_index_matches_closed_form(dtype, eb):
    t = np.float32 if dtype == O.F32 else np.float64
    _, ebT = O.error_bound(O.make_params([4], eb, dtype=dtype), np.arange(4, dtype=t))
    ebT = t(ebT)
    r = 32768
    rng = np.random.default_rng(7)
    # dense sweep around bin edges (2h+1) eb and random interior points
    hs = np.arange(0, 40)
    edges = (2 * hs + 1) * float(ebT)
    ds = []
    for e in edges:
        for k in range(-3, 4):
            v = t(e)
            for _ in range(abs(k)):
                v = np.nextafter(v, t(np.inf) if k > 0 else t(0))
            ds.append(v)
    ds.extend(t(v) for v in rng.uniform(-100, 100, 400) * float(ebT))
    n_near = 0
    for d in ds:
        for sgn in (1, -1):
            x = t(sgn * d)
            code, recon = O.quantize1(x, t(0), ebT, r, dtype)
            h = exact_bin(Fr(float(x)), Fr(float(ebT)))
            q = code - r
            # the oracle evaluates |d| * fl(1/eb) in T: away from an edge the
            # bin must be exact; within a few ulps of an edge the neighbour bin
            # is also a correct reading of the rounding
            rel = abs(Fr(float(abs(x))) / Fr(float(ebT)) - (2 * h + 1))
            near = rel < Fr(1, 10 ** 4) or abs(Fr(float(abs(x))) / Fr(float(ebT)) - (2 * h - 1)) < Fr(1, 10 ** 4)
            if near:
                n_near += 1
                if code == 0:  # rounding pushed it past the bound check
                    assert recon == x
                    continue
                assert abs(q) in (h, h - 1, h + 1)
            else:
                assert code != 0
                assert abs(q) == h, (float(x), float(ebT), q, h)
            if x != 0:
                assert (q > 0) == (x > 0) or q == 0
            # recover(): pred + 2 q eb, within eb of x (exact check)
            assert Fr(float(recon)) == Fr(float(t(t(2 * q) * ebT)))
            assert abs(Fr(float(recon)) - Fr(float(x))) <= Fr(float(ebT))
    assert n_near > 0


@pytest.mark.parametrize("dtype", [O.F32, O.F64])
def test_out_of_range_is_unpredictable(dtype):
    t = np.float32 if dtype == O.F32 else np.float64
    ebT = t(0.25)
    for r in (2, 3, 100, 32768):
        lim = (2 * r - 1) * 0.25  # |d| >= (2r-1) eb  <=>  h would reach r
        for d in (lim, lim * 1.5, lim * 1e6, -lim, -lim * 3):
            code, recon = O.quantize1(t(d), t(0), ebT, r, dtype)
            assert code == 0 and recon == t(d)
        # just inside the range: largest bin r-1
        d = t(lim) - t(0.25) * t(0.5)
        code, recon = O.quantize1(d, t(0), ebT, r, dtype)
        assert code == r + (r - 1) or code == r + (r - 2)


def test_nonzero_prediction_and_codes_cover_alphabet():
    # with pred != 0 the error is x - pred; codes land in [1, 2r)
    r = 4
    ebT = np.float32(0.5)
    seen = set()
    for x in np.arange(-10, 10.25, 0.25, dtype=np.float32):
        code, recon = O.quantize1(x, np.float32(1.0), ebT, r, O.F32)
        assert 0 <= code < 2 * r
        seen.add(code)
        if code:
            assert abs(float(recon) - float(x)) <= 0.5
            assert code - r == exact_bin(Fr(float(x)) - 1, Fr(1, 2)) * (1 if x > 1 else -1)
        else:
            assert recon == x
            assert exact_bin(Fr(float(x)) - 1, Fr(1, 2)) >= r
    assert seen == set(range(2 * r))
