"""Oracle: the per-level selection estimate, its features and the network's
reference, pinned independently of the oracle's own C code."""
import json
import math
import os

import numpy as np

import oracle as O
from oracle import mlp as M
from paper_2111_02925_gb300 import synthetic as S


def _brute_costs(x, eb_rel, level):
    """A second transcription of the cost estimate (numpy float32 scalars,
    pure-Python loops).  It guards the C code against transcription slips but
    pins nothing of the reading itself: the pins of the estimate are the
    behavioural tests below (constant field, one-axis field, blocks covering
    the grid) and the closed-form feature and block tests."""
    x = np.asarray(x, np.float32)
    nd = x.ndim
    n = x.shape
    eb = float(eb_rel) * (float(x.max()) - float(x.min()))
    ebT = np.float32(eb)
    if float(ebT) > eb:
        ebT = np.nextafter(ebT, np.float32(0))
    ebr = np.float32(1) / ebT
    s = 1 << (level - 1)
    m = [(e + s - 1) // s for e in n]
    orders = O._SEL_ORDERS[nd]
    out = []
    for c in range(8):
        it, order = c % 2, orders[c // 2]
        hist = {}
        for g in np.ndindex(*m):
            if not any(v & 1 for v in g):
                continue
            a = [ax for ax in order if g[ax] & 1][-1]
            p = [v * s for v in g]

            def at(off):
                q = list(p)
                q[a] += off
                return x[tuple(q)]
            i, na = p[a], n[a]
            hb, hc, hd = i + s < na, i >= 3 * s, i + 3 * s < na
            A = at(-s)
            if it == 1 and hc and hd:
                pred = ((np.float32(9) * (A + at(s))) - (at(-3 * s) + at(3 * s))) * np.float32(0.0625)
            elif it == 1 and (not hc) and hd:
                pred = ((np.float32(3) * A + np.float32(6) * at(s)) - at(3 * s)) * np.float32(0.125)
            elif it == 1 and hc and hb:
                pred = ((np.float32(6) * A + np.float32(3) * at(s)) - at(-3 * s)) * np.float32(0.125)
            elif hb:
                pred = (A + at(s)) * np.float32(0.5)
            elif hc:
                pred = np.float32(1.5) * A - np.float32(0.5) * at(-3 * s)
            else:
                pred = A
            code = int(O.quantize1(np.float32(x[tuple(p)]), np.float32(pred), ebT)[0])
            hist[code] = hist.get(code, 0) + 1
        cnt = np.array(list(hist.values()), np.float64)
        N = cnt.sum()
        bits = N * np.log2(N) - (cnt * np.log2(cnt)).sum() + 32.0 * hist.get(0, 0) if N else 0.0
        out.append(bits)
    return np.array(out)


def test_costs_match_brute_force():
    x = S.grf((9, 11, 7), 3)
    p = O.make_params(x.shape, 1e-3, eb_mode=O.REL)
    for level in (1, 2, 3):
        assert np.allclose(O.select_costs(p, x, level), _brute_costs(x, 1e-3, level), rtol=1e-12, atol=1e-9)
    x2 = S.grf((13, 10), 4)
    p2 = O.make_params(x2.shape, 1e-2, eb_mode=O.REL)
    for level in (1, 2):
        assert np.allclose(O.select_costs(p2, x2, level), _brute_costs(x2, 1e-2, level), rtol=1e-12, atol=1e-9)


def test_blocks_covering_the_grid_equal_exhaustive():
    # grids of at most 16 points per axis: every sample block is the whole grid
    x = S.grf((16, 12, 10), 5)
    p = O.make_params(x.shape, 1e-3, eb_mode=O.REL)
    for level in (1, 2, 3, 4):
        assert np.array_equal(O.select_costs(p, x, level, 5, 9), O.select_costs(p, x, level))


def test_a_field_varying_along_one_axis_prefers_refining_it_first():
    # x = f(k): predictions along axes 0 and 1 are exact, so orders that leave
    # the fewest points to axis 2 (it refined first: (2,0,1), (2,1,0)) win
    k = np.arange(40, dtype=np.float64)
    f = np.sin(k * 0.7) + 0.3 * np.cos(k * 2.1)
    x = np.broadcast_to(f, (24, 20, 40)).astype(np.float32).copy()
    p = O.make_params(x.shape, 1e-3, eb_mode=O.REL)
    for level in (1, 2):
        c = O.select_costs(p, x, level)
        assert int(np.argmin(c)) in (4, 5, 6, 7)
        assert min(c[4:]) < min(c[:4])


def test_constant_and_affine_fields():
    x = np.full((20, 18, 16), 3.25, np.float32)
    p = O.make_params(x.shape, 1e-3)  # ABS
    for level in (1, 2):
        assert np.all(O.select_costs(p, x, level) == 0.0)  # every code is the radius
        f = O.select_features(p, x, level)
        assert np.all(f[:9] == 0.0) and f[12] == 1.0
    # a ramp along axis 0: exact linear prediction, lag-2 differences twice the lag-1
    i = np.arange(32, dtype=np.float64)[:, None, None]
    x = np.broadcast_to(0.01 * i, (32, 8, 8)).astype(np.float32).copy()
    p = O.make_params(x.shape, 1e-3)
    f = O.select_features(p, x, 1)
    assert f[0] < 1e-3 and abs(f[2] - 2.0) < 1e-6  # lin error ~0, log2((2d)^2 / d^2) = 2
    assert f[5] == 0.0 and f[8] == 0.0  # flat along axes 1 and 2
    assert f[9] == 1.0 / 5 and f[10] == 0.0


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    feat = rng.normal(size=(24, 16))
    mask = np.ones((24, 8), bool)
    mask[:6, 4:] = False  # 2-D rows
    label = np.where(np.arange(24) < 6, rng.integers(0, 4, 24), rng.integers(0, 8, 24))
    w = M.init(feat, 2)
    loss, g = M.loss_and_grad(w, feat, mask, label)
    for k in list(range(M.OFF_W1, M.OFF_W1 + 20)) + list(range(M.OFF_W2, M.OFF_W2 + 20)) + [M.OFF_B1 + 3,
                                                                                           M.N_WEIGHTS - 1]:
        e = np.zeros_like(w)
        e[k] = 1e-6
        num = (M.loss_and_grad(w + e, feat, mask, label)[0] - M.loss_and_grad(w - e, feat, mask, label)[0]) / 2e-6
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(num))
    assert np.all(g[:M.OFF_W1] == 0.0)


_GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_matches_published_outputs():
    """The block placement hashes with SplitMix64; its first outputs from
    state 1234567 are the published reference values."""
    g = json.load(open(os.path.join(_GOLDEN, "splitmix64_1234567.json")))
    gamma = int(g["gamma"], 16)
    for i, want in enumerate(g["outputs"]):
        assert O.splitmix64((g["seed"] + i * gamma) % (1 << 64)) == int(want)


def test_sample_blocks_hand_worked():
    g = json.load(open(os.path.join(_GOLDEN, "select_blocks.json")))
    for c in g["cases"]:
        p = O.make_params(tuple(c["dims"]), 1e-3)
        lo, hi = O.select_blocks(p, c["level"], c["nblocks"], int(c["seed"]))
        assert lo.shape == (c["nblocks"], 3)
        b, d = c["block"], c["axis"]
        assert c["modulus"] == c["m"] - c["span"] + 1
        assert lo[b, d] == c["start"] and hi[b, d] - lo[b, d] == c["span"]
        # every block lies in the grid of the level and spans min(16, m) points
        s = 1 << (c["level"] - 1)
        m = [(n + s - 1) // s for n in c["dims"]]
        for e in range(3):
            assert np.all(lo[:, e] >= 0) and np.all(hi[:, e] <= m[e])
            assert np.all(hi[:, e] - lo[:, e] == min(16, m[e]))


def _quartic(shape, axis):
    """x = i_axis^4 (exact small integers in float32)."""
    i = np.arange(shape[axis], dtype=np.float64) ** 4
    sh = [1, 1, 1]
    sh[axis] = shape[axis]
    return np.broadcast_to(i.reshape(sh), shape).astype(np.float32).copy()


def test_features_closed_forms_on_a_quartic():
    """x = i^4 along one axis of 20 points, constant along the others, ABS
    eb = 1.  At stride s = 1, for odd i with a +1 neighbour (i = 1..17):
    linear error |((i-1)^4 + (i+1)^4)/2 - i^4| = 6 i^2 + 1 (mean 5823/9 =
    647); cubic error |(9((i-1)^4 + (i+1)^4) - ((i-3)^4 + (i+3)^4))/16 - i^4|
    = 9 where i >= 3 and i + 3 < 20, the linear error elsewhere (mean
    (63 + 7 + 1735)/9).  The level's points whose pass axis (order (0,1,2))
    is the quartic one: linear error above 64 at i = 5..17 and at i = 19
    (extrapolation 1.5 x(18) - 0.5 x(16): error 5625), cubic above 64 only
    at i = 17 ((6 x(16) + 3 x(18) - x(14))/8: error 195) and i = 19."""
    others = (6, 8)
    for a in range(3):
        shape = list(others)
        shape.insert(a, 20)
        shape = tuple(shape)
        x = _quartic(shape, a)
        p = O.make_params(shape, 1.0)  # ABS eb = 1 (exact in float32)
        f = O.select_features(p, x, 1)
        for d in range(3):
            if d == a:
                assert f[3 * d] == math.log2(1.0 + 647.0)
                assert abs(f[3 * d + 1] - math.log2(1.0 + 1805.0 / 9.0)) < 1e-12
            else:
                assert f[3 * d] == 0.0 and f[3 * d + 1] == 0.0
        assert f[9] == 1.0 / 5 and f[10] == 0.0          # l / L with L = ceil(log2 20) = 5; l - 1
        assert abs(f[11] - math.log10(1.0 / 130321.0)) < 1e-12  # range 19^4
        # +1 differences all within eb: only where i = 0 on the quartic axis
        assert abs(f[12] - 1.0 / 19.0) < 1e-15
        # points whose pass axis is a: odd on a, any on earlier axes, even on later ones
        m = list(shape)
        n_pass_a = 10 * int(np.prod([m[b] for b in range(a)])) * int(np.prod([(m[b] + 1) // 2 for b in range(a + 1, 3)]))
        n_lvl = int(np.prod(m)) - int(np.prod([(e + 1) // 2 for e in m]))
        assert abs(f[13] - (8 / 10) * n_pass_a / n_lvl) < 1e-15
        assert abs(f[14] - (2 / 10) * n_pass_a / n_lvl) < 1e-15
        assert abs(f[15] - math.log2(shape[2] / shape[0])) < 1e-15


def test_features_closed_forms_at_stride_two():
    """Level 2 (stride 2) of the quartic along axis 0: the grid values are
    16 g^4 (g = 0..9), so the errors are 16 times those of g^4 on a 10-point
    axis: odd g with g + 1 < 10 (1, 3, 5, 7): linear 16 (6 g^2 + 1), mean
    16 * 508 / 4 = 2032; cubic 16 * 9 at g = 3, 5, the linear error at
    g = 1, 7: mean (112 + 144 + 144 + 4720) / 4 = 1280."""
    shape = (20, 6, 8)
    x = _quartic(shape, 0)
    p = O.make_params(shape, 1.0)
    f = O.select_features(p, x, 2)
    assert f[0] == math.log2(1.0 + 2032.0)
    assert f[1] == math.log2(1.0 + 1280.0)
    assert f[3] == f[4] == f[6] == f[7] == 0.0
    assert f[9] == 2.0 / 5 and f[10] == 1.0
    assert abs(f[15] - math.log2(4 / 10)) < 1e-15


def test_lag_ratio_on_ramps_along_each_axis():
    """A ramp along axis d: lag-2 differences are twice the lag-1 ones, so
    log2 of the ratio of their mean squares is 2; the other axes are flat
    (ratio of zeros, 0 by the regularised form)."""
    for a in range(3):
        shape = [10, 12, 14]
        i = np.arange(shape[a], dtype=np.float64) * 0.5
        sh = [1, 1, 1]
        sh[a] = shape[a]
        x = np.broadcast_to(i.reshape(sh), shape).astype(np.float32).copy()
        p = O.make_params(tuple(shape), 1e-3)
        f = O.select_features(p, x, 1)
        for d in range(3):
            if d == a:
                assert abs(f[3 * d + 2] - 2.0) < 1e-6
                assert f[3 * d] < 1e-9  # linear prediction exact on a ramp
            else:
                assert f[3 * d + 2] == 0.0 and f[3 * d] == 0.0
