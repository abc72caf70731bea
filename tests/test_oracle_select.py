"""Oracle: the per-level selection estimate, its features and the network's
reference, pinned independently of the oracle's own C code."""
import numpy as np

import oracle as O
from oracle import mlp as M
from paper_2111_02925_gb300 import synthetic as S


def _brute_costs(x, eb_rel, level):
    """Independent restatement on a small field: every point of the level,
    the pass axis by its odd coordinates, the predictor and quantizer written
    out with numpy float32 scalars, Shannon bits of the code histogram."""
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
