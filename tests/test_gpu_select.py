"""GPU: per-level selection against the oracle (estimated bits and features on
the same seeded sample blocks), the network's kernels against the float64
reference, and the trained selector against the sampling selector and a fixed
choice."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_2111_02925_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2111_02925_gb300 import build as B  # noqa: E402
from paper_2111_02925_gb300 import sz3g as G  # noqa: E402

B.build()
G.load()
DEV = "cuda"
SH = None


def _sh():
    return G._stream_handle()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(DEV)


FIELDS = [
    (lambda: S.grf_fronts((40, 36, 44), 11, 8), 1e-3, O.F32),
    (lambda: S.grf((33, 50, 21), 12), 1e-4, O.F32),
    (lambda: S.latlon(90, 180, seed=13), 1e-5, O.F64),
    (lambda: S.grf((300,), 14), 1e-3, O.F32),
]


@pytest.mark.parametrize("case", range(len(FIELDS)))
@pytest.mark.parametrize("nblocks", [0, 6])
def test_costs_and_features_match_oracle(case, nblocks):
    make, eb, dt = FIELDS[case]
    x = make().astype(np.float32 if dt == O.F32 else np.float64)
    op = O.make_params(x.shape, eb, dtype=dt, eb_mode=O.REL)
    gp = G.make_params(x.shape, eb, dtype=dt, eb_mode=G.REL)
    xd = _dev(x)
    gc = G.sz3g_select_costs(gp, xd.data_ptr(), nblocks, 77, _sh())
    gf = G.sz3g_select_features(gp, xd.data_ptr(), nblocks, 77, _sh())
    _, L = O.shape(op)
    assert gc.shape == (L, 8) and gf.shape == (L, 16)
    for l in range(1, L + 1):
        oc = O.select_costs(op, x, l, nblocks, 77)
        of = O.select_features(op, x, l, nblocks, 77)
        assert np.allclose(gc[l - 1], oc, rtol=1e-10, atol=1e-8), (l, gc[l - 1], oc)
        assert np.allclose(gf[l - 1], of, rtol=1e-10, atol=1e-10), (l, gf[l - 1], of)
    ch = G.sz3g_select_sampled(gp, xd.data_ptr(), nblocks, 77, _sh())
    valid = 8 if x.ndim == 3 else (4 if x.ndim == 2 else 2)
    for l in range(1, L + 1):
        oc = O.select_costs(op, x, l, nblocks, 77)[:valid]
        best = int(np.argmin(oc))
        if ch[l] != best:  # only a near-tie may differ in rounding
            assert abs(oc[ch[l]] - oc[best]) <= 1e-9 * max(1.0, abs(oc[best]))


def test_network_kernels_match_reference():
    rng = np.random.default_rng(3)
    n = 300
    feat = rng.normal(size=(n, 16)) * 2.0 + 1.0
    mask = np.ones((n, 8), np.uint8)
    mask[:50, 4:] = 0
    mask[50:70, 2:] = 0
    label = np.where(np.arange(n) < 50, rng.integers(0, 4, n),
                     np.where(np.arange(n) < 70, rng.integers(0, 2, n), rng.integers(0, 8, n)))
    w = M.init(feat, 4)
    wd = _dev(w.astype(np.float32))
    fd, md = _dev(feat.astype(np.float32)), _dev(mask)
    ld = _dev(label.astype(np.int32))
    logits = torch.empty(n * 8, dtype=torch.float32, device=DEV)
    G.sz3g_mlp_forward(wd.data_ptr(), fd.data_ptr(), md.data_ptr(), n, logits.data_ptr(), _sh())
    ref, _, _ = M.forward(w.astype(np.float32).astype(np.float64), feat.astype(np.float32), mask)
    got = logits.cpu().numpy().reshape(n, 8)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got))
    assert np.allclose(got[fin], ref[fin], rtol=1e-4, atol=1e-4)
    grad = torch.empty(G.MLP_WEIGHTS, dtype=torch.float32, device=DEV)
    loss = G.sz3g_mlp_gradient(wd.data_ptr(), fd.data_ptr(), md.data_ptr(), ld.data_ptr(), n, grad.data_ptr(), _sh())
    rl, rg = M.loss_and_grad(w.astype(np.float32).astype(np.float64), feat.astype(np.float32), mask, label)
    assert abs(loss - rl) <= 1e-4 * max(1.0, rl)
    g = grad.cpu().numpy()
    assert np.allclose(g, rg, rtol=2e-3, atol=2e-5)
    # a few steps of descent lower the loss
    l1 = G.sz3g_mlp_train(wd.data_ptr(), fd.data_ptr(), md.data_ptr(), ld.data_ptr(), n, 0.5, 200, _sh())
    l2 = G.sz3g_mlp_gradient(wd.data_ptr(), fd.data_ptr(), md.data_ptr(), ld.data_ptr(), n, grad.data_ptr(), _sh())
    assert l2 < rl and l2 <= l1 + 1e-6


def _train_set(count, size, seed):
    """Features (GPU, 8 sample blocks) and oracle labels (exhaustive trial)."""
    rng = np.random.default_rng(seed)
    feats, labels = [], []
    for i in range(count):
        shape = tuple(int(v) for v in rng.integers(size // 2, size + 1, 3))
        x = S.grf_fronts(shape, seed * 1000 + i, int(rng.integers(0, 17)))
        eb = float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-2))))
        op = O.make_params(shape, eb, eb_mode=O.REL)
        gp = G.make_params(shape, eb, eb_mode=G.REL)
        _, L = O.shape(op)
        f = G.sz3g_select_features(gp, _dev(x).data_ptr(), 8, i, _sh())
        for l in range(1, L + 1):
            feats.append(f[l - 1])
            labels.append(int(np.argmin(O.select_costs(op, x, l))))
    return np.array(feats), np.array(labels, np.int32)


def _size(x, p):
    xd = _dev(x)
    cap = G.sz3g_compress_bound(p)
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    rc, nb = G.sz3g_compress(p, xd.data_ptr(), out.data_ptr(), cap, stream=_sh())
    assert rc == 0
    return nb


def test_trained_selector_gains_over_fixed_choice_and_tracks_sampling():
    feat, label = _train_set(120, 48, 21)
    w = M.init(feat, 5)
    wd = _dev(w.astype(np.float32))
    n = len(label)
    fd, ld = _dev(feat.astype(np.float32)), _dev(label)
    md = _dev(np.ones((n, 8), np.uint8))
    loss = G.sz3g_mlp_train(wd.data_ptr(), fd.data_ptr(), md.data_ptr(), ld.data_ptr(), n, 0.3, 3000, _sh())
    logits = torch.empty(n * 8, dtype=torch.float32, device=DEV)
    G.sz3g_mlp_forward(wd.data_ptr(), fd.data_ptr(), md.data_ptr(), n, logits.data_ptr(), _sh())
    acc = float(np.mean(logits.cpu().numpy().reshape(n, 8).argmax(1) == label))
    assert np.isfinite(loss) and acc > 0.5
    fixed = sampled = learned = 0
    for i in range(6):
        x = S.grf_fronts((64, 60, 56), 9000 + i, 16)
        p = G.make_params(x.shape, 1e-4, eb_mode=G.REL, interp=G.LINEAR)
        xd = _dev(x)
        cs = G.sz3g_select_sampled(p, xd.data_ptr(), 32, i, _sh())
        cl = G.sz3g_select_learned(p, xd.data_ptr(), wd.data_ptr(), 8, i, _sh())
        fixed += _size(x, p)
        sampled += _size(x, G.params_for_choices(p, cs))
        learned += _size(x, G.params_for_choices(p, cl))
    assert learned <= 1.02 * sampled, (learned, sampled)
    assert learned < fixed, (learned, fixed)
