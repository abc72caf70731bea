"""The selector's network in float64 numpy (TEST INFRASTRUCTURE): the reference
that the CUDA forward / backward kernels are checked against.

16 features, standardised by (f - mu) / sd, -> 64 hidden units (ReLU) -> 8
logits; masked softmax cross-entropy, averaged over the batch.  Weights are
packed as in the library: mu[16], sd[16], W1[64][16], b1[64], W2[8][64], b2[8].
"""
import numpy as np

N_IN, N_HID, N_OUT = 16, 64, 8
OFF_MU, OFF_SD, OFF_W1 = 0, 16, 32
OFF_B1 = OFF_W1 + N_HID * N_IN
OFF_W2 = OFF_B1 + N_HID
OFF_B2 = OFF_W2 + N_OUT * N_HID
N_WEIGHTS = OFF_B2 + N_OUT


def unpack(w):
    w = np.asarray(w, np.float64)
    return (w[OFF_MU:OFF_SD], w[OFF_SD:OFF_W1], w[OFF_W1:OFF_B1].reshape(N_HID, N_IN), w[OFF_B1:OFF_W2],
            w[OFF_W2:OFF_B2].reshape(N_OUT, N_HID), w[OFF_B2:N_WEIGHTS])


def forward(w, feat, mask):
    """Logits (masked entries -inf) and the hidden layer."""
    mu, sd, W1, b1, W2, b2 = unpack(w)
    z = (np.asarray(feat, np.float64) - mu) / sd
    a = z @ W1.T + b1
    h = np.maximum(a, 0.0)
    lg = h @ W2.T + b2
    lg = np.where(np.asarray(mask, bool), lg, -np.inf)
    return lg, h, z


def loss_and_grad(w, feat, mask, label):
    """Mean masked softmax cross-entropy and its gradient (zero for mu, sd)."""
    mu, sd, W1, b1, W2, b2 = unpack(w)
    lg, h, z = forward(w, feat, mask)
    B = lg.shape[0]
    mx = lg.max(axis=1, keepdims=True)
    e = np.where(np.isfinite(lg), np.exp(lg - mx), 0.0)
    p = e / e.sum(axis=1, keepdims=True)
    y = np.asarray(label, np.int64)
    loss = -np.mean(lg[np.arange(B), y] - mx[:, 0] - np.log(e.sum(axis=1)))
    dl = p.copy()
    dl[np.arange(B), y] -= 1.0
    dl /= B
    g = np.zeros(N_WEIGHTS)
    g[OFF_W2:OFF_B2] = (dl.T @ h).reshape(-1)
    g[OFF_B2:N_WEIGHTS] = dl.sum(axis=0)
    dh = (dl @ W2) * (h > 0)
    g[OFF_W1:OFF_B1] = (dh.T @ z).reshape(-1)
    g[OFF_B1:OFF_W2] = dh.sum(axis=0)
    return loss, g


def init(feat, seed=0):
    """Initial weights: standardisation from the features, small random layers."""
    rng = np.random.default_rng(seed)
    feat = np.asarray(feat, np.float64)
    w = np.zeros(N_WEIGHTS)
    w[OFF_MU:OFF_SD] = feat.mean(axis=0)
    sd = feat.std(axis=0)
    w[OFF_SD:OFF_W1] = np.where(sd > 1e-12, sd, 1.0)
    w[OFF_W1:OFF_B1] = rng.normal(0.0, 1.0 / np.sqrt(N_IN), N_HID * N_IN)
    w[OFF_W2:OFF_B2] = rng.normal(0.0, 1.0 / np.sqrt(N_HID), N_OUT * N_HID)
    return w
