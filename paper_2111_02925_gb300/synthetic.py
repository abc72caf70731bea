"""Seeded synthetic input fields (numpy PCG64), shared by the tests, the smoke
check and the benchmark.

This module only makes inputs.  It holds none of the compressor's arithmetic
and imports neither the CUDA library nor the oracle.

The SZ3 paper evaluates on scientific datasets (its dataset table: NYX
512x512x512, ATM 1800x3600, Hurricane, Miranda, ...) that are not available
here; these generators stand in for them with the same shapes, precisions and
kinds of structure:

* ``gaussian_bumps``  -- 64^3 FP32: 8 random 3-D Gaussians + one period of
  sin(x) cos(y) sin(z) per axis + N(0, sigma=1e-4) noise.
* ``grf``             -- Gaussian random field with power spectrum ~ k^-3
  (amplitude |k|^-3/2, k = 0 removed), normalised to mean 0 / variance 1,
  FP32.  At 512^3 it stands in for NYX 512^3.
* ``latlon``          -- 1800x3600 FP64 lat-lon-like field, 64 separable
  sinusoids a_k sin(m_k lon + phi_k) cos(n_k lat + psi_k), a_k ~ N(0, 1/k),
  then exactly 30% of the points set to 0.0 in random discs.  Stands in for
  ATM 1800x3600.
* ``batch_shapes``    -- the uneven 256-field mix: each axis log-uniform in
  [32, 256], REL bound log-uniform in [1e-5, 1e-2], interpolation Bernoulli(0.5).
"""
from __future__ import annotations

import math

import numpy as np

try:  # multithreaded FFT when scipy is present
    import scipy.fft as _fft

    def _irfftn(a, s):
        return _fft.irfftn(a, s=s, workers=-1)

except Exception:  # pragma: no cover
    def _irfftn(a, s):
        return np.fft.irfftn(a, s=s)


def gaussian_bumps(n: int = 64, seed: int = 1) -> np.ndarray:
    """64^3-style smooth field: 8 Gaussians (centre U[0,n)^3, sigma U[4,16],
    amplitude U[-1,1]) + sin(2 pi i/n) cos(2 pi j/n) sin(2 pi k/n) + noise."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    X, Y, Z = i[:, None, None], i[None, :, None], i[None, None, :]
    f = np.zeros((n, n, n), np.float64)
    for _ in range(8):
        c = rng.uniform(0, n, 3)
        s = rng.uniform(4, 16)
        a = rng.uniform(-1, 1)
        f += a * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * s * s))
    w = 2 * math.pi / n
    f += np.sin(w * X) * np.cos(w * Y) * np.sin(w * Z)
    f += rng.normal(0.0, 1e-4, (n, n, n))
    return f.astype(np.float32)


def grf(shape, seed: int, slope: float = -3.0) -> np.ndarray:
    """Gaussian random field with power ~ |k|^slope (FP32, mean 0, var 1)."""
    shape = tuple(int(s) for s in shape)
    rng = np.random.default_rng(seed)
    half = shape[:-1] + (shape[-1] // 2 + 1,)
    re = rng.standard_normal(half, dtype=np.float32)
    im = rng.standard_normal(half, dtype=np.float32)
    spec = re + 1j * im
    del re, im
    k2 = np.zeros(half, np.float32)
    for ax, n in enumerate(shape):
        kk = (np.fft.rfftfreq(n) if ax == len(shape) - 1 else np.fft.fftfreq(n)) * n
        sh = [1] * len(shape)
        sh[ax] = kk.size
        k2 = k2 + (kk.astype(np.float32) ** 2).reshape(sh)
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** np.float32(slope / 4.0), np.float32(0))
    spec *= amp
    del amp, k2
    f = _irfftn(spec, shape).astype(np.float32, copy=False)
    del spec
    m = float(f.mean(dtype=np.float64))
    s = float(f.std(dtype=np.float64))
    f -= np.float32(m)
    f *= np.float32(1.0 / s)
    return f


def latlon(nlat: int = 1800, nlon: int = 3600, seed: int = 3, zero_frac: float = 0.30) -> np.ndarray:
    """FP64 lat-lon-like field with `zero_frac` of its points set to 0.0 in
    random discs (radius U[20, 200] px), trimmed to the exact fraction in
    raster order of the last disc."""
    rng = np.random.default_rng(seed)
    th = np.linspace(-math.pi / 2, math.pi / 2, nlat)
    lam = np.arange(nlon) * (2 * math.pi / nlon)
    K = 64
    m = rng.integers(1, 33, K)
    nn = rng.integers(1, 33, K)
    a = rng.normal(0.0, 1.0, K) / np.sqrt(np.arange(1, K + 1))
    phi = rng.uniform(0, 2 * math.pi, K)
    psi = rng.uniform(0, 2 * math.pi, K)
    A = np.cos(np.outer(th, nn) + psi) * a  # nlat x K
    B = np.sin(np.outer(m, lam) + phi[:, None])  # K x nlon
    f = A @ B
    target = int(round(zero_frac * nlat * nlon))
    mask = np.zeros((nlat, nlon), bool)
    covered = 0
    while covered < target:
        ci, cj = rng.uniform(0, nlat), rng.uniform(0, nlon)
        r = rng.uniform(20, 200)
        i0, i1 = max(0, int(ci - r)), min(nlat, int(ci + r) + 1)
        j0, j1 = max(0, int(cj - r)), min(nlon, int(cj + r) + 1)
        ii = np.arange(i0, i1)[:, None]
        jj = np.arange(j0, j1)[None, :]
        disc = (ii - ci) ** 2 + (jj - cj) ** 2 <= r * r
        new = disc & ~mask[i0:i1, j0:j1]
        cnt = int(new.sum())
        if covered + cnt > target:
            keep = target - covered
            flat = np.flatnonzero(new)[:keep]
            new = np.zeros_like(new)
            new.flat[flat] = True
            cnt = keep
        mask[i0:i1, j0:j1] |= new
        covered += cnt
    f[mask] = 0.0
    return f


def batch_shapes(count: int = 256, seed: int = 4):
    """Shapes, REL bounds and interpolation kinds of the uneven batch mix."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(32), math.log(256)
    out = []
    for _ in range(count):
        dims = tuple(int(round(math.exp(rng.uniform(lo, hi)))) for _ in range(3))
        eb = math.exp(rng.uniform(math.log(1e-5), math.log(1e-2)))
        interp = int(rng.random() < 0.5)
        out.append((dims, eb, interp))
    return out


def grf_fronts(shape, seed: int, n_fronts: int = 16) -> np.ndarray:
    """k^-3 Gaussian random field plus n_fronts sharp fronts
    A tanh((n . p - c) / w): n uniform on the sphere, c uniform over the
    projection of the box on n, w ~ U[1, 8] cells, A ~ U[0.5, 2] (float32)."""
    x = grf(shape, seed).astype(np.float64)
    rng = np.random.default_rng(seed + 7919)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    for _ in range(n_fronts):
        nv = rng.normal(size=len(shape))
        nv /= np.linalg.norm(nv)
        corners = np.array(np.meshgrid(*[[0, n - 1] for n in shape], indexing="ij")).reshape(len(shape), -1)
        proj = nv @ corners
        c = rng.uniform(proj.min(), proj.max())
        w = rng.uniform(1.0, 8.0)
        a = rng.uniform(0.5, 2.0)
        t = sum(nv[i] * grids[i] for i in range(len(shape)))
        x += a * np.tanh((t - c) / w)
    return x.astype(np.float32)
