"""GPU parity: the CUDA path (called through the C ABI) against the oracle,
element by element on seeded inputs.  Integer and byte results (codes,
unpredictable lists, histograms, code lengths, payload words, whole streams)
must be identical; reconstructed floats must be bit-identical, because both
sides evaluate the same operations in the same order in the field's type.
"""
import numpy as np
import pytest

import oracle as O
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


def both_params(dims, eb, **kw):
    return O.make_params(dims, eb, **kw), G.make_params(dims, eb, **kw)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_predict_quantize(gp, x):
    t = torch.float32 if gp.dtype == G.F32 else torch.float64
    xd = dev(x.reshape(-1)).to(t)
    n = x.size
    codes = torch.empty(n, dtype=torch.int16, device=DEV)
    unpred = torch.empty(max(n, 1), dtype=t, device=DEV)
    hist = torch.empty(65536, dtype=torch.int32, device=DEV)
    rc, nu, eb = G.sz3g_predict_quantize(gp, xd.data_ptr(), codes.data_ptr(), unpred.data_ptr(), hist.data_ptr(),
                                         stream=G._stream_handle())
    return rc, codes.cpu().numpy().view(np.uint16), unpred[:nu].cpu().numpy(), hist.cpu().numpy().view(np.uint32), eb


def gpu_compress(gp, x, cap=None):
    t = torch.float32 if gp.dtype == G.F32 else torch.float64
    xd = dev(x.reshape(-1)).to(t)
    cap = cap if cap is not None else G.sz3g_compress_bound(gp)
    out = torch.empty(max(cap, 16), dtype=torch.uint8, device=DEV)
    rc, nb = G.sz3g_compress(gp, xd.data_ptr(), out.data_ptr(), cap, stream=G._stream_handle())
    return rc, out[:nb].cpu().numpy().tobytes()


def gpu_decompress(stream: bytes, n, dtype):
    s = torch.from_numpy(np.frombuffer(stream, np.uint8).copy()).to(DEV)
    t = torch.float32 if dtype == G.F32 else torch.float64
    out = torch.empty(max(n, 1), dtype=t, device=DEV)
    rc = G.sz3g_decompress(s.data_ptr(), len(stream), out.data_ptr(), n * out.element_size(),
                           stream=G._stream_handle())
    return rc, out[:n].cpu().numpy()


CASES = [
    # name, field maker, dtype, eb_mode, eb, interp, order, radius, chunk
    ("bumps64_lin", lambda: S.gaussian_bumps(64, 1), O.F32, O.ABS, 1e-3 * 3.1, O.LINEAR, (0, 1, 2), 32768, 4096),
    ("grf_ragged_cubic", lambda: S.grf((37, 50, 29), 2), O.F32, O.REL, 1e-3, O.CUBIC, (0, 1, 2), 32768, 4096),
    ("grf_order201", lambda: S.grf((33, 17, 65), 3), O.F32, O.REL, 1e-2, O.CUBIC, (2, 0, 1), 32768, 512),
    ("grf_tight_unpred", lambda: S.grf((24, 24, 24), 4), O.F32, O.REL, 1e-5, O.LINEAR, (1, 2, 0), 64, 256),
    ("latlon_lin", lambda: S.latlon(180, 360, 3), O.F64, O.ABS, 1e-6 * 9.0, O.LINEAR, (0, 1), 32768, 4096),
    ("latlon_cubic", lambda: S.latlon(181, 363, 5), O.F64, O.ABS, 1e-5, O.CUBIC, (1, 0), 32768, 4096),
    ("grf1d", lambda: S.grf((5000,), 6), O.F32, O.REL, 1e-3, O.CUBIC, (0,), 32768, 1024),
    ("grf4d", lambda: S.grf((7, 9, 6, 10), 7), O.F32, O.REL, 1e-3, O.LINEAR, (3, 1, 0, 2), 32768, 256),
    # 3-D FP64 on the register-blocked level kernel: G_0 stages its code rows
    # by tensor copies (rows of 40 odd-k codes), G_1 by per-row copies (20)
    ("grf3d_f64_cubic", lambda: S.grf((40, 48, 80), 12).astype(np.float64), O.F64, O.REL, 1e-4, O.CUBIC,
     (0, 1, 2), 32768, 4096),
    # 2-D FP32: code rows by per-row copies (rows of 100 odd-k codes) and,
    # on the power-of-two grid, by tensor copies
    ("grf2d_f32_cubic", lambda: S.grf((136, 200), 13), O.F32, O.REL, 1e-3, O.CUBIC, (0, 1), 32768, 4096),
    ("grf2d_f32_pow2_lin", lambda: S.grf((128, 256), 14), O.F32, O.REL, 1e-3, O.LINEAR, (0, 1), 32768, 4096),
    ("grf4d_f64", lambda: S.grf((5, 8, 9, 6), 8).astype(np.float64), O.F64, O.REL, 1e-4, O.CUBIC, (0, 1, 2, 3), 512,
     64),
    ("tiny_1", lambda: np.array([3.5], np.float32), O.F32, O.ABS, 0.1, O.LINEAR, (0,), 32768, 4096),
    ("tiny_2x1x3", lambda: np.arange(6, dtype=np.float32).reshape(2, 1, 3), O.F32, O.ABS, 0.1, O.CUBIC, (0, 1, 2),
     32768, 8),
    ("all_unpred", lambda: S.grf((12, 13, 14), 9), O.F32, O.REL, 1e-7, O.LINEAR, (0, 1, 2), 2, 8),
]


def _case(c):
    name, make, dtype, mode, eb, interp, order, radius, chunk = c
    x = make()
    x = x.astype(np.float32 if dtype == O.F32 else np.float64)
    kw = dict(dtype=dtype, eb_mode=mode, interp=interp, order=order, radius=radius, chunk=chunk)
    op, gp = both_params(x.shape, eb, **kw)
    return x, op, gp


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_predict_quantize_matches_oracle(case):
    x, op, gp = _case(case)
    codes, unpred, recon, ebT = O.quantize(op, x)
    rc, gcodes, gunpred, ghist, geb = gpu_predict_quantize(gp, x)
    assert rc == G.OK
    t = np.float32 if op.dtype == O.F32 else np.float64
    assert np.frombuffer(geb[: np.dtype(t).itemsize], t)[0] == ebT
    assert np.array_equal(gcodes, codes), f"first diff at {np.flatnonzero(gcodes != codes)[:5]}"
    assert np.array_equal(gunpred.view(np.uint8), unpred.view(np.uint8))
    assert np.array_equal(ghist.astype(np.uint64), O.histogram(codes))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_recover_matches_oracle(case):
    x, op, gp = _case(case)
    codes, unpred, recon, ebT = O.quantize(op, x)
    t = torch.float32 if op.dtype == O.F32 else torch.float64
    out = torch.empty(x.size, dtype=t, device=DEV)
    cd = dev(codes.view(np.int16))
    ud = dev(unpred) if unpred.size else torch.empty(1, dtype=t, device=DEV)
    ebb = np.array([ebT]).astype(np.float32 if op.dtype == O.F32 else np.float64).tobytes()
    rc = G.sz3g_recover(gp, ebb, cd.data_ptr(), ud.data_ptr(), unpred.size, out.data_ptr(), stream=G._stream_handle())
    assert rc == G.OK
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.uint8), recon.view(np.uint8))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_stream_matches_oracle_bytes(case):
    x, op, gp = _case(case)
    s_or = O.compress(op, x)
    rc, s_gpu = gpu_compress(gp, x)
    assert rc == G.OK
    assert len(s_gpu) == len(s_or)
    if s_gpu != s_or:
        a, b = np.frombuffer(s_gpu, np.uint8), np.frombuffer(s_or, np.uint8)
        raise AssertionError(f"stream differs first at byte {np.flatnonzero(a != b)[:8]}")
    rc, y = gpu_decompress(s_or, x.size, op.dtype)
    assert rc == G.OK
    recon = O.quantize(op, x)[2]
    assert np.array_equal(y.view(np.uint8), recon.view(np.uint8))


@pytest.mark.parametrize("seed,nsym,spread", [(0, 65536, 3.0), (1, 65536, 300.0), (2, 1024, 20.0), (3, 8, 0.3),
                                             (4, 65536, 20000.0), (5, 65536, 1100.0), (6, 65536, 2600.0)])
def test_huffman_build_encode_decode(seed, nsym, spread):
    rng = np.random.default_rng(seed)
    n = 200_003
    c = nsym // 2 if nsym > 2 else 0
    codes = np.clip(np.round(rng.laplace(c, spread, n)), 0, nsym - 1).astype(np.uint16)
    hist = O.histogram(codes)
    ln = O.huffman_lengths(hist[:nsym])
    cc = O.canonical_codes(ln)
    hd = dev(hist.astype(np.uint32).view(np.int32))
    glen = torch.empty(nsym, dtype=torch.uint8, device=DEV)
    gcode = torch.empty(nsym, dtype=torch.int32, device=DEV)
    assert G.sz3g_huffman_build(hd.data_ptr(), nsym, glen.data_ptr(), gcode.data_ptr(), G._stream_handle()) == G.OK
    assert np.array_equal(glen.cpu().numpy(), ln)
    assert np.array_equal(gcode.cpu().numpy().view(np.uint32), cc)
    for chunk in (8, 1000 * 8, 4096, 520):
        words, cw, sub = O.huffman_encode(codes, ln, cc, chunk, with_sub=True)
        cd = dev(codes.view(np.int16))
        nch = (n + chunk - 1) // chunk
        nsb = O.sub_blocks(chunk)
        cap = nch * ((chunk * 24 + 31) // 32)
        gw = torch.zeros(cap, dtype=torch.int32, device=DEV)
        gcw = torch.zeros(nch, dtype=torch.int32, device=DEV)
        gsub = torch.zeros(max(nch * nsb, 1), dtype=torch.int16, device=DEV)
        rc, nw = G.sz3g_huffman_encode(cd.data_ptr(), n, glen.data_ptr(), gcode.data_ptr(), nsym, chunk, gw.data_ptr(),
                                       cap, gcw.data_ptr(), gsub.data_ptr(), G._stream_handle())
        assert rc == G.OK and nw == words.size
        assert np.array_equal(gcw.cpu().numpy().view(np.uint32), cw)
        assert np.array_equal(gw[:nw].cpu().numpy().view(np.uint32), words)
        assert np.array_equal(gsub[:nch * nsb].cpu().numpy().view(np.uint16), sub)
        for use_sub in (True, False):
            back = torch.empty(n, dtype=torch.int16, device=DEV)
            rc = G.sz3g_huffman_decode(gw.data_ptr(), nw, gcw.data_ptr(), gsub.data_ptr() if use_sub else 0, chunk,
                                       glen.data_ptr(), nsym, back.data_ptr(), n, G._stream_handle())
            assert rc == G.OK
            assert np.array_equal(back.cpu().numpy().view(np.uint16), codes)
        if nsb:  # a moved sub-block boundary is reported
            bad = gsub.clone()
            bad[0] += 1
            back = torch.empty(n, dtype=torch.int16, device=DEV)
            rc = G.sz3g_huffman_decode(gw.data_ptr(), nw, gcw.data_ptr(), bad.data_ptr(), chunk, glen.data_ptr(), nsym,
                                       back.data_ptr(), n, G._stream_handle())
            assert rc == G.E_CORRUPT


def test_length_limit_matches_oracle():
    fib = [1, 1]
    while len(fib) < 30:
        fib.append(fib[-1] + fib[-2])
    hist = np.zeros(65536, np.uint64)
    hist[100:130] = fib
    ln = O.huffman_lengths(hist)
    hd = dev(hist.astype(np.uint32).view(np.int32))
    glen = torch.empty(65536, dtype=torch.uint8, device=DEV)
    gcode = torch.empty(65536, dtype=torch.int32, device=DEV)
    assert G.sz3g_huffman_build(hd.data_ptr(), 65536, glen.data_ptr(), gcode.data_ptr(), G._stream_handle()) == G.OK
    assert np.array_equal(glen.cpu().numpy(), ln)
    assert glen.cpu().numpy().max() <= 24


@pytest.mark.parametrize("nfib", [26, 30, 36, 44])
def test_length_limit_rounds_match_oracle(nfib):
    # Fibonacci weights: one halving round after another is needed, up to
    # beyond the rounds the codebook kernel tries at once
    fib = [1, 1]
    while len(fib) < nfib:
        fib.append(fib[-1] + fib[-2])
    hist = np.zeros(65536, np.uint64)
    hist[1000:1000 + nfib] = fib
    ln = O.huffman_lengths(hist)
    hd = dev(hist.astype(np.uint32).view(np.int32))
    glen = torch.empty(65536, dtype=torch.uint8, device=DEV)
    gcode = torch.empty(65536, dtype=torch.int32, device=DEV)
    assert G.sz3g_huffman_build(hd.data_ptr(), 65536, glen.data_ptr(), gcode.data_ptr(), G._stream_handle()) == G.OK
    assert np.array_equal(glen.cpu().numpy(), ln)
    assert np.array_equal(gcode.cpu().numpy().view(np.uint32), O.canonical_codes(ln))


def test_codebook_rounds_beyond_the_parallel_ones():
    # 500 heavy symbols above an 18-long Fibonacci chain scaled by 256: 518
    # used symbols whose code fits 24 bits only at halving round 9 -- past the
    # eight rounds computed at once, so the sequential rounds finish it
    fib = [1, 1]
    while len(fib) < 18:
        fib.append(fib[-1] + fib[-2])
    hist = np.zeros(65536, np.uint64)
    hist[3000:3018] = [f * 256 for f in fib]
    hist[20000:20500] = 2_900_000
    assert int(hist.sum()) < 2 ** 31
    ln = O.huffman_lengths(hist)
    hd = dev(hist.astype(np.uint32).view(np.int32))
    glen = torch.empty(65536, dtype=torch.uint8, device=DEV)
    gcode = torch.empty(65536, dtype=torch.int32, device=DEV)
    assert G.sz3g_huffman_build(hd.data_ptr(), 65536, glen.data_ptr(), gcode.data_ptr(), G._stream_handle()) == G.OK
    assert np.array_equal(glen.cpu().numpy(), ln)
    assert np.array_equal(gcode.cpu().numpy().view(np.uint32), O.canonical_codes(ln))


@pytest.mark.parametrize("k", [2, 3, 511, 512, 513, 900, 3000, 12000, 40000])
def test_codebook_alphabet_sizes_match_oracle(k):
    # steeply falling weights over k symbols (deep trees, several rounds)
    rng = np.random.default_rng(k)
    w = np.floor(2.0 ** (30.0 * (1.0 - np.arange(k) / k))).astype(np.uint64) // max(1, k // 16) + 1
    assert w.sum() < 2 ** 31  # totals of a field of at most 2^31 points
    hist = np.zeros(65536, np.uint64)
    hist[rng.permutation(65536)[:k]] = w
    ln = O.huffman_lengths(hist)
    hd = dev(hist.astype(np.uint32).view(np.int32))
    glen = torch.empty(65536, dtype=torch.uint8, device=DEV)
    gcode = torch.empty(65536, dtype=torch.int32, device=DEV)
    assert G.sz3g_huffman_build(hd.data_ptr(), 65536, glen.data_ptr(), gcode.data_ptr(), G._stream_handle()) == G.OK
    assert np.array_equal(glen.cpu().numpy(), ln)
    assert np.array_equal(gcode.cpu().numpy().view(np.uint32), O.canonical_codes(ln))


def test_error_statuses_match_oracle():
    x = np.zeros((8, 8, 8), np.float32)
    op, gp = both_params(x.shape, 1e-3, eb_mode=O.REL)
    assert gpu_compress(gp, x)[0] == G.E_ZERO_RANGE_REL == O.compress_status(op, x)
    y = S.grf((8, 8, 8), 1)
    y[3, 3, 3] = np.nan
    for mode in (O.ABS, O.REL):
        op, gp = both_params(y.shape, 1e-3, eb_mode=mode)
        assert gpu_compress(gp, y)[0] == G.E_NONFINITE == O.compress_status(op, y)
    op, gp = both_params(x.shape, 1e-60)
    assert gpu_compress(gp, x)[0] == G.E_INVAL == O.compress_status(op, x)
    # output buffer too small
    z = S.grf((16, 16, 16), 2)
    op, gp = both_params(z.shape, 1e-4, eb_mode=O.REL)
    need = len(O.compress(op, z))
    assert gpu_compress(gp, z, cap=need)[0] == G.OK
    assert gpu_compress(gp, z, cap=need - 8)[0] == G.E_CAPACITY
    assert gpu_compress(gp, z, cap=400)[0] == G.E_CAPACITY


def test_corrupt_streams_are_rejected():
    x = S.grf((20, 20, 20), 5)
    op, gp = both_params(x.shape, 1e-3, eb_mode=O.REL, chunk=256)
    s = bytearray(O.compress(op, x))
    import struct

    assert gpu_decompress(bytes(s), x.size, O.F32)[0] == G.OK
    for cut in (0, 100, 287, len(s) // 2, len(s) - 1):
        t = torch.from_numpy(np.frombuffer(bytes(s[:max(cut, 1)]), np.uint8).copy()).to(DEV)
        out = torch.empty(x.size, dtype=torch.float32, device=DEV)
        assert G.sz3g_decompress(t.data_ptr(), cut, out.data_ptr(), x.size * 4, stream=G._stream_handle()) == G.E_CORRUPT
    b = bytearray(s)
    b[0] = ord("X")
    assert gpu_decompress(bytes(b), x.size, O.F32)[0] == G.E_CORRUPT
    n_unpred = struct.unpack_from("<Q", s, 88)[0]
    n_used = struct.unpack_from("<I", s, 76)[0]
    off_table = 288 + ((n_unpred * 4 + 7) & ~7)
    b = bytearray(s)
    b[off_table + 2] = 30
    assert gpu_decompress(bytes(b), x.size, O.F32)[0] == G.E_CORRUPT
    off_chunks = off_table + ((n_used * 3 + 7) & ~7)
    b = bytearray(s)
    struct.pack_into("<I", b, off_chunks, struct.unpack_from("<I", s, off_chunks)[0] + 1)
    assert gpu_decompress(bytes(b), x.size, O.F32)[0] == G.E_CORRUPT
    rng = np.random.default_rng(1)
    nch = struct.unpack_from("<Q", s, 96)[0]
    off_payload = off_chunks + ((nch * 4 + 7) & ~7)  # chunk 256: no sub-block table
    for _ in range(20):  # random payload bit flips: decode or report, never crash
        b = bytearray(s)
        i = int(rng.integers(off_payload, len(s)))
        b[i] ^= 1 << int(rng.integers(8))
        assert gpu_decompress(bytes(b), x.size, O.F32)[0] in (G.OK, G.E_CORRUPT)


# ---- full-size workloads (the benchmark's launch configuration) -------------------
def test_full_64cube_bumps_abs_linear():
    x = S.gaussian_bumps(64, 1)
    eb = 1e-3 * float(x.max() - x.min())
    op, gp = both_params(x.shape, eb, interp=O.LINEAR)
    rc, s = gpu_compress(gp, x)
    assert rc == G.OK and s == O.compress(op, x)


@pytest.mark.parametrize("interp", [O.LINEAR, O.CUBIC])
def test_full_latlon_fp64(interp):
    x = S.latlon(1800, 3600, 3)
    eb = 1e-6 * float(x.max() - x.min())
    op, gp = both_params(x.shape, eb, dtype=O.F64, interp=interp)
    rc, s = gpu_compress(gp, x)
    assert rc == G.OK
    ref = O.compress(op, x)
    assert s == ref
    rc, y = gpu_decompress(s, x.size, O.F64)
    assert rc == G.OK
    assert np.array_equal(y, O.decompress(ref))
    assert np.max(np.abs(y - x.ravel())) <= eb


_GRF512 = {}


def _grf512():
    if "x" not in _GRF512:
        _GRF512["x"] = S.grf((512, 512, 512), 2)
    return _GRF512["x"]


@pytest.mark.parametrize("eb", [1e-4, 1e-5, 1e-6])
def test_large_alphabets_whole_stream(eb):
    # thousands to all 65536 codes used: the codebook's parallel length-limit
    # rounds (shared-memory and global-scratch forms) inside the pipeline
    x = S.grf((128, 128, 128), 6).astype(np.float32)
    op, gp = both_params(x.shape, eb, eb_mode=O.REL, interp=O.CUBIC)
    rc, s = gpu_compress(gp, x)
    assert rc == G.OK
    assert s == O.compress(op, x)
    rc, y = gpu_decompress(s, x.size, O.F32)
    assert rc == G.OK
    assert np.array_equal(y.view(np.uint32), O.decompress(s).reshape(-1).view(np.uint32))


@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4])
def test_full_512cube_rel_cubic(eb):
    """The benchmark's field in the benchmark's launch configuration: the
    whole compressed stream and every reconstructed value against the oracle,
    at each bound of the sweep."""
    x = _grf512()
    op, gp = both_params(x.shape, eb, eb_mode=O.REL, interp=O.CUBIC)
    rc, s = gpu_compress(gp, x)
    assert rc == G.OK
    ref = O.compress(op, x)
    assert s == ref
    rc, y = gpu_decompress(s, x.size, O.F32)
    assert rc == G.OK
    want = O.decompress(ref).reshape(-1)
    assert np.array_equal(y.view(np.uint32), want.view(np.uint32))
    eb_abs = eb * (float(x.max()) - float(x.min()))
    assert float(np.max(np.abs(y.astype(np.float64) - x.ravel()))) <= eb_abs
