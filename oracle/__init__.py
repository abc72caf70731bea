"""Serial CPU oracle of the SZ3-Interp hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

The arithmetic lives in ``sz3o.c`` / ``sz3o_typed.inc`` (the hot path),
``szlz.c`` (the lossless stage after the Huffman coder) and ``szpastri.c``
(the SZ3-Pastri modules: unpred-aware quantizer, fixed Huffman code) -- plain
C, serial, compiled with ``-O2 -ffp-contract=off -fno-fast-math``; this
module only builds that library and marshals numpy arrays into it (``mlp.py``
is the selector network's numpy reference).  What each C function
computes, and the passage of the SZ3 paper (arXiv 2111.02925) it follows, is
documented in ``sz3o.h``.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, brute force, hand-worked fixtures in
``tests/golden/``) except the compression ratio itself, which the paper gives
only in figures ("parity unpinned" for the ratio).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsz3o.so")
_SOURCES = ("sz3o.c", "sz3o_typed.inc", "sz3o.h", "szlz.c", "szpastri.c")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
_lock = threading.Lock()
_lib = None

F32, F64 = 0, 1
ABS, REL = 0, 1
LINEAR, CUBIC = 0, 1
MAX_LEVELS = 32
LMAX = 24
HEADER_BYTES = 288
SUBBLOCK = 512

OK = 0
E_INVAL = -1
E_NONFINITE = -2
E_ZERO_RANGE_REL = -3
E_CAPACITY = -4
E_CORRUPT = -5
E_NOMEM = -7


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: oracle status {code}")
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("dtype", C.c_uint32),
        ("ndim", C.c_uint32),
        ("dims", C.c_uint64 * 4),
        ("eb_mode", C.c_uint32),
        ("interp", C.c_uint32),
        ("eb", C.c_double),
        ("dim_order", C.c_uint8 * 4),
        ("per_level", C.c_uint8),
        ("reserved", C.c_uint8 * 3),
        ("radius", C.c_uint32),
        ("chunk_codes", C.c_uint32),
        ("level_interp", C.c_uint8 * MAX_LEVELS),
        ("level_order", (C.c_uint8 * 4) * MAX_LEVELS),
    ]


def build(force: bool = False) -> str:
    """Compile libsz3o.so next to the sources (gcc, no GPU needed)."""
    with _lock:
        srcs = [os.path.join(_HERE, s) for s in _SOURCES]
        if not force and os.path.exists(_LIB_PATH):
            t = os.path.getmtime(_LIB_PATH)
            if all(os.path.getmtime(s) <= t for s in srcs):
                return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", *_CFLAGS, "-o", tmp, os.path.join(_HERE, "sz3o.c"), os.path.join(_HERE, "szlz.c"),
               os.path.join(_HERE, "szpastri.c"), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER(Params)
        vp, u64p = C.c_void_p, C.POINTER(C.c_uint64)
        sig = {
            "sz3o_shape": [P, u64p, C.POINTER(C.c_uint32)],
            "sz3o_error_bound": [P, vp, C.POINTER(C.c_double), vp],
            "sz3o_traversal": [P, vp, C.c_uint64],
            "sz3o_quantize1": [C.c_uint32, vp, vp, vp, C.c_uint32, C.POINTER(C.c_uint32), vp],
            "sz3o_quantize": [P, vp, vp, vp, u64p, vp, vp],
            "sz3o_recover": [P, vp, vp, vp, C.c_uint64, vp],
            "sz3o_histogram": [vp, C.c_uint64, vp],
            "sz3o_huffman_lengths": [vp, C.c_uint32, C.c_uint32, vp],
            "sz3o_canonical_codes": [vp, C.c_uint32, vp],
            "sz3o_huffman_encode": [vp, C.c_uint64, vp, vp, C.c_uint32, vp, C.c_uint64, vp, vp, u64p],
            "sz3o_huffman_decode": [vp, C.c_uint64, vp, vp, C.c_uint32, vp, C.c_uint32, vp, C.c_uint64],
            "sz3o_compress_bound": [P, u64p],
            "sz3o_compress": [P, vp, vp, C.c_uint64, u64p],
            "sz3o_read_header": [vp, C.c_uint64, P, u64p],
            "sz3o_decompress": [vp, C.c_uint64, vp, C.c_uint64],
            "sz3o_select_costs": [P, vp, C.c_uint32, C.c_uint32, C.c_uint64, vp],
            "sz3o_select_features": [P, vp, C.c_uint32, C.c_uint32, C.c_uint64, vp],
            "sz3o_lz_compress": [vp, C.c_uint64, vp, C.c_uint64, u64p],
            "sz3o_lz_decompress": [vp, C.c_uint64, vp, C.c_uint64, u64p],
            "sz3o_bitplane_exponent": [C.c_double, C.POINTER(C.c_int32)],
            "sz3o_bitplane_encode": [C.c_uint32, vp, C.c_uint64, C.c_double, vp, C.c_uint64, u64p],
            "sz3o_bitplane_decode": [vp, C.c_uint64, vp, C.c_uint64, u64p],
            "sz3o_huffman_fixed_lengths": [C.c_uint32, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.sz3o_splitmix64.argtypes = [C.c_uint64]
        L.sz3o_splitmix64.restype = C.c_uint64
        L.sz3o_select_blocks.argtypes = [P, C.c_uint32, C.c_uint32, C.c_uint64, u64p, u64p]
        L.sz3o_select_blocks.restype = C.c_uint32
        L.sz3o_lz_bound.argtypes = [C.c_uint64]
        L.sz3o_lz_bound.restype = C.c_uint64
        L.sz3o_bitplane_bound.argtypes = [C.c_uint64]
        L.sz3o_bitplane_bound.restype = C.c_uint64
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int, where: str) -> None:
    if rc != OK:
        raise OracleError(rc, where)


def make_params(dims, eb, *, dtype=F32, eb_mode=ABS, interp=LINEAR, order=None, radius=32768,
                chunk=4096, level_interp=None, level_order=None) -> Params:
    """Parameter block.  ``level_interp`` / ``level_order`` map level l (1..L)
    to a choice and switch on the per-level override."""
    p = Params()
    dims = [int(d) for d in dims]
    p.dtype = dtype
    p.ndim = len(dims)
    for i in range(4):
        p.dims[i] = dims[i] if i < len(dims) else 1
    p.eb_mode = eb_mode
    p.interp = interp
    p.eb = float(eb)
    order = list(range(len(dims))) if order is None else list(order)
    for i in range(4):
        p.dim_order[i] = order[i] if i < len(order) else 0
    p.radius = radius
    p.chunk_codes = chunk
    if level_interp is not None or level_order is not None:
        p.per_level = 1
        for l in range(1, MAX_LEVELS):
            li = (level_interp or {}).get(l, interp)
            lo = (level_order or {}).get(l, order)
            p.level_interp[l] = li
            for i in range(4):
                p.level_order[l][i] = lo[i] if i < len(lo) else 0
    return p


def np_dtype(p: Params):
    return np.float32 if p.dtype == F32 else np.float64


def shape(p: Params):
    n, L = C.c_uint64(), C.c_uint32()
    _check(lib().sz3o_shape(C.byref(p), C.byref(n), C.byref(L)), "shape")
    return n.value, L.value


def error_bound(p: Params, x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np_dtype(p))
    eb_abs = C.c_double()
    ebT = np.zeros(1, dtype=np_dtype(p))
    _check(lib().sz3o_error_bound(C.byref(p), _ptr(x), C.byref(eb_abs), _ptr(ebT)), "error_bound")
    return eb_abs.value, ebT[0]


def traversal(p: Params) -> np.ndarray:
    n, _ = shape(p)
    out = np.zeros(n, dtype=np.uint64)
    _check(lib().sz3o_traversal(C.byref(p), _ptr(out), n), "traversal")
    return out


def quantize1(x, pred, ebT, radius=32768, dtype=F32):
    t = np.float32 if dtype == F32 else np.float64
    xa, pa, ea = np.array([x], t), np.array([pred], t), np.array([ebT], t)
    r = np.zeros(1, t)
    code = C.c_uint32()
    _check(lib().sz3o_quantize1(dtype, _ptr(xa), _ptr(pa), _ptr(ea), radius, C.byref(code), _ptr(r)),
           "quantize1")
    return code.value, r[0]


def quantize(p: Params, x: np.ndarray):
    """Returns (codes uint16[N], unpred T[n_unpred], recon T[N], eb_T)."""
    t = np_dtype(p)
    x = np.ascontiguousarray(x, dtype=t).reshape(-1)
    n, _ = shape(p)
    codes = np.zeros(n, np.uint16)
    unpred = np.zeros(n, t)
    recon = np.zeros(n, t)
    nu = C.c_uint64()
    ebT = np.zeros(1, t)
    _check(lib().sz3o_quantize(C.byref(p), _ptr(x), _ptr(codes), _ptr(unpred), C.byref(nu), _ptr(recon),
                               _ptr(ebT)), "quantize")
    return codes, unpred[: nu.value].copy(), recon, ebT[0]


def recover(p: Params, ebT, codes: np.ndarray, unpred: np.ndarray) -> np.ndarray:
    t = np_dtype(p)
    n, _ = shape(p)
    e = np.array([ebT], t)
    codes = np.ascontiguousarray(codes, np.uint16)
    unpred = np.ascontiguousarray(unpred, t)
    out = np.zeros(n, t)
    _check(lib().sz3o_recover(C.byref(p), _ptr(e), _ptr(codes), _ptr(unpred) if unpred.size else None,
                              unpred.size, _ptr(out)), "recover")
    return out


def histogram(codes: np.ndarray) -> np.ndarray:
    codes = np.ascontiguousarray(codes, np.uint16)
    h = np.zeros(65536, np.uint64)
    _check(lib().sz3o_histogram(_ptr(codes), codes.size, _ptr(h)), "histogram")
    return h


def huffman_lengths(freq, lmax=LMAX) -> np.ndarray:
    f = np.ascontiguousarray(freq, np.uint64)
    ln = np.zeros(f.size, np.uint8)
    _check(lib().sz3o_huffman_lengths(_ptr(f), f.size, lmax, _ptr(ln)), "huffman_lengths")
    return ln


def canonical_codes(lengths) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, np.uint8)
    c = np.zeros(ln.size, np.uint32)
    _check(lib().sz3o_canonical_codes(_ptr(ln), ln.size, _ptr(c)), "canonical_codes")
    return c


def sub_blocks(chunk: int) -> int:
    """Sub-block entries recorded per chunk."""
    return (chunk + SUBBLOCK - 1) // SUBBLOCK - 1


def huffman_encode(codes, lengths, canon, chunk=4096, with_sub=False):
    """Returns (payload words, words per chunk[, sub-block bit lengths])."""
    codes = np.ascontiguousarray(codes, np.uint16)
    ln = np.ascontiguousarray(lengths, np.uint8)
    cc = np.ascontiguousarray(canon, np.uint32)
    nch = (codes.size + chunk - 1) // chunk
    cap = nch * ((chunk * LMAX + 31) // 32)
    words = np.zeros(max(cap, 1), np.uint32)
    cw = np.zeros(max(nch, 1), np.uint32)
    sub = np.zeros(max(nch * sub_blocks(chunk), 1), np.uint16)
    nw = C.c_uint64()
    _check(lib().sz3o_huffman_encode(_ptr(codes), codes.size, _ptr(ln), _ptr(cc), chunk, _ptr(words), cap,
                                     _ptr(cw), _ptr(sub), C.byref(nw)), "huffman_encode")
    out = (words[: nw.value].copy(), cw[:nch].copy())
    if with_sub:
        out = out + (sub[: nch * sub_blocks(chunk)].copy(),)
    return out


def huffman_decode(words, chunk_words, lengths, n, chunk=4096, sub_bits=None) -> np.ndarray:
    w = np.ascontiguousarray(words, np.uint32)
    cw = np.ascontiguousarray(chunk_words, np.uint32)
    ln = np.ascontiguousarray(lengths, np.uint8)
    sb = None if sub_bits is None else np.ascontiguousarray(sub_bits, np.uint16)
    out = np.zeros(n, np.uint16)
    _check(lib().sz3o_huffman_decode(_ptr(w) if w.size else None, w.size, _ptr(cw),
                                     _ptr(sb) if sb is not None and sb.size else None, chunk, _ptr(ln), ln.size,
                                     _ptr(out), n), "huffman_decode")
    return out


def compress_bound(p: Params) -> int:
    b = C.c_uint64()
    _check(lib().sz3o_compress_bound(C.byref(p), C.byref(b)), "compress_bound")
    return b.value


def compress(p: Params, x: np.ndarray) -> bytes:
    x = np.ascontiguousarray(x, dtype=np_dtype(p)).reshape(-1)
    cap = compress_bound(p)
    out = np.zeros(cap, np.uint8)
    nb = C.c_uint64()
    _check(lib().sz3o_compress(C.byref(p), _ptr(x), _ptr(out), cap, C.byref(nb)), "compress")
    return out[: nb.value].tobytes()


def compress_status(p: Params, x: np.ndarray) -> int:
    """Status code of sz3o_compress (for error-path tests)."""
    x = np.ascontiguousarray(x, dtype=np_dtype(p)).reshape(-1)
    try:
        cap = compress_bound(p)
    except OracleError as e:
        return e.code
    out = np.zeros(cap, np.uint8)
    nb = C.c_uint64()
    return lib().sz3o_compress(C.byref(p), _ptr(x), _ptr(out), cap, C.byref(nb))


def read_header(stream: bytes):
    buf = np.frombuffer(stream, np.uint8)
    p = Params()
    n = C.c_uint64()
    _check(lib().sz3o_read_header(_ptr(buf) if buf.size else None, buf.size, C.byref(p), C.byref(n)),
           "read_header")
    return p, n.value


def decompress_status(stream: bytes, out: np.ndarray) -> int:
    buf = np.frombuffer(stream, np.uint8)
    return lib().sz3o_decompress(_ptr(buf) if buf.size else None, buf.size, _ptr(out), out.nbytes)


def decompress(stream: bytes) -> np.ndarray:
    p, n = read_header(stream)
    out = np.zeros(n, np_dtype(p))
    _check(decompress_status(stream, out), "decompress")
    return out


# ---------------------------------------------------------------------------
# Per-level selection of interpolation and axis order (rank <= 3).
# ---------------------------------------------------------------------------
SEL_CANDIDATES = 8
SEL_FEATURES = 16
_SEL_ORDERS = {3: [(0, 1, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)], 2: [(0, 1), (1, 0), (0, 1), (1, 0)], 1: [(0,)] * 4}


def candidate(ndim: int, c: int):
    """(interp, axis order) of candidate c = 2 o + interp."""
    return c % 2, _SEL_ORDERS[ndim][c // 2]


def select_costs(p: Params, x: np.ndarray, level: int, nblocks: int = 0, seed: int = 0) -> np.ndarray:
    """Estimated bits of level `level` under the 8 candidates (all points of
    the level when nblocks == 0, else those in the seeded sample blocks)."""
    x = np.ascontiguousarray(x, dtype=np_dtype(p)).reshape(-1)
    out = np.zeros(SEL_CANDIDATES, np.float64)
    _check(lib().sz3o_select_costs(C.byref(p), _ptr(x), level, nblocks, seed, _ptr(out)), "select_costs")
    return out


def select_features(p: Params, x: np.ndarray, level: int, nblocks: int = 0, seed: int = 0) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np_dtype(p)).reshape(-1)
    out = np.zeros(SEL_FEATURES, np.float64)
    _check(lib().sz3o_select_features(C.byref(p), _ptr(x), level, nblocks, seed, _ptr(out)), "select_features")
    return out


def splitmix64(key: int) -> int:
    """The SplitMix64 output function of the sample-block placement."""
    return int(lib().sz3o_splitmix64(key & 0xFFFFFFFFFFFFFFFF))


def select_blocks(p: Params, level: int, nblocks: int, seed: int):
    """(lo, hi): int arrays [n, ndim] of the sample blocks of `level`."""
    nd = int(p.ndim)
    lo = np.zeros(4 * 1024, np.uint64)
    hi = np.zeros(4 * 1024, np.uint64)
    n = int(lib().sz3o_select_blocks(C.byref(p), level, nblocks, seed & 0xFFFFFFFFFFFFFFFF,
                                     lo.ctypes.data_as(C.POINTER(C.c_uint64)),
                                     hi.ctypes.data_as(C.POINTER(C.c_uint64))))
    return (lo.reshape(1024, 4)[:n, :nd].astype(np.int64), hi.reshape(1024, 4)[:n, :nd].astype(np.int64))


def select_levels(p: Params, x: np.ndarray, nblocks: int = 0, seed: int = 0):
    """{level: candidate} minimising the estimated bits of every level
    (ties: the lower candidate)."""
    _, L = shape(p)
    return {l: int(np.argmin(select_costs(p, x, l, nblocks, seed))) for l in range(1, L + 1)}


def params_for_choices(p: Params, dims, choices) -> Params:
    """Copy of p with the per-level interpolation / order of `choices`."""
    nd = len(dims)
    li = {l: candidate(nd, c)[0] for l, c in choices.items()}
    lo = {l: list(candidate(nd, c)[1]) for l, c in choices.items()}
    q = make_params(dims, p.eb, dtype=p.dtype, eb_mode=p.eb_mode, interp=p.interp,
                    order=[p.dim_order[i] for i in range(nd)], radius=p.radius, chunk=p.chunk_codes,
                    level_interp=li, level_order=lo)
    return q


LZ_BLOCK = 32768


def lz_compress(data: bytes) -> bytes:
    """The lossless stage (szlz.c): byte-level LZ77 over 32 KiB blocks."""
    n = len(data)
    src = np.frombuffer(data, np.uint8) if n else np.zeros(1, np.uint8)
    cap = int(lib().sz3o_lz_bound(n))
    out = np.zeros(cap, np.uint8)
    nb = C.c_uint64(0)
    _check(lib().sz3o_lz_compress(_ptr(src), n, _ptr(out), cap, C.byref(nb)), "sz3o_lz_compress")
    return out[: nb.value].tobytes()


def lz_decompress_status(stream: bytes, cap: int):
    """(status, bytes) of decoding an SZLZ stream into at most cap bytes."""
    src = np.frombuffer(stream, np.uint8) if len(stream) else np.zeros(1, np.uint8)
    out = np.zeros(max(cap, 1), np.uint8)
    n = C.c_uint64(0)
    rc = lib().sz3o_lz_decompress(_ptr(src), len(stream), _ptr(out), cap, C.byref(n))
    return rc, (out[: n.value].tobytes() if rc == OK else b"")


def lz_decompress(stream: bytes) -> bytes:
    if len(stream) < 16:
        raise OracleError(E_CORRUPT, "sz3o_lz_decompress")
    n = int(np.frombuffer(stream[8:16], np.uint64)[0])
    rc, out = lz_decompress_status(stream, n)
    _check(rc, "sz3o_lz_decompress")
    return out


# ---- SZ3-Pastri modules (szpastri.c) ----------------------------------------
BP_HEADER = 32


def bitplane_exponent(eb: float) -> int:
    """e = floor(log2(eb)) of the unpred-aware quantizer (Sec. 4.2)."""
    e = C.c_int32()
    _check(lib().sz3o_bitplane_exponent(eb, C.byref(e)), "sz3o_bitplane_exponent")
    return e.value


def bitplane_encode_status(values: np.ndarray, eb: float):
    """(status, stream bytes) of the unpred-aware quantizer on a float32 /
    float64 array."""
    v = np.ascontiguousarray(values).reshape(-1)
    dt = {np.dtype(np.float32): F32, np.dtype(np.float64): F64}[v.dtype]
    cap = int(lib().sz3o_bitplane_bound(v.size))
    out = np.zeros(max(cap, 1), np.uint8)
    nb = C.c_uint64()
    rc = lib().sz3o_bitplane_encode(dt, _ptr(v), v.size, eb, _ptr(out), cap, C.byref(nb))
    return rc, (out[:nb.value].tobytes() if rc == OK else b"")


def bitplane_encode(values: np.ndarray, eb: float) -> bytes:
    rc, s = bitplane_encode_status(values, eb)
    _check(rc, "sz3o_bitplane_encode")
    return s


def bitplane_decode_status(stream: bytes, n: int, dtype):
    out = np.zeros(max(n, 1), dtype)
    buf = np.frombuffer(stream, np.uint8) if len(stream) else np.zeros(1, np.uint8)
    nn = C.c_uint64()
    rc = lib().sz3o_bitplane_decode(_ptr(buf), len(stream), _ptr(out), n * np.dtype(dtype).itemsize, C.byref(nn))
    return rc, out[:nn.value] if rc == OK else None


def bitplane_decode(stream: bytes) -> np.ndarray:
    n = int(np.frombuffer(stream[8:16], np.uint64)[0])
    dt = np.float32 if int(np.frombuffer(stream[4:8], np.uint32)[0]) == F32 else np.float64
    rc, out = bitplane_decode_status(stream, n, dt)
    _check(rc, "sz3o_bitplane_decode")
    return out


def huffman_fixed_lengths(radius: int) -> np.ndarray:
    """Predefined code lengths over the 2 radius quantization codes."""
    out = np.zeros(2 * radius, np.uint8)
    _check(lib().sz3o_huffman_fixed_lengths(radius, _ptr(out)), "sz3o_huffman_fixed_lengths")
    return out
