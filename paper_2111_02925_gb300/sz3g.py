"""Python binding of libsz3g.so (the C ABI in include/sz3g.h).

Argument marshalling only: every step of compression and decompression runs
in the library's CUDA kernels.  PyTorch supplies device memory and the
stream.  If the library has not been built, every call raises -- there is no
CPU fallback.

Functions named ``sz3g_*`` mirror the C entry points one to one and take raw
pointers (ints); the lower-case helpers below them take torch tensors.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

F32, F64 = 0, 1
ABS, REL = 0, 1
LINEAR, CUBIC = 0, 1
MAX_LEVELS = 32
LMAX = 24
HEADER_BYTES = 288

OK = 0
E_INVAL = -1
E_NONFINITE = -2
E_ZERO_RANGE_REL = -3
E_CAPACITY = -4
E_CORRUPT = -5
E_CUDA = -6
E_NOMEM = -7
E_TIMEOUT = -8
E_CHECK = -9  # checking build only


class SZ3GError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {code} ({strerror(code) if _lib else 'library not loaded'})")
        self.code = code


class Params(C.Structure):
    """sz3g_params (232 bytes)."""

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


assert C.sizeof(Params) == 232

_lib = None

# name -> argtypes (restype int unless noted)
_P = C.POINTER(Params)
_vp, _sz, _u64, _u32 = C.c_void_p, C.c_size_t, C.c_uint64, C.c_uint32
_SIGS = {
    "sz3g_compress_bound": [_P, C.POINTER(_sz)],
    "sz3g_workspace_size": [_P, C.c_int, C.POINTER(_sz)],
    "sz3g_compress": [_P, _vp, _vp, _sz, C.POINTER(_sz), _vp, _sz, _vp],
    "sz3g_read_header": [_vp, _sz, C.c_int, _P, C.POINTER(_u64)],
    "sz3g_decompress": [_vp, _sz, _vp, _sz, _vp, _sz, _vp],
    "sz3g_compress_host": [_P, _vp, _vp, _sz, C.POINTER(_sz), _vp],
    "sz3g_decompress_host": [_vp, _sz, _vp, _sz, _vp],
    "sz3g_predict_quantize": [_P, _vp, _vp, _vp, _vp, C.POINTER(_u64), _vp, _vp, _sz, _vp],
    "sz3g_recover": [_P, _vp, _vp, _vp, _u64, _vp, _vp, _sz, _vp],
    "sz3g_huffman_build": [_vp, _u32, _vp, _vp, _vp],
    "sz3g_huffman_encode": [_vp, _u64, _vp, _vp, _u32, _u32, _vp, _u64, _vp, _vp, C.POINTER(_u64), _vp],
    "sz3g_huffman_decode": [_vp, _u64, _vp, _vp, _u32, _vp, _u32, _vp, _u64, _vp],
    "sz3g_huffman_decode_static": [_vp, _u64, _vp, _vp, _u32, _vp, _u32, _vp, _u64, _vp],
    "sz3g_batch_create": [C.c_int, C.c_int, _P, C.POINTER(_vp), C.POINTER(_sz), C.POINTER(_vp), C.POINTER(_sz),
                          C.POINTER(_vp)],
    "sz3g_batch_run": [_vp, _vp],
    "sz3g_batch_results": [_vp, C.POINTER(_u64), C.POINTER(C.c_int)],
    "sz3g_batch_configure": [_vp, C.c_int, C.c_int],
    "sz3g_batch_tune": [_vp, _vp, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "sz3g_batch_info": [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(_u64)],
    "sz3g_batch_set_queue": [_vp, C.c_int],
    "sz3g_batch_queue_info": [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "sz3g_batch_destroy": [_vp],
    "sz3g_graph_cache": [C.c_int],
    "sz3g_debug_inject": [C.c_int, C.c_longlong],
    "sz3g_trim": [],
    "sz3g_bitplane_bound": [_u64, C.POINTER(_u64)],
    "sz3g_bitplane_encode": [_u32, _vp, _u64, C.c_double, _vp, _sz, C.POINTER(_sz), _vp],
    "sz3g_bitplane_decode": [_vp, _sz, _vp, _sz, C.POINTER(_u64), _vp],
    "sz3g_huffman_fixed": [_u32, _vp, _vp, _vp],
    "sz3g_compress_async": [_P, _vp, _vp, _sz, _vp, _vp, _vp, _sz, _vp],
    "sz3g_decompress_async": [_vp, _vp, _sz, _vp, _sz, _vp, _vp, _sz, _vp],
    "sz3g_lossless_bound": [_u64, C.POINTER(_u64)],
    "sz3g_lossless_compress": [_vp, _u64, _vp, _sz, C.POINTER(_sz), _vp],
    "sz3g_lossless_decompress": [_vp, _sz, _vp, _sz, C.POINTER(_u64), _vp],
    "sz3g_select_costs": [_P, _vp, _u32, _u64, _vp, _vp],
    "sz3g_select_features": [_P, _vp, _u32, _u64, _vp, _vp],
    "sz3g_select_sampled": [_P, _vp, _u32, _u64, _vp, _vp],
    "sz3g_select_learned": [_P, _vp, _vp, _u32, _u64, _vp, _vp],
    "sz3g_mlp_forward": [_vp, _vp, _vp, _u32, _vp, _vp],
    "sz3g_mlp_gradient": [_vp, _vp, _vp, _vp, _u32, _vp, C.POINTER(C.c_float), _vp],
    "sz3g_mlp_train": [_vp, _vp, _vp, _vp, _u32, C.c_float, _u32, C.POINTER(C.c_float), _vp],
}
MLP_WEIGHTS = 1640
SEL_CANDIDATES = 8
SEL_FEATURES = 16


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None, reload: bool = False):
    """Load the built library (raises if it is missing).  reload: drop the
    library loaded so far and load `path` (the checking build, or back)."""
    global _lib
    if _lib is not None and not reload:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (paper_2111_02925_gb300.build)")
    L = C.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.sz3g_launch_count.argtypes = [C.POINTER(_u64)]
    L.sz3g_launch_count.restype = C.c_int
    L.sz3g_profile_enable.argtypes = [C.c_int]
    L.sz3g_profile_enable.restype = C.c_int
    L.sz3g_profile_read.argtypes = [C.c_char_p, C.POINTER(C.c_double), C.POINTER(_u64)]
    L.sz3g_profile_read.restype = C.c_int
    L.sz3g_profile_kernel_name.argtypes = [C.c_int]
    L.sz3g_profile_kernel_name.restype = C.c_char_p
    L.sz3g_strerror.argtypes = [C.c_int]
    L.sz3g_strerror.restype = C.c_char_p
    _lib = L
    return L


def strerror(code: int) -> str:
    return load().sz3g_strerror(code).decode()


def _chk(rc: int, where: str):
    if rc != OK:
        raise SZ3GError(rc, where)


def make_params(dims, eb, *, dtype=F32, eb_mode=ABS, interp=LINEAR, order=None, radius=32768, chunk=4096,
                level_interp=None, level_order=None) -> Params:
    p = Params()
    dims = [int(d) for d in dims]
    p.dtype, p.ndim = dtype, len(dims)
    for i in range(4):
        p.dims[i] = dims[i] if i < len(dims) else 1
    p.eb_mode, p.interp, p.eb = eb_mode, interp, float(eb)
    order = list(range(len(dims))) if order is None else list(order)
    for i in range(4):
        p.dim_order[i] = order[i] if i < len(order) else 0
    p.radius, p.chunk_codes = radius, chunk
    if level_interp is not None or level_order is not None:
        p.per_level = 1
        for l in range(1, MAX_LEVELS):
            li = (level_interp or {}).get(l, interp)
            lo = (level_order or {}).get(l, order)
            p.level_interp[l] = li
            for i in range(4):
                p.level_order[l][i] = lo[i] if i < len(lo) else 0
    return p


# ---- raw C entry points ----------------------------------------------------
def sz3g_compress_bound(p: Params) -> int:
    n = _sz()
    _chk(load().sz3g_compress_bound(C.byref(p), C.byref(n)), "sz3g_compress_bound")
    return n.value


def sz3g_workspace_size(p: Params, for_decompress: int) -> int:
    n = _sz()
    _chk(load().sz3g_workspace_size(C.byref(p), int(for_decompress), C.byref(n)), "sz3g_workspace_size")
    return n.value


def sz3g_compress(p: Params, d_in: int, d_out: int, out_capacity: int, d_ws: int = 0, ws_bytes: int = 0,
                  stream: int = 0):
    """Returns (status, out_bytes)."""
    nb = _sz(0)
    rc = load().sz3g_compress(C.byref(p), d_in, d_out, out_capacity, C.byref(nb), d_ws or None, ws_bytes,
                              stream or None)
    return rc, nb.value


def sz3g_read_header(stream_ptr: int, nbytes: int, on_device: int):
    p, n = Params(), _u64()
    rc = load().sz3g_read_header(stream_ptr, nbytes, on_device, C.byref(p), C.byref(n))
    return rc, p, n.value


def sz3g_decompress(d_stream: int, nbytes: int, d_out: int, out_capacity: int, d_ws: int = 0, ws_bytes: int = 0,
                    stream: int = 0) -> int:
    return load().sz3g_decompress(d_stream, nbytes, d_out, out_capacity, d_ws or None, ws_bytes, stream or None)


def sz3g_compress_host(p: Params, h_in: int, h_out: int, out_capacity: int, stream: int = 0):
    nb = _sz(0)
    rc = load().sz3g_compress_host(C.byref(p), h_in, h_out, out_capacity, C.byref(nb), stream or None)
    return rc, nb.value


def sz3g_compress_async(p: Params, d_in: int, d_out: int, out_capacity: int, d_out_bytes: int, d_status: int,
                        d_ws: int, ws_bytes: int, stream: int = 0) -> int:
    """Enqueue a compress; the stream length and status land in d_out_bytes (u64) and d_status (i32)."""
    return load().sz3g_compress_async(C.byref(p), d_in, d_out, out_capacity, d_out_bytes or None, d_status,
                                      d_ws or None, ws_bytes, stream or None)


def sz3g_decompress_async(h_header: int, d_stream: int, nbytes: int, d_out: int, out_capacity: int, d_status: int,
                          d_ws: int, ws_bytes: int, stream: int = 0) -> int:
    """Enqueue a decompress of a stream whose header bytes are at host address h_header."""
    return load().sz3g_decompress_async(h_header, d_stream, nbytes, d_out, out_capacity, d_status, d_ws or None,
                                        ws_bytes, stream or None)


def sz3g_decompress_host(h_stream: int, nbytes: int, h_out: int, out_capacity: int, stream: int = 0) -> int:
    return load().sz3g_decompress_host(h_stream, nbytes, h_out, out_capacity, stream or None)


def sz3g_predict_quantize(p: Params, d_in: int, d_codes: int, d_unpred: int, d_hist: int, d_ws: int = 0,
                          ws_bytes: int = 0, stream: int = 0):
    nu = _u64()
    eb = (C.c_uint8 * 8)()
    rc = load().sz3g_predict_quantize(C.byref(p), d_in, d_codes, d_unpred, d_hist, C.byref(nu), eb, d_ws or None,
                                      ws_bytes, stream or None)
    return rc, nu.value, bytes(eb)


def sz3g_recover(p: Params, ebT_bytes: bytes, d_codes: int, d_unpred: int, n_unpred: int, d_out: int,
                 d_ws: int = 0, ws_bytes: int = 0, stream: int = 0) -> int:
    eb = (C.c_uint8 * 8)(*ebT_bytes[:8].ljust(8, b"\0"))
    return load().sz3g_recover(C.byref(p), eb, d_codes, d_unpred or None, n_unpred, d_out, d_ws or None, ws_bytes,
                               stream or None)


def sz3g_huffman_build(d_hist: int, nsym: int, d_len: int, d_code: int, stream: int = 0) -> int:
    return load().sz3g_huffman_build(d_hist, nsym, d_len, d_code, stream or None)


def sz3g_huffman_encode(d_codes: int, n: int, d_len: int, d_code: int, nsym: int, chunk: int, d_words: int,
                        cap_words: int, d_chunk_words: int, d_sub_bits: int = 0, stream: int = 0):
    nw = _u64()
    rc = load().sz3g_huffman_encode(d_codes, n, d_len, d_code, nsym, chunk, d_words, cap_words, d_chunk_words,
                                    d_sub_bits or None, C.byref(nw), stream or None)
    return rc, nw.value


def sz3g_huffman_decode(d_words: int, n_words: int, d_chunk_words: int, d_sub_bits: int, chunk: int, d_len: int,
                        nsym: int, d_codes: int, n: int, stream: int = 0) -> int:
    return load().sz3g_huffman_decode(d_words, n_words, d_chunk_words, d_sub_bits or None, chunk, d_len, nsym,
                                      d_codes, n, stream or None)


def sz3g_huffman_decode_static(d_words: int, n_words: int, d_chunk_words: int, d_sub_bits: int, chunk: int,
                               d_len: int, nsym: int, d_codes: int, n: int, stream: int = 0) -> int:
    """sz3g_huffman_decode with its scratch in the library's fixed device array (allocates nothing)."""
    return load().sz3g_huffman_decode_static(d_words, n_words, d_chunk_words, d_sub_bits or None, chunk, d_len, nsym,
                                             d_codes, n, stream or None)


class Batch:
    """sz3g_batch_* over device pointers: many fields (or streams) per call.

    compress:   Batch(params_list, in_ptrs, out_ptrs, out_caps)
    decompress: Batch(None, stream_ptrs, out_ptrs, out_caps, in_bytes=stream_lengths, decompress=True)
    """

    def __init__(self, params, d_in, d_out, out_capacity, in_bytes=None, decompress=False):
        n = len(d_in)
        L = load()
        pa = (Params * n)(*params) if params is not None else None
        ins = (_vp * n)(*[int(v) for v in d_in])
        outs = (_vp * n)(*[int(v) for v in d_out])
        caps = (_sz * n)(*[int(v) for v in out_capacity])
        ib = (_sz * n)(*[int(v) for v in in_bytes]) if in_bytes is not None else None
        h = _vp()
        _chk(L.sz3g_batch_create(n, int(decompress), pa, ins, ib, outs, caps, C.byref(h)), "sz3g_batch_create")
        self.n, self.h = n, h

    def run(self, stream: int = 0) -> None:
        _chk(load().sz3g_batch_run(self.h, _vp(stream)), "sz3g_batch_run")

    def results(self):
        """(rc, stream lengths, per-field statuses) of the last run (synchronises)."""
        b = (_u64 * self.n)()
        st = (C.c_int * self.n)()
        rc = load().sz3g_batch_results(self.h, b, st)
        return rc, list(b), list(st)

    def configure(self, branches: int, cta_cap: int = 0) -> None:
        _chk(load().sz3g_batch_configure(self.h, branches, cta_cap), "sz3g_batch_configure")

    def set_queue(self, on: bool) -> None:
        """Level-queue mode: the grid levels of all fields in one persistent
        launch per type from a cross-field work queue."""
        _chk(load().sz3g_batch_set_queue(self.h, int(on)), "sz3g_batch_set_queue")

    def queue_info(self):
        """(level-queue mode on, grid levels in the queue)."""
        on, lv = C.c_int(), C.c_int()
        _chk(load().sz3g_batch_queue_info(self.h, C.byref(on), C.byref(lv)), "sz3g_batch_queue_info")
        return bool(on.value), lv.value

    def tune(self, stream: int = 0):
        br, cap = C.c_int(), C.c_int()
        _chk(load().sz3g_batch_tune(self.h, _vp(stream), C.byref(br), C.byref(cap)), "sz3g_batch_tune")
        return br.value, cap.value

    def info(self):
        br, cap, nodes = C.c_int(), C.c_int(), _u64()
        _chk(load().sz3g_batch_info(self.h, C.byref(br), C.byref(cap), C.byref(nodes)), "sz3g_batch_info")
        return br.value, cap.value, nodes.value

    def close(self) -> None:
        if self.h:
            load().sz3g_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _levels(p: Params) -> int:
    m = max(p.dims[i] for i in range(p.ndim))
    L = 0
    while (1 << L) < m:
        L += 1
    return L


def sz3g_select_costs(p: Params, d_x: int, nblocks: int = 0, seed: int = 0, stream: int = 0):
    """(L x 8) estimated bits per level and candidate."""
    import numpy as np

    L = _levels(p)
    out = np.zeros((max(L, 1), SEL_CANDIDATES), np.float64)
    _chk(load().sz3g_select_costs(C.byref(p), d_x, nblocks, seed, out.ctypes.data, stream), "sz3g_select_costs")
    return out[:L]


def sz3g_select_features(p: Params, d_x: int, nblocks: int = 0, seed: int = 0, stream: int = 0):
    import numpy as np

    L = _levels(p)
    out = np.zeros((max(L, 1), SEL_FEATURES), np.float64)
    _chk(load().sz3g_select_features(C.byref(p), d_x, nblocks, seed, out.ctypes.data, stream),
         "sz3g_select_features")
    return out[:L]


def sz3g_select_sampled(p: Params, d_x: int, nblocks: int, seed: int = 0, stream: int = 0):
    """{level: candidate} of least estimated bits."""
    L = _levels(p)
    ch = (C.c_uint8 * (L + 1))()
    _chk(load().sz3g_select_sampled(C.byref(p), d_x, nblocks, seed, ch, stream), "sz3g_select_sampled")
    return {l: int(ch[l]) for l in range(1, L + 1)}


def sz3g_select_learned(p: Params, d_x: int, d_w: int, nblocks: int, seed: int = 0, stream: int = 0):
    L = _levels(p)
    ch = (C.c_uint8 * (L + 1))()
    _chk(load().sz3g_select_learned(C.byref(p), d_x, d_w, nblocks, seed, ch, stream), "sz3g_select_learned")
    return {l: int(ch[l]) for l in range(1, L + 1)}


def sz3g_mlp_forward(d_w: int, d_feat: int, d_mask: int, n: int, d_logits: int, stream: int = 0) -> None:
    _chk(load().sz3g_mlp_forward(d_w, d_feat, d_mask, n, d_logits, stream), "sz3g_mlp_forward")


def sz3g_mlp_gradient(d_w: int, d_feat: int, d_mask: int, d_label: int, n: int, d_grad: int, stream: int = 0):
    loss = C.c_float()
    _chk(load().sz3g_mlp_gradient(d_w, d_feat, d_mask, d_label, n, d_grad, C.byref(loss), stream),
         "sz3g_mlp_gradient")
    return loss.value


def sz3g_mlp_train(d_w: int, d_feat: int, d_mask: int, d_label: int, n: int, lr: float, steps: int,
                   stream: int = 0) -> float:
    loss = C.c_float()
    _chk(load().sz3g_mlp_train(d_w, d_feat, d_mask, d_label, n, lr, steps, C.byref(loss), stream),
         "sz3g_mlp_train")
    return loss.value


_ORDERS = {3: [(0, 1, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)], 2: [(0, 1), (1, 0), (0, 1), (1, 0)], 1: [(0,)] * 4}


def params_for_choices(p: Params, choices) -> Params:
    """Copy of p with per-level interpolation / axis order from {level: candidate}."""
    nd = p.ndim
    li = {l: c % 2 for l, c in choices.items()}
    lo = {l: list(_ORDERS[nd][c // 2]) for l, c in choices.items()}
    return make_params([p.dims[i] for i in range(nd)], p.eb, dtype=p.dtype, eb_mode=p.eb_mode, interp=p.interp,
                       order=[p.dim_order[i] for i in range(nd)], radius=p.radius, chunk=p.chunk_codes,
                       level_interp=li, level_order=lo)


def sz3g_launch_count() -> int:
    n = _u64()
    _chk(load().sz3g_launch_count(C.byref(n)), "sz3g_launch_count")
    return n.value


def sz3g_profile_enable(on: bool) -> None:
    _chk(load().sz3g_profile_enable(int(on)), "sz3g_profile_enable")


def sz3g_profile_read(kernel: str):
    t, n = C.c_double(), _u64()
    _chk(load().sz3g_profile_read(kernel.encode(), C.byref(t), C.byref(n)), "sz3g_profile_read")
    return t.value, n.value


def sz3g_profile_kernel_names():
    out, i = [], 0
    while True:
        nm = load().sz3g_profile_kernel_name(i)
        if nm is None:
            return out
        out.append(nm.decode())
        i += 1


# ---- torch-tensor helpers ----------------------------------------------------
def _torch():
    import torch

    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def params_for(x, eb, **kw) -> Params:
    torch = _torch()
    dtype = F32 if x.dtype == torch.float32 else F64
    return make_params(tuple(x.shape), eb, dtype=dtype, **kw)


def compress(x, p: Params, workspace=None, out=None, stream=None):
    """Compress a contiguous CUDA tensor; returns a uint8 CUDA tensor (a view of `out`)."""
    torch = _torch()
    assert x.is_cuda and x.is_contiguous()
    cap = sz3g_compress_bound(p)
    if out is None:
        out = torch.empty(cap, dtype=torch.uint8, device=x.device)
    ws, wsb = (workspace.data_ptr(), workspace.numel() * workspace.element_size()) if workspace is not None else (0, 0)
    rc, nb = sz3g_compress(p, x.data_ptr(), out.data_ptr(), out.numel(), ws, wsb, _stream_handle(stream))
    _chk(rc, "sz3g_compress")
    return out[:nb]


def decompress(stream_bytes, out=None, workspace=None, stream=None):
    """Decompress a uint8 CUDA tensor holding a stream; returns a flat tensor."""
    torch = _torch()
    assert stream_bytes.is_cuda and stream_bytes.dtype == torch.uint8
    head = stream_bytes[:HEADER_BYTES].cpu().numpy().tobytes()
    buf = C.create_string_buffer(head, len(head))
    rc, p, n = sz3g_read_header(C.addressof(buf), stream_bytes.numel(), 0)
    _chk(rc, "sz3g_read_header")
    dt = torch.float32 if p.dtype == F32 else torch.float64
    if out is None:
        out = torch.empty(n, dtype=dt, device=stream_bytes.device)
    ws, wsb = (workspace.data_ptr(), workspace.numel() * workspace.element_size()) if workspace is not None else (0, 0)
    rc = sz3g_decompress(stream_bytes.data_ptr(), stream_bytes.numel(), out.data_ptr(),
                         out.numel() * out.element_size(), ws, wsb, _stream_handle(stream))
    _chk(rc, "sz3g_decompress")
    return out


def workspace(p: Params, for_decompress: bool, device="cuda"):
    torch = _torch()
    n = sz3g_workspace_size(p, int(for_decompress))
    return torch.empty(n, dtype=torch.uint8, device=device)


DEBUG_RESET, DEBUG_WAIT_LIMIT, DEBUG_QUEUE_STALL, DEBUG_SILENT_CHUNK, DEBUG_ALLOC_FAIL = 0, 1, 2, 3, 4


def sz3g_debug_inject(kind: int, value: int = 0) -> int:
    """Failure injection for tests (see include/sz3g.h); returns the status."""
    return int(load().sz3g_debug_inject(kind, value))


def sz3g_graph_cache(on: bool) -> None:
    """Turn the compress / decompress graph cache on or off (on by default)."""
    _chk(load().sz3g_graph_cache(int(on)), "sz3g_graph_cache")


def sz3g_trim() -> None:
    """Free the cached graphs, the host-buffer staging sets and the pool's free memory."""
    _chk(load().sz3g_trim(), "sz3g_trim")


BP_HEADER = 32


def sz3g_bitplane_bound(n: int) -> int:
    b = _u64(0)
    _chk(load().sz3g_bitplane_bound(n, C.byref(b)), "sz3g_bitplane_bound")
    return b.value


def sz3g_bitplane_encode(dtype: int, d_values: int, n: int, eb: float, d_out: int, out_capacity: int,
                         stream: int = 0):
    """Unpred-aware quantizer (bitplanes); returns (status, stream bytes)."""
    nb = _sz(0)
    rc = load().sz3g_bitplane_encode(dtype, d_values or None, n, eb, d_out, out_capacity, C.byref(nb),
                                     stream or None)
    return rc, nb.value


def sz3g_bitplane_decode(d_stream: int, nbytes: int, d_out: int, out_capacity: int, stream: int = 0):
    """Returns (status, n values)."""
    n = _u64(0)
    rc = load().sz3g_bitplane_decode(d_stream, nbytes, d_out or None, out_capacity, C.byref(n), stream or None)
    return rc, n.value


def sz3g_huffman_fixed(radius: int, d_len: int, d_code: int, stream: int = 0) -> int:
    """Predefined Huffman lengths / canonical codewords over the 2 radius codes."""
    return load().sz3g_huffman_fixed(radius, d_len, d_code, stream or None)


def sz3g_lossless_bound(n: int) -> int:
    b = _u64(0)
    _chk(load().sz3g_lossless_bound(n, C.byref(b)), "sz3g_lossless_bound")
    return b.value


def sz3g_lossless_compress(d_in: int, n: int, d_out: int, out_capacity: int, stream: int = 0):
    """The lossless stage over n device bytes; returns (status, stream bytes)."""
    nb = _sz(0)
    rc = load().sz3g_lossless_compress(d_in or None, n, d_out, out_capacity, C.byref(nb), stream or None)
    return rc, nb.value


def sz3g_lossless_decompress(d_stream: int, nbytes: int, d_out: int, out_capacity: int, stream: int = 0):
    """Returns (status, decoded bytes)."""
    n = _u64(0)
    rc = load().sz3g_lossless_decompress(d_stream, nbytes, d_out, out_capacity, C.byref(n), stream or None)
    return rc, n.value
