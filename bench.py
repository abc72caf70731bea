#!/usr/bin/env python
"""Throughput of the SZ3-Interp hot path (multilevel interpolation + linear-
scaling quantizer + histogram + chunked Huffman) on GB300.

Workload: one 512^3 FP32 Gaussian random field with power spectrum ~ k^-3
(unit variance, seed 2; a synthetic stand-in for NYX 512^3), REL error bound
1e-3 (the bound of the paper's throughput figure), cubic interpolation, axis
order (0,1,2), radius 32768, 4096-code Huffman chunks.  One step = compress
the field and decompress the stream, i.e. every step of the hot path once.
The 512 MiB input is larger than L2 (129 MB), so no flush is needed between
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sz3g|reference]
  python bench.py --workload batch   # the uneven 256-field batch, batched vs one call per field
  python bench.py --workload selector  # per-level selection on a 1024^3 field with fronts
  python bench.py --workload lossless  # the optional lossless stage on two workloads' streams
  python bench.py --workload pastri    # unpred-aware quantizer (bitplanes) and the fixed Huffman table

--impl reference times the serial CPU oracle on the host cores, on a bounded
sample (a 128^3 corner of the same field) per step.  N > 1 (torchrun) runs
independent replicas, one per GPU: a single field does not shard without
changing its result, so there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress/decompress GB/s (input bytes) on 1 GB300 and % of HBM roofline, at stated eb"
SIZE = 512
EB = 1e-3
SEED = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sz3g", choices=["sz3g", "reference"])
    ap.add_argument("--size", type=int, default=SIZE)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the REL 1e-2 / 1e-4 timings of the field")
    ap.add_argument("--workload", default="field", choices=["field", "batch", "selector", "lossless", "pastri"])
    ap.add_argument("--train-fields", type=int, default=2000)
    ap.add_argument("--train-size", type=int, default=128,
                    help="points per axis of the selector workload's training fields (0: 32..64 at random)")
    ap.add_argument("--fields", type=int, default=256)
    ap.add_argument("--no-extras", action="store_true", help="skip the batch / selector / lossless figures")
    ap.add_argument("--extra-train-fields", type=int, default=160)
    return ap.parse_args()


def workload_config(n):
    return {
        "workload": f"{n}^3 FP32 k^-3 Gaussian random field (seed {SEED}), REL eb {EB:g}, cubic, order (0,1,2), "
                    "radius 32768, 4096-code chunks; step = compress + decompress",
        "dims": [n, n, n],
        "dtype": "f32",
        "eb_mode": "REL",
        "eb": EB,
        "interp": "cubic",
        "radius": 32768,
        "chunk_codes": 4096,
        "l2": "inputs larger than L2 (512 MiB field vs 129 MB L2), no flush",
    }


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_units(n: int, ws: int, rank: int):
    """Global indices of the units rank `rank` of `ws` processes when every
    rank takes n units of its own (weak scaling): a contiguous block."""
    return list(range(rank * n, (rank + 1) * n))


def reduce_over_ranks(values, op: str = "max", device=None):
    """Element-wise max or sum of a list of floats over the process group
    (the values themselves without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(kernel: str, info: dict) -> float:
    """A kernel's share of the algorithmic bytes of its direction: compress
    (REL) must read the field twice (range, then the values) and write the
    stream; decompress must read the stream and write the field.  The shares
    partition those totals: range and the quantize levels one field read
    each, the encoder the stream it writes; the decoder the stream it reads,
    the recover levels the field they write.  Kernels with no share (the
    codebook, the coarse grids' helpers) move only implementation bytes."""
    N, esz = info["N"], info["esz"]
    stream = info["stream_bytes"]
    return {
        "range": N * esz,
        "level_quantize": N * esz,
        "encode": stream,
        "decode": stream,
        "level_recover": N * esz,
    }.get(kernel, 0.0)


def implementation_bytes(kernel: str, info: dict) -> float:
    """Bytes a kernel moves beyond its algorithmic share, counted once each:
    the 2-byte code of every point (written by the quantize levels, read by
    the encoder; written by the decoder, read by the recover levels) and the
    reconstruction of the coarser grids (written once, read once by the
    level above)."""
    N, esz = info["N"], info["esz"]
    coarse = info["coarse_points"]
    return {
        "level_quantize": 2 * N + 2 * coarse * esz,
        "encode": 2 * N,
        "decode": 2 * N,
        "level_recover": 2 * N + 2 * coarse * esz,
    }.get(kernel, 0.0)


def host_cpu():
    """The host CPU's model name and logical core count."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count()}


def traffic_for(kernel: str):
    """ncu DRAM bytes (read + write) of one step's launches of `kernel`,
    recorded in profiles/traffic.json for the current kernel sources, else
    None (the kernels changed since the counters were taken)."""
    try:
        from paper_2111_02925_gb300 import build as B

        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)
        e = d.get(kernel)
        if e and kernel in B.KERNEL_SOURCES and e.get("source_stamp") == B.kernel_stamp(kernel):
            return e.get("bytes_per_step")
    except Exception:
        pass
    return None


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle as O
    from paper_2111_02925_gb300 import synthetic as S

    O.build()
    x = S.grf((args.size,) * 3, SEED)
    m = min(256, args.size)
    sample = np.ascontiguousarray(x[:m, :m, :m])
    p = O.make_params(sample.shape, EB, eb_mode=O.REL, interp=O.CUBIC)
    for _ in range(args.warmup):
        O.decompress(O.compress(p, sample))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = O.compress(p, sample)
        O.decompress(s)
    dt = (time.perf_counter() - t0) / args.steps
    gbs = sample.nbytes / dt / 1e9
    cfg = workload_config(args.size)
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{m}^3 corner of the {args.size}^3 field ({sample.nbytes} bytes), compress + "
                                   "decompress per step, one thread", **host_cpu()},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(x):
    import numpy as np

    import oracle as O

    O.build()
    m = min(256, x.shape[0])
    sample = np.ascontiguousarray(x[:m, :m, :m])
    p = O.make_params(sample.shape, EB, eb_mode=O.REL, interp=O.CUBIC)
    t0 = time.perf_counter()
    reps = 0
    while True:
        O.decompress(O.compress(p, sample))
        reps += 1
        if time.perf_counter() - t0 > 8.0 or reps >= 3:
            break
    dt = (time.perf_counter() - t0) / reps
    return {"value": sample.nbytes / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{m}^3 corner of the field, compress + decompress, {reps} run(s), one thread", **host_cpu()}


def grf_gpu(shape, seed, dev):
    """k^-3 Gaussian random field generated on the GPU (seeded white noise
    shaped by |k|^-3/2, unit variance); the batch inputs."""
    import torch

    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    w = torch.randn(shape, generator=g, device=dev, dtype=torch.float32)
    f = torch.fft.rfftn(w)
    ks = [torch.fft.fftfreq(n, device=dev) for n in shape[:-1]] + [torch.fft.rfftfreq(shape[-1], device=dev)]
    k2 = sum(torch.meshgrid(*[k * k for k in ks], indexing="ij"))
    k2[(0,) * len(shape)] = 1.0
    f = f * k2.pow(-0.75)
    f[(0,) * len(shape)] = 0
    x = torch.fft.irfftn(f, s=shape)
    x = (x - x.mean()) / x.std()
    return x.contiguous()


def run_batch(args):
    """The uneven batch: `--fields` FP32 fields, each axis log-uniform in
    [32, 256], k^-3 random fields, REL bounds log-uniform in [1e-5, 1e-2],
    linear / cubic at random.  One step = compress every field, then
    decompress every stream.  Timed (a) batched: one graph launch per
    direction, branches and CTA cap picked by the autotuner; (b) one
    sz3g_compress / sz3g_decompress call per field on one stream."""
    import torch

    from paper_2111_02925_gb300 import build as B
    from paper_2111_02925_gb300 import synthetic as S
    from paper_2111_02925_gb300 import sz3g as G

    ws, rank, local = dist_env()
    torch.cuda.set_device(local if ws > 1 else 0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    B.build()
    G.load()
    # every rank its own `fields` fields (weak scaling); field g of the whole
    # job has the g-th shape of the mix and seed 4000 + g
    own = shard_units(args.fields, ws, rank)
    full = S.batch_shapes(args.fields * ws, 4)
    mix = [full[g] for g in own]
    xs = [grf_gpu(d, 4000 + g, dev).reshape(-1) for g, (d, _, _) in zip(own, mix)]
    params = [G.make_params(d, eb, eb_mode=G.REL, interp=it) for d, eb, it in mix]
    caps = [G.sz3g_compress_bound(p) for p in params]
    streams = [torch.empty(c, dtype=torch.uint8, device=dev) for c in caps]
    outs = [torch.empty_like(x) for x in xs]
    in_bytes = sum(x.numel() * 4 for x in xs)
    sh = int(torch.cuda.current_stream().cuda_stream)
    # (b) one call per field (workspace allocated once per field, outside the timing)
    wsc = [G.workspace(p, False, dev) for p in params]
    wsd = [G.workspace(p, True, dev) for p in params]

    def per_field():
        nbs = []
        for p, x, s, w in zip(params, xs, streams, wsc):
            rc, nb = G.sz3g_compress(p, x.data_ptr(), s.data_ptr(), s.numel(), w.data_ptr(), w.numel(), sh)
            assert rc == 0
            nbs.append(nb)
        for s, nb, o, w in zip(streams, nbs, outs, wsd):
            rc = G.sz3g_decompress(s.data_ptr(), nb, o.data_ptr(), o.numel() * 4, w.data_ptr(), w.numel(), sh)
            assert rc == 0
        return nbs

    nbs = per_field()
    # (a) batched
    bc = G.Batch(params, [x.data_ptr() for x in xs], [s.data_ptr() for s in streams], caps)
    bd = G.Batch(None, [s.data_ptr() for s in streams], [o.data_ptr() for o in outs], [o.numel() * 4 for o in outs],
                 in_bytes=nbs, decompress=True)
    tc = bc.tune(sh)
    td = bd.tune(sh)

    def batched():
        bc.run(sh)
        bd.run(sh)

    def timeit(fn, k):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    k = max(1, min(args.steps, 20))
    t_batch = timeit(batched, k)
    rc, nb2, st = bc.results()
    assert rc == 0 and list(nb2) == list(nbs)
    rc, _, st = bd.results()
    assert rc == 0
    qc, qd = bc.queue_info()[0], bd.queue_info()[0]
    tuned = {"compress": {"branches": tc[0], "cta_cap": tc[1], "level_queue": qc, "graph_nodes": bc.info()[2],
                          "ms": timeit(lambda: bc.run(sh), 3)},
             "decompress": {"branches": td[0], "cta_cap": td[1], "level_queue": qd, "graph_nodes": bd.info()[2],
                            "ms": timeit(lambda: bd.run(sh), 3)}}
    # the cross-field level queue at its best branch count, each direction (after the tuned run)
    queue = {}
    for b, lab in ((bc, "compress"), (bd, "decompress")):
        br0, cap0 = b.info()[:2]
        on0 = b.queue_info()[0]
        b.set_queue(True)
        best = None
        for br in (16, 64, 128):
            b.configure(min(br, len(xs)), 0)
            t = timeit(lambda: b.run(sh), 3)
            if best is None or t < best[0]:
                best = (t, br)
        queue[lab] = {"ms": best[0], "branches": best[1], "levels": b.queue_info()[1]}
        b.set_queue(on0)
        b.configure(br0, cap0)
    t_single = timeit(per_field, max(1, min(k, 3)))
    t_batch, t_single = reduce_over_ranks([t_batch, t_single], "max", dev)
    in_bytes, stream_total = reduce_over_ranks([in_bytes, sum(nbs)], "sum", dev)
    if rank != 0:
        bc.close()
        bd.close()
        dist.destroy_process_group()
        return 0
    line = {
        "metric": "batch compress+decompress GB/s (input bytes), uneven fields, 1 GB300",
        "value": in_bytes / (t_batch * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": ws, "steps": k,
        "warmup": max(args.warmup, 3), "ms_per_step": t_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.fields} FP32 3-D k^-3 random fields, axes log-uniform in [32, 256], "
                               "REL eb log-uniform in [1e-5, 1e-2], linear/cubic at random (seed 4); "
                               "step = compress all + decompress all",
                   "fields": args.fields * ws, "fields_per_gpu": args.fields, "input_bytes": int(in_bytes),
                   "stream_bytes": int(stream_total)},
        "per_field_calls": {"ms_per_step": t_single, "GB/s": in_bytes / (t_single * 1e-3) / 1e9},
        "speedup_vs_per_field_calls": t_single / t_batch,
        "tuned": tuned,
        "level_queue_ms": queue,
    }
    print(json.dumps(line), flush=True)
    bc.close()
    bd.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def _label_field(job):
    """Oracle labels (exhaustive trial) and input features (8 sampled blocks
    per level) of one training field, per level; runs in a spawned worker.
    The GPU's features equal the oracle's to 1e-10 (tests/test_gpu_select.py),
    so the network trained on these is applied to the GPU's."""
    import numpy as np

    import oracle as O
    from paper_2111_02925_gb300 import synthetic as S

    shape, seed, fronts, eb = job
    x = S.grf_fronts(shape, seed, fronts)
    op = O.make_params(shape, eb, eb_mode=O.REL)
    _, L = O.shape(op)
    labels = [int(np.argmin(O.select_costs(op, x, l))) for l in range(1, L + 1)]
    feats = [O.select_features(op, x, l, 8, seed).tolist() for l in range(1, L + 1)]
    return labels, feats


def fronts_gpu(shape, seed, n_fronts, dev):
    """k^-3 random field plus n_fronts tanh fronts (as synthetic.grf_fronts,
    generated on the GPU for fields too large for the host FFT)."""
    import numpy as np
    import torch

    x = grf_gpu(shape, seed, dev)
    rng = np.random.default_rng(seed + 7919)
    coords = [torch.arange(n, device=dev, dtype=torch.float32) for n in shape]
    for _ in range(n_fronts):
        nv = rng.normal(size=3)
        nv /= np.linalg.norm(nv)
        corners = np.array(np.meshgrid(*[[0, n - 1] for n in shape], indexing="ij")).reshape(3, -1)
        proj = nv @ corners
        c = rng.uniform(proj.min(), proj.max())
        w = rng.uniform(1.0, 8.0)
        a = rng.uniform(0.5, 2.0)
        t = (nv[0] * coords[0])[:, None, None] + (nv[1] * coords[1])[None, :, None] + (nv[2] * coords[2])[None, None, :]
        x += a * torch.tanh((t - c) / w)
    return x.contiguous()


def run_selector(args):
    """Per-level selection of interpolation and axis order on one 1024^3 FP32
    field (k^-3 random field + 16 tanh fronts, REL 1e-4).  The network is
    trained on the GPU (own kernels) on small fields labelled by the oracle's
    exhaustive trial; reported: stream size / compression ratio under a fixed
    choice, the exhaustive, sampling and learned selections, and the time of
    each selection."""
    import numpy as np

    jobs, labels, tfeats = label_jobs(args.train_fields, args.train_size)  # before any GPU call
    import torch

    from oracle import mlp as M
    from paper_2111_02925_gb300 import build as B
    from paper_2111_02925_gb300 import synthetic as S
    from paper_2111_02925_gb300 import sz3g as G

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    B.build()
    G.load()
    sh = int(torch.cuda.current_stream().cuda_stream)
    feats, ys = [], []
    for f, lab in zip(tfeats, labels):
        feats.extend(f)
        ys.extend(lab)
    feats = np.array(feats)
    ys = np.array(ys, np.int32)
    w = torch.from_numpy(M.init(feats, 5).astype(np.float32)).to(dev)
    fd = torch.from_numpy(feats.astype(np.float32).reshape(-1)).to(dev)
    yd = torch.from_numpy(ys).to(dev)
    md = torch.ones(len(ys) * 8, dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    loss = G.sz3g_mlp_train(w.data_ptr(), fd.data_ptr(), md.data_ptr(), yd.data_ptr(), len(ys), 0.3, 3000, sh)
    train_s = time.perf_counter() - t0
    n = 1024
    x = fronts_gpu((n, n, n), 5, 16, dev).reshape(-1)
    p = G.make_params((n, n, n), 1e-4, eb_mode=G.REL, interp=G.LINEAR)
    cap = G.sz3g_compress_bound(p)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    wsc = G.workspace(p, False, dev)

    def size(q):
        rc, nb = G.sz3g_compress(q, x.data_ptr(), out.data_ptr(), cap, wsc.data_ptr(), wsc.numel(), sh)
        assert rc == 0
        return nb

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, (time.perf_counter() - t) * 1e3

    def kernel_ms(fn):
        """Time of the selection's own kernels (not the range pass it shares
        with the compressor), from the library's CUDA-event profile."""
        G.sz3g_profile_enable(True)
        fn()
        torch.cuda.synchronize()
        t = G.sz3g_profile_read("select")[0] + G.sz3g_profile_read("mlp")[0]
        G.sz3g_profile_enable(False)
        return t

    sel_s = lambda: G.sz3g_select_sampled(p, x.data_ptr(), 64, 1, sh)  # noqa: E731
    sel_l = lambda: G.sz3g_select_learned(p, x.data_ptr(), w.data_ptr(), 16, 1, sh)  # noqa: E731
    sel_e = lambda: G.sz3g_select_sampled(p, x.data_ptr(), 0, 1, sh)  # noqa: E731
    ch_s, ms_s = timed(sel_s)
    ch_l, ms_l = timed(sel_l)
    ch_e, ms_e = timed(sel_e)
    ks_s, ks_l, ks_e = kernel_ms(sel_s), kernel_ms(sel_l), kernel_ms(sel_e)
    raw = x.numel() * 4
    res = {
        "fixed_linear_012": size(p),
        "fixed_cubic_012": size(G.make_params((n, n, n), 1e-4, eb_mode=G.REL, interp=G.CUBIC)),
        "exhaustive": size(G.params_for_choices(p, ch_e)),
        "sampled": size(G.params_for_choices(p, ch_s)),
        "learned": size(G.params_for_choices(p, ch_l)),
    }
    line = {
        "metric": "compression ratio with the learned per-level selector (1024^3 FP32, REL 1e-4)",
        "value": raw / res["learned"], "unit": "ratio", "n_gpus": 1, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "1024^3 FP32 k^-3 random field + 16 tanh fronts (seed 5), REL eb 1e-4; network "
                               f"trained on {args.train_fields} oracle-labelled fields of "
                               + (f"{args.train_size}^3 points" if args.train_size > 0 else "32..64 points per axis"),
                   "sample_blocks": {"sampled": 64, "learned_features": 16}},
        "ratio": {k: raw / v for k, v in res.items()},
        "learned_vs_sampled": res["sampled"] / res["learned"],
        "selection_ms": {"sampled": ms_s, "learned": ms_l, "exhaustive": ms_e,
                         "note": "wall time of the call, including one pass over the field for its value range"},
        "selection_kernel_ms": {"sampled": ks_s, "learned": ks_l, "exhaustive": ks_e},
        "choices": {"sampled": ch_s, "learned": ch_l, "exhaustive": ch_e},
        "training": {"examples": int(len(ys)), "steps": 3000, "final_loss": loss, "seconds": train_s},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_lossless(args):
    """The optional lossless stage after the Huffman coder on the streams of
    two workloads: the 512^3 k^-3 field (REL 1e-3, cubic) and the 1800 x 3600
    FP64 lat-lon field with 30% exact zeros (ABS 1e-6 of the range, cubic).
    Reports stream GB/s of the stage each way and the extra ratio."""
    import numpy as np
    import torch

    from paper_2111_02925_gb300 import build as B
    from paper_2111_02925_gb300 import synthetic as S
    from paper_2111_02925_gb300 import sz3g as G

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    B.build()
    G.load()
    sh = int(torch.cuda.current_stream().cuda_stream)
    res = {}
    for name, x, p in (
        ("grf512_rel1e-3", S.grf((args.size,) * 3, SEED), None),
        ("latlon1800x3600_f64_abs1e-6", S.latlon(1800, 3600, seed=3), None),
    ):
        if p is None:
            if x.dtype == np.float64:
                p = G.make_params(x.shape, 1e-6 * (float(x.max()) - float(x.min())), dtype=G.F64, eb_mode=G.ABS,
                                  interp=G.CUBIC)
            else:
                p = G.make_params(x.shape, EB, eb_mode=G.REL, interp=G.CUBIC)
        xd = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(dev)
        cap = G.sz3g_compress_bound(p)
        st = torch.empty(cap, dtype=torch.uint8, device=dev)
        rc, nb = G.sz3g_compress(p, xd.data_ptr(), st.data_ptr(), cap, stream=sh)
        assert rc == 0
        lcap = G.sz3g_lossless_bound(nb)
        lz = torch.empty(lcap, dtype=torch.uint8, device=dev)
        back = torch.empty(nb + 16, dtype=torch.uint8, device=dev)

        def comp():
            rc, m = G.sz3g_lossless_compress(st.data_ptr(), nb, lz.data_ptr(), lcap, sh)
            assert rc == 0
            return m

        def dec(m):
            rc, n2 = G.sz3g_lossless_decompress(lz.data_ptr(), m, back.data_ptr(), nb, sh)
            assert rc == 0 and n2 == nb

        m = comp()
        dec(m)
        assert bool(torch.equal(back[:nb], st[:nb]))
        k = max(3, min(args.steps, 20))
        tc, td = [], []
        for _ in range(k):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            comp()
            e[1].record()
            dec(m)
            e[2].record()
            torch.cuda.synchronize()
            tc.append(e[0].elapsed_time(e[1]))
            td.append(e[1].elapsed_time(e[2]))
        res[name] = {"input_bytes": int(x.nbytes), "stream_bytes": int(nb), "lossless_bytes": int(m),
                     "ratio_before": x.nbytes / nb, "ratio_after": x.nbytes / m, "gain": nb / m,
                     "compress_ms": statistics.median(tc), "decompress_ms": statistics.median(td),
                     "compress_GB/s": nb / (statistics.median(tc) * 1e-3) / 1e9,
                     "decompress_GB/s": nb / (statistics.median(td) * 1e-3) / 1e9}
    line = {"metric": "lossless stage GB/s (stream bytes) and ratio gain, 1 GB300", "unit": "GB/s",
            "value": res["grf512_rel1e-3"]["compress_GB/s"], "n_gpus": 1, "higher_is_better": True,
            "dtype": "u8", "data": "synthetic", "config": {"workload": "streams of sz3g_compress", "fields": res}}
    print(json.dumps(line), flush=True)
    return 0


def _median_ms(fn, k):
    """Median of k CUDA-event timings of fn() on the current stream."""
    import torch

    ts = []
    for _ in range(k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def run_pastri(args):
    """The SZ3-Pastri modules.  (1) The unpred-aware quantizer on 2^26 FP32
    prediction differences of unpredictable points (Laplace, scale 200 eb,
    5% of them 100x wider; eb 1e-3): encode / decode GB/s of input bytes and
    the dominant kernel's roofline, and the lossless stage's size on the
    bitplane stream against the same integers stored one int32 per value.
    (2) The fixed Huffman table against the built codebook on the codes of
    the 512^3 field (REL 1e-3, cubic): table time, encode GB/s, payload."""
    import numpy as np
    import torch

    from paper_2111_02925_gb300 import build as B
    from paper_2111_02925_gb300 import synthetic as S
    from paper_2111_02925_gb300 import sz3g as G

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    B.build()
    G.load()
    sh = int(torch.cuda.current_stream().cuda_stream)
    peak, peak_kind = peaks()
    k = max(3, min(args.steps, 20))
    # (1) unpred-aware quantizer
    rng = np.random.default_rng(SEED)
    n, eb = 1 << 26, 1e-3
    v = rng.laplace(0.0, 200 * eb, n)
    wide = rng.random(n) < 0.05
    v[wide] *= 100.0
    vd = torch.from_numpy(v.astype(np.float32)).to(dev)
    cap = G.sz3g_bitplane_bound(n)
    bp = torch.empty(cap, dtype=torch.uint8, device=dev)
    back = torch.empty(n, dtype=torch.float32, device=dev)
    nb = [0]

    def enc():
        rc, nb[0] = G.sz3g_bitplane_encode(G.F32, vd.data_ptr(), n, eb, bp.data_ptr(), cap, sh)
        assert rc == 0

    def dec():
        rc, m = G.sz3g_bitplane_decode(bp.data_ptr(), nb[0], back.data_ptr(), n * 4, sh)
        assert rc == 0 and m == n

    for _ in range(3):
        enc()
        dec()
    e = int(np.floor(np.log2(eb)))
    assert float((back - vd).abs().max()) < 2.0 ** e
    t_enc, t_dec = _median_ms(enc, k), _median_ms(dec, k)
    planes = int(np.frombuffer(bp[20:24].cpu().numpy().tobytes(), np.uint32)[0])
    # the lossless stage on the bitplane stream and on one int32 per value
    q32 = torch.trunc(vd.double() / 2.0 ** e).to(torch.int32).contiguous()
    sizes = {}
    for name, buf, nbytes in (("bitplane", bp, nb[0]), ("int32_per_value", q32, n * 4)):
        lcap = G.sz3g_lossless_bound(nbytes)
        lz = torch.empty(lcap, dtype=torch.uint8, device=dev)
        rc, m = G.sz3g_lossless_compress(buf.data_ptr(), nbytes, lz.data_ptr(), lcap, sh)
        assert rc == 0
        sizes[name] = {"bytes": int(nbytes), "after_lossless": int(m)}
    bp_res = {
        "values": n, "input_bytes": n * 4, "stream_bytes": int(nb[0]), "planes": planes,
        "encode_ms": t_enc, "decode_ms": t_dec,
        "encode_GB/s": n * 4 / (t_enc * 1e-3) / 1e9, "decode_GB/s": n * 4 / (t_dec * 1e-3) / 1e9,
        "encode_frac_of_hbm_algorithmic": (n * 4 + nb[0]) / (t_enc * 1e-3) / 1e9 / peak,
        "decode_frac_of_hbm_algorithmic": (n * 4 + nb[0]) / (t_dec * 1e-3) / 1e9 / peak,
        "lossless": sizes,
    }
    del q32, bp, back, vd
    # (2) fixed Huffman table against the built codebook
    x = S.grf((args.size,) * 3, SEED)
    p = G.make_params(x.shape, EB, eb_mode=G.REL, interp=G.CUBIC)
    xd = torch.from_numpy(x.reshape(-1)).to(dev)
    N = x.size
    codes = torch.empty(N + 128, dtype=torch.int16, device=dev)
    unpred = torch.empty(N, dtype=torch.float32, device=dev)
    hist = torch.zeros(65536, dtype=torch.int32, device=dev)
    ws = G.workspace(p, False, dev)
    rc, n_unpred, _ = G.sz3g_predict_quantize(p, xd.data_ptr(), codes.data_ptr(), unpred.data_ptr(), hist.data_ptr(),
                                              ws.data_ptr(), ws.numel(), sh)
    assert rc == 0
    del ws, unpred
    radius, chunk = 32768, 4096
    nsym = 2 * radius
    nch = (N + chunk - 1) // chunk
    wcap = nch * ((chunk * 24 + 31) // 32)
    words = torch.empty(wcap, dtype=torch.int32, device=dev)
    cw = torch.empty(nch, dtype=torch.int32, device=dev)
    tabs = {}
    for name in ("built", "fixed"):
        ln = torch.zeros(65536, dtype=torch.uint8, device=dev)
        cd = torch.zeros(65536, dtype=torch.int32, device=dev)

        def table():
            if name == "built":
                assert G.sz3g_huffman_build(hist.data_ptr(), nsym, ln.data_ptr(), cd.data_ptr(), sh) == 0
            else:
                assert G.sz3g_huffman_fixed(radius, ln.data_ptr(), cd.data_ptr(), sh) == 0

        nw = [0]

        def encode():
            rc, nw[0] = G.sz3g_huffman_encode(codes.data_ptr(), N, ln.data_ptr(), cd.data_ptr(), nsym, chunk,
                                              words.data_ptr(), wcap, cw.data_ptr(), 0, sh)
            assert rc == 0

        table()
        encode()
        t_tab, t_e = _median_ms(table, k), _median_ms(encode, k)
        used = int((ln > 0).sum())
        tabs[name] = {"table_ms": t_tab, "encode_ms": t_e, "encode_GB/s_codes": N * 2 / (t_e * 1e-3) / 1e9,
                      "payload_bytes": nw[0] * 4, "stored_table_bytes": 3 * used if name == "built" else 0}
    line = {"metric": "SZ3-Pastri modules on 1 GB300: unpred-aware quantizer GB/s (input bytes); fixed Huffman",
            "unit": "GB/s", "value": bp_res["encode_GB/s"], "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic", "peak_gbs": peak, "peak_kind": peak_kind,
            "config": {"workload": "2^26 FP32 Laplace prediction differences (scale 200 eb, 5% x100), eb 1e-3; "
                                   f"codes of the {args.size}^3 k^-3 field (REL 1e-3, cubic)",
                       "bitplane": bp_res, "huffman": tabs, "n_unpred": int(n_unpred)}}
    print(json.dumps(line), flush=True)
    return 0


def extras(args, dev, xd, out, nb, pool_labels):
    """Figures of the extensions on the same box, outside the timed region,
    each bounded and each wrapped so that a failure only records its error:
    the uneven 256-field batch (batched graph vs one call per field), the
    per-level selector on the 1024^3 fronts field at REL 1e-4 (fixed,
    sampled, exhaustive and learned choices; network trained on the GPU on
    oracle-labelled small fields) and the lossless stage on the headline
    stream."""
    import numpy as np
    import torch

    from paper_2111_02925_gb300 import synthetic as S
    from paper_2111_02925_gb300 import sz3g as G

    sh = int(torch.cuda.current_stream().cuda_stream)
    res = {}

    def ev_ms(fn, k):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    # (1) batch: 256 uneven fields, one step = compress all + decompress all
    try:
        t0 = time.perf_counter()
        mix = S.batch_shapes(args.fields, 4)
        xs = [grf_gpu(d, 4000 + g, dev).reshape(-1) for g, (d, _, _) in enumerate(mix)]
        params = [G.make_params(d, eb, eb_mode=G.REL, interp=it) for d, eb, it in mix]
        caps = [G.sz3g_compress_bound(p) for p in params]
        streams = [torch.empty(c, dtype=torch.uint8, device=dev) for c in caps]
        outs = [torch.empty_like(x) for x in xs]
        wsc = [G.workspace(p, False, dev) for p in params]
        wsd = [G.workspace(p, True, dev) for p in params]
        nbs = [0] * len(xs)

        def per_field():
            for i, (p, x, s, w) in enumerate(zip(params, xs, streams, wsc)):
                rc, nbs[i] = G.sz3g_compress(p, x.data_ptr(), s.data_ptr(), s.numel(), w.data_ptr(), w.numel(), sh)
                assert rc == 0
            for s, n, o, w in zip(streams, nbs, outs, wsd):
                assert G.sz3g_decompress(s.data_ptr(), n, o.data_ptr(), o.numel() * 4, w.data_ptr(), w.numel(),
                                         sh) == 0

        t_single = ev_ms(per_field, 2)
        del wsc, wsd
        bc = G.Batch(params, [x.data_ptr() for x in xs], [s.data_ptr() for s in streams], caps)
        bd = G.Batch(None, [s.data_ptr() for s in streams], [o.data_ptr() for o in outs],
                     [o.numel() * 4 for o in outs], in_bytes=list(nbs), decompress=True)
        try:
            bc.configure(64, 0)  # branch counts the autotuner picks on this mix
            bd.configure(256, 0)
            t_batch = ev_ms(lambda: (bc.run(sh), bd.run(sh)), 3)
            rc, nb2, _ = bc.results()
            ok = rc == 0 and list(nb2) == list(nbs) and bd.results()[0] == 0
        finally:
            bc.close()
            bd.close()
        in_bytes = sum(x.numel() * 4 for x in xs)
        res["batch"] = {"fields": len(xs), "input_bytes": int(in_bytes), "batched_ms": t_batch,
                        "per_field_ms": t_single, "batched_GB/s": in_bytes / (t_batch * 1e-3) / 1e9,
                        "per_field_GB/s": in_bytes / (t_single * 1e-3) / 1e9, "speedup": t_single / t_batch,
                        "streams_identical": bool(ok), "branches": {"compress": 64, "decompress": 256},
                        "seconds": time.perf_counter() - t0}
        del xs, streams, outs
    except Exception as exc:  # noqa: BLE001
        res["batch"] = {"error": repr(exc)[:300]}
    torch.cuda.empty_cache()

    # (2) selector at the 1024^3 fronts field, REL 1e-4
    try:
        from oracle import mlp as M

        t0 = time.perf_counter()
        jobs, labels, tfeats = pool_labels
        feats, ys = [], []
        for f, lab in zip(tfeats, labels):
            feats.extend(f)
            ys.extend(lab)
        feats = np.array(feats)
        ys = np.array(ys, np.int32)
        w = torch.from_numpy(M.init(feats, 5).astype(np.float32)).to(dev)
        fd = torch.from_numpy(feats.astype(np.float32).reshape(-1)).to(dev)
        yd = torch.from_numpy(ys).to(dev)
        md = torch.ones(len(ys) * 8, dtype=torch.uint8, device=dev)
        loss = G.sz3g_mlp_train(w.data_ptr(), fd.data_ptr(), md.data_ptr(), yd.data_ptr(), len(ys), 0.3, 3000, sh)
        n = 1024
        x = fronts_gpu((n, n, n), 5, 16, dev).reshape(-1)
        p = G.make_params((n, n, n), 1e-4, eb_mode=G.REL, interp=G.LINEAR)
        cap = G.sz3g_compress_bound(p)
        o = torch.empty(cap, dtype=torch.uint8, device=dev)
        wsx = G.workspace(p, False, dev)

        def size(q):
            rc, m = G.sz3g_compress(q, x.data_ptr(), o.data_ptr(), cap, wsx.data_ptr(), wsx.numel(), sh)
            assert rc == 0
            return m

        def sel_ms(fn):
            fn()
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            return r, (time.perf_counter() - t) * 1e3

        ch_s, ms_s = sel_ms(lambda: G.sz3g_select_sampled(p, x.data_ptr(), 64, 1, sh))
        ch_l, ms_l = sel_ms(lambda: G.sz3g_select_learned(p, x.data_ptr(), w.data_ptr(), 16, 1, sh))
        ch_e, ms_e = sel_ms(lambda: G.sz3g_select_sampled(p, x.data_ptr(), 0, 1, sh))
        raw = x.numel() * 4
        sizes = {"fixed_linear_012": size(p),
                 "fixed_cubic_012": size(G.make_params((n, n, n), 1e-4, eb_mode=G.REL, interp=G.CUBIC)),
                 "exhaustive": size(G.params_for_choices(p, ch_e)), "sampled": size(G.params_for_choices(p, ch_s)),
                 "learned": size(G.params_for_choices(p, ch_l))}
        res["selector"] = {"workload": "1024^3 FP32 k^-3 field + 16 tanh fronts (seed 5), REL 1e-4",
                           "ratio": {k: raw / v for k, v in sizes.items()},
                           "learned_vs_sampled": sizes["sampled"] / sizes["learned"],
                           "learned_vs_fixed_linear": sizes["fixed_linear_012"] / sizes["learned"],
                           "selection_ms": {"sampled": ms_s, "learned": ms_l, "exhaustive": ms_e},
                           "training": {"fields": len(jobs), "examples": int(len(ys)), "final_loss": loss},
                           "seconds": time.perf_counter() - t0}
        del x, o, wsx
    except Exception as exc:  # noqa: BLE001
        res["selector"] = {"error": repr(exc)[:300]}
    torch.cuda.empty_cache()

    # (3) lossless stage on the headline stream
    try:
        lcap = G.sz3g_lossless_bound(nb)
        lz = torch.empty(lcap, dtype=torch.uint8, device=dev)
        back = torch.empty(nb + 16, dtype=torch.uint8, device=dev)
        m = [0]

        def comp():
            rc, m[0] = G.sz3g_lossless_compress(out.data_ptr(), nb, lz.data_ptr(), lcap, sh)
            assert rc == 0

        def dec():
            rc, n2 = G.sz3g_lossless_decompress(lz.data_ptr(), m[0], back.data_ptr(), nb, sh)
            assert rc == 0 and n2 == nb

        tc = ev_ms(comp, 3)
        td = ev_ms(dec, 3)
        res["lossless"] = {"stream_bytes": int(nb), "lossless_bytes": int(m[0]), "gain": nb / m[0],
                           "compress_GB/s": nb / (tc * 1e-3) / 1e9, "decompress_GB/s": nb / (td * 1e-3) / 1e9,
                           "identical": bool(torch.equal(back[:nb], out[:nb]))}
    except Exception as exc:  # noqa: BLE001
        res["lossless"] = {"error": repr(exc)[:300]}
    return res


def label_jobs(n_fields, size=0):
    """Oracle labels (exhaustive trial) and features of n training fields (size^3
    points, or 32..64 per axis at random for size 0), in a spawned process
    pool: (jobs, labels, features)."""
    import multiprocessing as mp

    import numpy as np

    rng = np.random.default_rng(31)
    jobs = []
    for i in range(n_fields):
        shape = (size, size, size) if size > 0 else tuple(int(v) for v in rng.integers(32, 65, 3))
        eb = float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-2))))
        jobs.append((shape, 20000 + i, int(rng.integers(0, 17)), eb))
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        out = pool.map(_label_field, jobs, chunksize=4)
    return jobs, [o[0] for o in out], [o[1] for o in out]


def main():
    args = parse()
    if args.workload == "lossless":
        return run_lossless(args)
    if args.workload == "pastri":
        return run_pastri(args)
    if args.workload == "selector":
        return run_selector(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    import numpy as np
    import torch

    from paper_2111_02925_gb300 import build as B
    from paper_2111_02925_gb300 import synthetic as S
    from paper_2111_02925_gb300 import sz3g as G

    ws, rank, local = dist_env()
    pool_labels = None
    if rank == 0 and ws == 1 and not args.no_extras:
        try:  # the oracle's labels for the selector figure, before any GPU call
            pool_labels = label_jobs(args.extra_train_fields)
        except Exception:  # noqa: BLE001
            pool_labels = None
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    B.build()
    G.load()
    n = args.size
    x = S.grf((n, n, n), SEED)
    xd = torch.from_numpy(x).to(dev)
    p = G.make_params(x.shape, EB, eb_mode=G.REL, interp=G.CUBIC)
    wsc, wsd = G.workspace(p, False, dev), G.workspace(p, True, dev)
    out = torch.empty(G.sz3g_compress_bound(p), dtype=torch.uint8, device=dev)
    y = torch.empty(x.size, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)

    def step():
        rc, nb = G.sz3g_compress(p, xd.data_ptr(), out.data_ptr(), out.numel(), wsc.data_ptr(), wsc.numel(), sh)
        if rc:
            raise G.SZ3GError(rc, "compress")
        rc = G.sz3g_decompress(out.data_ptr(), nb, y.data_ptr(), y.numel() * 4, wsd.data_ptr(), wsd.numel(), sh)
        if rc:
            raise G.SZ3GError(rc, "decompress")
        return nb

    nb = 0
    for _ in range(max(args.warmup, 3)):
        nb = step()
    torch.cuda.synchronize()
    diff = (y - xd.reshape(-1)).double()
    maxerr = float(diff.abs().max().item())
    mse = float((diff * diff).mean().item())
    vrange = float(xd.max().item()) - float(xd.min().item())
    psnr = 20.0 * np.log10(vrange) - 10.0 * np.log10(mse) if mse > 0 else float("inf")
    del diff
    # timed region
    clocks = Clocks(torch.cuda.current_device())
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.1)
    launches0 = G.sz3g_launch_count()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    e[0].record(stream)
    for k in range(args.steps):
        rc, nbk = G.sz3g_compress(p, xd.data_ptr(), out.data_ptr(), out.numel(), wsc.data_ptr(), wsc.numel(), sh)
        e[2 * k + 1].record(stream)
        rc2 = G.sz3g_decompress(out.data_ptr(), nbk, y.data_ptr(), y.numel() * 4, wsd.data_ptr(), wsd.numel(), sh)
        e[2 * k + 2].record(stream)
        if rc or rc2:
            raise RuntimeError(f"status {rc} {rc2}")
    torch.cuda.synchronize()
    launches = G.sz3g_launch_count() - launches0
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = e[0].elapsed_time(e[-1])
    comp_ms = sum(e[2 * k].elapsed_time(e[2 * k + 1]) for k in range(args.steps)) / args.steps
    dec_ms = sum(e[2 * k + 1].elapsed_time(e[2 * k + 2]) for k in range(args.steps)) / args.steps
    step_ms = total_ms / args.steps
    # per-kernel times from a separate profiled pass (CUDA events around every
    # launch; with profiling on the calls launch kernel by kernel, not as a
    # cached graph), outside the timed region
    nprof = max(1, min(args.steps, 10))
    torch.cuda.synchronize()
    G.sz3g_profile_enable(True)
    for _ in range(nprof):
        step()
    torch.cuda.synchronize()
    kern = {}
    for name in G.sz3g_profile_kernel_names():
        t, c = G.sz3g_profile_read(name)
        if c:
            kern[name] = (t / nprof, c / nprof)
    G.sz3g_profile_enable(False)
    step_ms, comp_ms, dec_ms = reduce_over_ranks([step_ms, comp_ms, dec_ms], "max", dev)
    in_bytes = x.nbytes
    value = ws * in_bytes / (step_ms * 1e-3) / 1e9
    # roofline of the dominant kernel
    import struct

    head = out[:288].cpu().numpy().tobytes()
    n_unpred = struct.unpack_from("<Q", head, 88)[0]
    n_words = struct.unpack_from("<Q", head, 104)[0]
    coarse = sum(int(np.prod([-(-n // (1 << k))] * 3)) for k in range(1, 10))
    info = {"N": x.size, "esz": 4, "coarse_points": coarse, "payload_bytes": n_words * 4, "n_unpred": n_unpred,
            "stream_bytes": nb}
    peak, peak_kind = peaks()
    dom = max(kern.items(), key=lambda kv: kv[1][0]) if kern else None
    comp_frac = (in_bytes * 2 + nb) / (comp_ms * 1e-3) / 1e9 / peak
    dec_frac = (in_bytes + nb) / (dec_ms * 1e-3) / 1e9 / peak
    roof = None
    if dom:
        name, (ms_per_step, l_per_step) = dom
        byts = algorithmic_bytes(name, info)
        ach = byts / (ms_per_step * 1e-3) / 1e9
        launches_per_step = max(l_per_step, 1.0)
        tr = traffic_for(name)
        roof = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_kind": peak_kind, "traffic": (tr / launches_per_step) if tr else None,
                "traffic_per_step": tr, "launches_per_step": l_per_step, "ms_per_step": ms_per_step,
                "algorithmic_bytes_per_step": byts, "implementation_bytes_per_step": implementation_bytes(name, info),
                "per_direction": {"compress": comp_frac, "decompress": dec_frac,
                                  "compress_algorithmic_bytes": in_bytes * 2 + nb,
                                  "decompress_algorithmic_bytes": in_bytes + nb}}
    # end to end through the host-buffer entry points (pinned host memory)
    e2e = None
    if not args.no_e2e:
        hx = torch.from_numpy(x).reshape(-1).pin_memory()
        hs = torch.empty(out.numel(), dtype=torch.uint8).pin_memory()
        hy = torch.empty(x.size, dtype=torch.float32).pin_memory()
        ke = min(args.steps, 5)
        nbh = 0
        hst = int(torch.cuda.Stream().cuda_stream)  # a stream of the caller's own, as a user would
        for _ in range(2):
            rc, nbh = G.sz3g_compress_host(p, hx.data_ptr(), hs.data_ptr(), hs.numel(), hst)
            G.sz3g_decompress_host(hs.data_ptr(), nbh, hy.data_ptr(), hy.numel() * 4, hst)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            rc, nbh = G.sz3g_compress_host(p, hx.data_ptr(), hs.data_ptr(), hs.numel(), hst)
            rc2 = G.sz3g_decompress_host(hs.data_ptr(), nbh, hy.data_ptr(), hy.numel() * 4, hst)
            if rc or rc2:
                raise RuntimeError(f"host status {rc} {rc2}")
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / ke
        e2e = {"value": ws * in_bytes / dt / 1e9, "unit": "GB/s", "h2d_bytes_per_step": in_bytes + nbh,
               "d2h_bytes_per_step": nbh + in_bytes, "ms_per_step": dt * 1e3}
    # the other bounds of the 512^3 configuration, outside the timed region
    sweep = None
    if rank == 0 and not args.no_sweep:
        sweep = {}
        for eb in (1e-2, 1e-4):
            pe = G.make_params(x.shape, eb, eb_mode=G.REL, interp=G.CUBIC)
            wse, wde = G.workspace(pe, False, dev), G.workspace(pe, True, dev)
            oute = torch.empty(G.sz3g_compress_bound(pe), dtype=torch.uint8, device=dev)
            nbe = [0]

            def comp_e():
                rc, nbe[0] = G.sz3g_compress(pe, xd.data_ptr(), oute.data_ptr(), oute.numel(), wse.data_ptr(),
                                             wse.numel(), sh)
                assert rc == 0

            def dec_e():
                rc = G.sz3g_decompress(oute.data_ptr(), nbe[0], y.data_ptr(), y.numel() * 4, wde.data_ptr(),
                                       wde.numel(), sh)
                assert rc == 0

            for _ in range(3):
                comp_e()
                dec_e()
            tc, td = _median_ms(comp_e, 20), _median_ms(dec_e, 20)
            err = float((y - xd.reshape(-1)).abs().max())
            sweep[f"rel{eb:g}"] = {"compress_ms": tc, "decompress_ms": td,
                                   "GB/s": in_bytes / ((tc + td) * 1e-3) / 1e9,  # per compress + decompress step
                                   "compression_ratio": in_bytes / nbe[0], "max_abs_error": err}
            del wse, wde, oute
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(x)
    ext = None
    if rank == 0 and ws == 1 and not args.no_extras:
        ext = extras(args, dev, xd, out, nb, pool_labels or ([], [], []))
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(n),
            "compress": {"ms": comp_ms, "GB/s": in_bytes / (comp_ms * 1e-3) / 1e9,
                         "frac_of_hbm_algorithmic": comp_frac},
            "decompress": {"ms": dec_ms, "GB/s": in_bytes / (dec_ms * 1e-3) / 1e9,
                           "frac_of_hbm_algorithmic": dec_frac},
            "compression_ratio": in_bytes / nb, "bits_per_value": 8.0 * nb / x.size, "psnr_db": psnr,
            "max_abs_error": maxerr, "stream_bytes": nb, "n_unpred": n_unpred,
            "roofline": roof, "kernels_ms_per_step": {k: v[0] for k, v in sorted(kern.items())},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk, "eb_sweep": sweep,
            "extras": ext,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
