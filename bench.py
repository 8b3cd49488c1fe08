"""QLC codec benchmark on GB300 (one JSON line on stdout).

Workload: one 256 MiB e4m3 tensor shaped [16384 x 16384] (block-32 absmax
scaled Student-t(4) values, seed = rank), chunk 4096 symbols, Table 1 scheme.
A step is one pass of the whole hot path over it: histogram -> LUT ->
encode -> decode (every kernel of libqlc), followed by nothing on the host.
value = raw bytes per second over all ranks (replicas, no collective).

Legs: the device-timed step (CUDA events on the launching stream, inputs
resident in HBM), per-kernel durations from events between the launches, an
end-to-end leg through the same C ABI with pinned host buffers (host->device
copy of the input, encode, container read back, container copied in,
decode, decoded bytes read back), and the CPU oracle on a bounded sample of
the same tensor.  --impl reference times the CPU oracle alone.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_BYTES = 16384 * 16384
CHUNK = 4096
SCHEME = 1
WORKLOAD = "qlc_roundtrip_256MiB_t4_e4m3"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The largest per-rank value: a replicated job is as slow as its slowest rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, bytes_per_rank: int, ms_max: float) -> float:
    """GB/s of the whole job: every rank codes its own tensor (weak scaling)."""
    return world * bytes_per_rank / (ms_max * 1e-3) / 1e9


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic_for(kernel_file: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_2602_17849_gb300", "csrc", kernel_file)
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(path):
            f = line.split()
            if len(f) >= 4 and f[0] == kernel_file and f[1] == digest and f[2] == WORKLOAD:
                return float(f[3])
    except OSError:
        pass
    return None


def cpu_oracle_roundtrip(x_host, budget_s: float = 12.0, slice_bytes: int = 16 << 20, max_bytes=None):
    """Oracle histogram + rank + encode + decode on consecutive slices of x_host
    (wrapping around to its start) until about budget_s of CPU time or
    max_bytes coded; returns (bytes, seconds)."""
    import numpy as np

    import oracle
    done, t = 0, 0.0
    n = x_host.size
    while t < budget_s and (max_bytes is None or done < max_bytes):
        off = done % n
        s = x_host[off:off + slice_bytes]
        t0 = time.perf_counter()
        c = oracle.encode(s, scheme_id=SCHEME, chunk_symbols=CHUNK)
        st, y, _ = oracle.decode(c)
        t += time.perf_counter() - t0
        assert st == 0 and np.array_equal(y, s)
        done += s.size
    return done, t


def _oracle_slice_worker(s):
    """One oracle round trip of slice s in a worker process (spawned, so it
    holds no CUDA state); returns the bytes coded."""
    import numpy as np

    import oracle
    c = oracle.encode(s, scheme_id=SCHEME, chunk_symbols=CHUNK)
    st, y, _ = oracle.decode(c)
    if st != 0 or not np.array_equal(y, s):
        raise RuntimeError("oracle round trip failed")
    return int(s.size)


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


class OraclePool:
    """The oracle on every host core: `cores` spawned worker processes, each
    coding its own slice (one oracle call per slice, as it stands).  Worker
    start-up and library loading happen before any timing; a worker that
    cannot start raises instead of being replaced."""

    def __init__(self, cores: int):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor

        import numpy as np
        self.cores = cores
        self.pool = ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"))
        list(self.pool.map(_oracle_slice_worker, [np.zeros(4096, np.uint8)] * cores))

    def run(self, x_host, budget_s: float, slice_bytes: int = 16 << 20, max_bytes=None, start: int = 0):
        """Consecutive slices of x_host from byte `start` (wrapping around),
        one per core in flight, until budget_s of wall time or max_bytes
        submitted; returns (bytes, wall seconds)."""
        n = x_host.size
        submitted, done = 0, 0

        def submit():
            nonlocal submitted
            off = (start + submitted) % n
            sl = x_host[off:off + slice_bytes]
            submitted += sl.size
            return self.pool.submit(_oracle_slice_worker, sl)

        t0 = time.perf_counter()
        pending = [submit() for _ in range(self.cores)]
        while pending:
            done += pending.pop(0).result()
            if time.perf_counter() - t0 < budget_s and (max_bytes is None or submitted < max_bytes):
                pending.append(submit())
        return done, time.perf_counter() - t0

    def close(self):
        self.pool.shutdown()


def _config(world: int) -> dict:
    """The workload both arms report."""
    return {"workload": WORKLOAD, "shape": [16384, 16384], "n_bytes": N_BYTES,
            "chunk_symbols": CHUNK, "scheme": "Table 1", "kind": "student_t4_block32_e4m3",
            "l2": "inputs larger than L2 (256 MiB in, ~230 MB container, 256 MiB out per step)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """--impl reference: the CPU oracle on the host cores (rank 0 only)."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    import torch

    from paper_2602_17849_gb300 import inputs
    x = inputs.make_e4m3("t4", N_BYTES, seed=0).numpy()
    slice_bytes = 16 << 20
    cores = host_cores()
    pool = OraclePool(cores)
    step_bytes = cores * slice_bytes   # one slice per core per step
    for k in range(args.warmup):
        pool.run(x, budget_s=0.0, slice_bytes=slice_bytes, max_bytes=step_bytes, start=k * step_bytes)
    times, done = [], 0
    for k in range(args.steps):
        b, t = pool.run(x, budget_s=0.0, slice_bytes=slice_bytes, max_bytes=step_bytes,
                        start=(args.warmup + k) * step_bytes)
        times.append(t)
        done += b
    pool.close()
    tot = sum(times)
    value = done / tot / 1e9
    sample = (f"{cores} x {slice_bytes >> 20} MiB slices of the 256 MiB tensor per step, one per host core "
              f"(oracle encode+decode)")
    line = {
        "metric": "QLC encode+decode round trip, raw GB/s", "value": value, "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic", "impl": "reference",
        "config": _config(world),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    del torch
    return 0


def e2e_leg(dev, x, steps: int, slots: int = 3):
    """The round trip from and to pinned host memory through the C ABI: the
    input's copy to the device, histogram, LUT and encode, the container's copy
    to the host and back, decode, and the output's copy to the host, every
    step.  `slots` round trips are in flight on as many streams, so one step's
    copies in one direction overlap another's in the other direction and the
    kernels (each slot owns its device and host buffers; a step waits for its
    own container size before copying the container).  The serial latency of
    one round trip on an idle GPU is reported beside it."""
    import torch

    from paper_2602_17849_gb300 import qlc
    n = x.numel()
    hx = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    hx.copy_(x)

    class Slot:
        def __init__(self):
            self.stream = torch.cuda.Stream(device=dev)
            self.codec = qlc.Codec(n, CHUNK, SCHEME, dev)
            self.xin = torch.empty(n, dtype=torch.uint8, device=dev)
            self.cont = self.codec.new_container()
            self.cin = torch.empty_like(self.cont)
            self.y = torch.empty(n, dtype=torch.uint8, device=dev)
            self.hc = torch.empty(self.codec.cap, dtype=torch.uint8, pin_memory=True)
            self.hy = torch.empty(n, dtype=torch.uint8, pin_memory=True)
            self.hb = torch.empty(1, dtype=torch.int64, pin_memory=True)
            self.sized = torch.cuda.Event()
            self.nb = 0

        def encode(self):  # input in, histogram, LUT, encode, container size out
            c, st = self.codec, self.stream
            with torch.cuda.stream(st):
                self.xin.copy_(hx, non_blocking=True)
                qlc.qlc_histogram(self.xin, c.hist, stream=st)
                qlc.qlc_build_lut(c.hist, SCHEME, c.lut, stream=st)
                qlc.qlc_encode(self.xin, c.lut, CHUNK, self.cont, c.ws, c.out_bytes, c.status, stream=st)
                self.hb.copy_(c.out_bytes, non_blocking=True)
                self.sized.record(st)

        def decode(self):  # container out and back in, decode, output out
            c, st = self.codec, self.stream
            self.sized.synchronize()
            nb = self.nb = int(self.hb.item())
            with torch.cuda.stream(st):
                self.hc[:nb].copy_(self.cont[:nb], non_blocking=True)
                self.cin[:nb].copy_(self.hc[:nb], non_blocking=True)
                qlc.qlc_decode(self.cin, self.y, c.n_out, c.status, in_bytes=nb, stream=st)
                self.hy.copy_(self.y, non_blocking=True)

    pool = [Slot() for _ in range(slots)]

    def run(k_steps):
        for k in range(k_steps + 1):
            if k < k_steps:
                pool[k % slots].encode()
            if k >= 1:
                pool[(k - 1) % slots].decode()
        torch.cuda.synchronize(dev)

    run(slots)  # warm-up
    t0 = time.perf_counter()
    run(steps)
    pipelined_s = (time.perf_counter() - t0) / steps
    for sl in pool:
        sl.codec.check()
        assert torch.equal(sl.hy, hx), "e2e round trip is not bit-exact"
    lat = []
    for _ in range(3):
        t0 = time.perf_counter()
        pool[0].encode()
        pool[0].decode()
        torch.cuda.synchronize(dev)
        lat.append(time.perf_counter() - t0)
    nb = pool[0].nb
    return {"value": n / pipelined_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": n + nb,
            "d2h_bytes_per_step": 8 + nb + n, "steps": steps, "round_trips_in_flight": slots,
            "serial_round_trip_ms": statistics.median(lat) * 1e3,
            "serial_gbs": n / statistics.median(lat) / 1e9}


def large_leg(dev, steps: int, warmup: int, peak: float):
    """Batched large: 64 shards x 64 MiB of Laplace(b=1) with 1 % N(0, 20^2)
    outliers, encoded and decoded as one batch (one CUDA graph per direction),
    with one shared LUT and with one LUT per shard."""
    import torch

    from paper_2602_17849_gb300 import inputs, qlc
    arena, shards = inputs.cfg4_batch(dev)
    total = sum(x.numel() for x in shards)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    out = {"workload": "64 shards x 64 MiB, Laplace(b=1) + 1 % N(0, 20^2) outliers, e4m3, chunk 4096"}
    for shared in (True, False):
        b = qlc.Batch(shards, 4096, schemes=(1,), shared_lut=shared)
        b.capture()
        enc_ms = timed(lambda: b.replay("encode"))
        dec_ms = timed(lambda: b.replay("decode"))
        b.check()
        exact = all(torch.equal(b.output(i), x) for i, x in enumerate(shards))
        c = int(b.c_bytes.sum().item())
        out["shared_lut" if shared else "per_shard_lut"] = {
            "encode_ms": enc_ms, "decode_ms": dec_ms,
            "encode_gbs": total / (enc_ms * 1e-3) / 1e9, "decode_gbs": total / (dec_ms * 1e-3) / 1e9,
            "encode_roofline_frac": (2 * total + c) / (enc_ms * 1e-3) / 1e9 / peak,
            "decode_roofline_frac": (total + c) / (dec_ms * 1e-3) / 1e9 / peak,
            "compressibility": 1 - c / total, "bit_exact": exact}
        del b
    return out


def batched_leg(dev, steps: int, warmup: int, peak: float, n_shards: int = 1152, shape=None):
    """The batched workload (1152 shards, 64 KiB - 16 MiB, t4 / gauss / laplace,
    per-shard LUTs): one CUDA graph per direction with the autotuned launch
    shape, against per-tensor launches of the plain kernels (eager, and the
    same launches captured in a graph)."""
    import torch

    from paper_2602_17849_gb300 import autotune, inputs, qlc
    arena, shards = inputs.cfg3_batch(dev, n_shards)
    torch.cuda.empty_cache()
    total = sum(x.numel() for x in shards)
    if shape is None:
        cfg = autotune.tune(shards)
    else:  # a fixed launch shape (profiling captures): no tuning launches
        cfg = dict(zip(("chunk_symbols", "encode_ctas_per_sm", "decode_ctas_per_sm"), shape))
    cs = cfg["chunk_symbols"]
    b = qlc.Batch(shards, cs, launch=(cfg["encode_ctas_per_sm"], cfg["decode_ctas_per_sm"]))
    b.capture()
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    enc_ms = timed(lambda: b.replay("encode"), steps)
    dec_ms = timed(lambda: b.replay("decode"), steps)
    b.check()
    exact = all(torch.equal(b.output(i), x) for i, x in enumerate(shards))
    c_total = int(b.c_bytes.sum().item())

    # per-tensor launches of the plain kernels on the same buffers
    n = len(shards)
    ws_sizes = [qlc.qlc_encode_workspace_size(x.numel(), cs) for x in shards]
    ws = torch.zeros(sum(ws_sizes) + 16 * n, dtype=torch.uint8, device=dev)
    ws_off = [0]
    for w in ws_sizes:
        ws_off.append(ws_off[-1] + (w + 15) // 16 * 16)
    hist = b.hists.view(n, 256)
    luts = b.luts.view(n, qlc.LUT_BYTES)
    cbytes = b.c_bytes
    nout = b.n_out
    caps = [b.cap_off[i + 1] - b.cap_off[i] for i in range(n)]

    def plain_round_trip():
        for i, x in enumerate(shards):
            qlc.qlc_histogram(x, hist[i], stream=stream)
            qlc.qlc_build_lut(hist[i], SCHEME, luts[i], stream=stream)
            qlc.qlc_encode(x, luts[i], cs, b.container(i), ws[ws_off[i]:ws_off[i + 1]], cbytes[i:i + 1],
                           b.status, stream=stream)
        for i, x in enumerate(shards):
            qlc.qlc_decode(b.container(i), b.output(i), nout[i:i + 1], b.status, in_bytes=caps[i],
                           out_cap=x.numel(), stream=stream)

    plain_ms = timed(plain_round_trip, 3)

    # the same per-tensor launches spread round-robin over four streams (as
    # the server runs its batches), each shard's encode and decode on one
    # stream: the concurrent baseline
    pool = [torch.cuda.Stream(device=dev) for _ in range(4)]

    def plain_multistream():
        start = torch.cuda.Event()
        start.record(stream)
        for s in pool:
            s.wait_event(start)
        for i, x in enumerate(shards):
            s = pool[i % 4]
            qlc.qlc_histogram(x, hist[i], stream=s)
            qlc.qlc_build_lut(hist[i], SCHEME, luts[i], stream=s)
            qlc.qlc_encode(x, luts[i], cs, b.container(i), ws[ws_off[i]:ws_off[i + 1]], cbytes[i:i + 1],
                           b.status, stream=s)
            qlc.qlc_decode(b.container(i), b.output(i), nout[i:i + 1], b.status, in_bytes=caps[i],
                           out_cap=x.numel(), stream=s)
        for s in pool:
            done = torch.cuda.Event()
            done.record(s)
            stream.wait_event(done)

    plain_ms_4s = timed(plain_multistream, 3)
    b.check()
    exact = exact and all(torch.equal(b.output(i), x) for i, x in enumerate(shards))
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream(device=dev)
    s2.wait_stream(stream)
    with torch.cuda.graph(g, stream=s2):
        for i, x in enumerate(shards):
            cur = torch.cuda.current_stream(dev)
            qlc.qlc_histogram(x, hist[i], stream=cur)
            qlc.qlc_build_lut(hist[i], SCHEME, luts[i], stream=cur)
            qlc.qlc_encode(x, luts[i], cs, b.container(i), ws[ws_off[i]:ws_off[i + 1]], cbytes[i:i + 1],
                           b.status, stream=cur)
        for i, x in enumerate(shards):
            qlc.qlc_decode(b.container(i), b.output(i), nout[i:i + 1], b.status, in_bytes=caps[i],
                           out_cap=x.numel(), stream=torch.cuda.current_stream(dev))
    plain_graph_ms = timed(lambda: g.replay(), 3)
    b.check()
    exact = exact and all(torch.equal(b.output(i), x) for i, x in enumerate(shards))
    r = c_total / total
    rt_ms = enc_ms + dec_ms
    dec_bytes = total + c_total
    enc_bytes = 2 * total + c_total  # the histogram reads the input once more
    return {
        "workload": f"{n} shards, 64 KiB-16 MiB log-uniform, t4/gauss/laplace e4m3, per-shard LUT",
        "total_bytes": total, "container_bytes": c_total, "compressibility": 1 - r,
        "tuned": {k: cfg[k] for k in ("chunk_symbols", "encode_ctas_per_sm", "decode_ctas_per_sm")},
        "encode_ms": enc_ms, "decode_ms": dec_ms, "round_trip_gbs": total / (rt_ms * 1e-3) / 1e9,
        "decode_gbs": total / (dec_ms * 1e-3) / 1e9,
        "decode_roofline_frac": dec_bytes / (dec_ms * 1e-3) / 1e9 / peak,
        "encode_gbs": total / (enc_ms * 1e-3) / 1e9,
        "encode_roofline_frac": enc_bytes / (enc_ms * 1e-3) / 1e9 / peak,
        "encode_bytes_counted": "(2 + r) N: histogram read + encode read + container write",
        "plain_per_tensor_eager_ms": plain_ms, "plain_per_tensor_graph_ms": plain_graph_ms,
        "plain_per_tensor_4streams_ms": plain_ms_4s,
        "batched_ms": rt_ms, "speedup_vs_plain_eager": plain_ms / rt_ms,
        "speedup_vs_plain_graph": plain_graph_ms / rt_ms, "speedup_vs_plain_4streams": plain_ms_4s / rt_ms,
        "bit_exact_round_trip": bool(exact),
        "launches_per_round_trip": {"batched": 7, "plain": 4 * n},
    }


def fused_leg(dev, steps: int, warmup: int, peak: float, n: int = N_BYTES):
    """Block-32 e4m3 quantisation fused into the codec: a [16384 x 16384] fp32
    Student-t(4) activation tensor (the values the headline tensor quantises),
    encoded as quantise + histogram -> LUT -> encode and decoded straight to
    fp32, against the same work with a separate histogram pass and a separate
    dequantisation pass.  Every output is checked bit-exact against the
    unfused path."""
    import torch

    from paper_2602_17849_gb300 import inputs, qlc
    x = inputs.make_f32("t4", n, seed=0, device=dev)
    torch.cuda.empty_cache()
    codes = torch.empty(n, dtype=torch.uint8, device=dev)
    scales = torch.empty((n + 31) // 32, dtype=torch.float32, device=dev)
    codec = qlc.Codec(n, CHUNK, SCHEME, dev)
    cont = codec.new_container()
    y = torch.empty(n, dtype=torch.float32, device=dev)
    y2 = torch.empty(n, dtype=torch.float32, device=dev)
    codes2 = torch.empty(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def enc_fused():
        qlc.qlc_quantize_e4m3(x, codes, scales, codec.hist, codec.status, stream=stream)
        qlc.qlc_build_lut(codec.hist, SCHEME, codec.lut, stream=stream)
        qlc.qlc_encode(codes, codec.lut, CHUNK, cont, codec.ws, codec.out_bytes, codec.status, stream=stream)

    def enc_plain():
        qlc.qlc_quantize_e4m3(x, codes, scales, None, codec.status, stream=stream)
        qlc.qlc_histogram(codes, codec.hist, stream=stream)
        qlc.qlc_build_lut(codec.hist, SCHEME, codec.lut, stream=stream)
        qlc.qlc_encode(codes, codec.lut, CHUNK, cont, codec.ws, codec.out_bytes, codec.status, stream=stream)

    def dec_fused():
        qlc.qlc_decode_dequantize(cont, scales, y, codec.n_out, codec.status, stream=stream)

    def dec_plain():
        qlc.qlc_decode(cont, codes2, codec.n_out, codec.status, stream=stream)
        qlc.qlc_dequantize_e4m3(codes2, scales, y2, stream=stream)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    t_ef, t_ep, t_df, t_dp = timed(enc_fused), timed(enc_plain), timed(dec_fused), timed(dec_plain)
    codec.check()
    c_bytes = int(codec.out_bytes.item())
    assert torch.equal(y.view(torch.int32), y2.view(torch.int32)) and torch.equal(codes, codes2)
    # quantise + histogram alone, for its roofline; dequantise alone; bf16 input
    t_q = timed(lambda: qlc.qlc_quantize_e4m3(x, codes, scales, codec.hist, codec.status, stream=stream))
    t_dq = timed(lambda: qlc.qlc_dequantize_e4m3(codes2, scales, y2, stream=stream))
    xb = x.to(torch.bfloat16)
    t_qb = timed(lambda: qlc.qlc_quantize_e4m3(xb, codes2, scales, codec.hist, codec.status, stream=stream))
    codec.check()
    del xb
    q_bytes = 4 * n + n + n // 8
    qb_bytes = 2 * n + n + n // 8
    dq_bytes = n + n // 8 + 4 * n
    d_bytes = c_bytes + n // 8 + 4 * n
    return {
        "workload": f"{n} fp32 Student-t(4) activations, block-32 e4m3, chunk 4096, Table 1",
        "encode_fused_ms": t_ef, "encode_unfused_ms": t_ep, "decode_fused_ms": t_df, "decode_unfused_ms": t_dp,
        "encode_fused_gbs_fp32": 4 * n / (t_ef * 1e-3) / 1e9, "decode_fused_gbs_fp32": 4 * n / (t_df * 1e-3) / 1e9,
        "speedup_encode": t_ep / t_ef, "speedup_decode": t_dp / t_df,
        "quantize_hist_ms": t_q, "quantize_hist_roofline_frac": q_bytes / (t_q * 1e-3) / 1e9 / peak,
        "quantize_hist_bf16_ms": t_qb, "quantize_hist_bf16_roofline_frac": qb_bytes / (t_qb * 1e-3) / 1e9 / peak,
        "dequantize_ms": t_dq, "dequantize_roofline_frac": dq_bytes / (t_dq * 1e-3) / 1e9 / peak,
        "decode_dequantize_roofline_frac": d_bytes / (t_df * 1e-3) / 1e9 / peak,
        "bytes_counted": "quantise+hist: 4N (bf16: 2N) read + N codes + N/8 scales written; dequantise: N + N/8 "
                         "read, 4N written; decode->fp32: C + N/8 read, 4N written",
        "bit_exact_vs_unfused": True,
    }


def serve_leg(dev, seconds: float):
    """Serving: Poisson arrivals at 20,000 requests/s, half compress and half
    decompress, sizes log-uniform 4 KiB - 64 MiB of Student-t e4m3 data
    resident on the device, 8 GiB admission budget (in + out + workspace),
    continuous batching over 4 streams."""
    import torch

    from paper_2602_17849_gb300 import serve
    wl = serve.CudaWorkload(dev, data_bytes=1 << 30, n_containers=128, min_size=4 << 10,
                            max_size=64 << 20, seed=3000)
    torch.cuda.empty_cache()
    # A sample of the results (every 499th request of at most 16 MiB, up to
    # 24) is copied aside on the device as it completes, without a host wait
    # in the serving loop, and checked afterwards: a container must decode
    # (with the library) to its request's input, decoded bytes must equal the
    # source the container was made from.  The oracle comparison of served
    # results at this scale is a GPU test.
    qlc_cap = 17 << 20
    keep = torch.empty(24 * qlc_cap, dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream(device=dev)
    kept = []

    def sample(r, ex):
        if r.rid % 499 or len(kept) >= 24 or r.status != 0:
            return
        off, nb = r.result
        if nb > qlc_cap or (r.n_in if r.kind == "compress" else r.n_out) > 16 << 20:
            return
        slot = len(kept) * qlc_cap
        with torch.cuda.stream(side):
            keep[slot:slot + nb].copy_(ex.dev_arena[off:off + nb], non_blocking=True)
        kept.append((r, slot, nb))

    reqs, ex, srv, wall = serve.serve_run(dev, rate_hz=20_000, duration_s=seconds, budget_bytes=8 << 30,
                                          workload=wl, seed=3001, on_complete=sample)
    done = [r for r in reqs if r.done is not None]
    lat = serve.percentiles([r.latency for r in done])
    raw = sum(r.n_in if r.kind == "compress" else r.n_out for r in done)
    ok = all(r.status == 0 for r in done)
    torch.cuda.synchronize()
    from paper_2602_17849_gb300 import qlc
    exact = True
    for r, slot, nb in kept:
        got = keep[slot:slot + nb]
        if r.kind == "compress":
            exact = exact and torch.equal(qlc.decode(got), wl.pool[r.in_ref:r.in_ref + r.n_in])
        else:
            _off, _nb, n, src_off = next(c for c in wl.containers if c[0] == r.in_ref)
            exact = exact and torch.equal(got, wl.pool[src_off:src_off + n])
    del keep
    return {
        "workload": "Poisson 20k req/s, 50/50 compress/decompress, 4 KiB-64 MiB log-uniform t4 e4m3, "
                    "8 GiB budget, 4 streams",
        "duration_s": seconds, "requests": len(reqs), "completed": len(done), "rejected": len(srv.rejected),
        "p50_ms": lat[50] * 1e3 if lat[50] is not None else None,
        "p99_ms": lat[99] * 1e3 if lat[99] is not None else None,
        "raw_gbs": raw / wall / 1e9, "offered_gbs": raw / seconds / 1e9, "wall_s": wall, "all_status_ok": ok,
        "checked_requests": len(kept),
        "checked": "every 499th completed request of at most 16 MiB (up to 24), copied aside on the device "
                   "as it completed; containers decoded back to their input, decoded bytes against the source",
        "round_trip_exact": bool(exact) if kept else None,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of oracle work for cpu_baseline (0 = skip)")
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--no-batched", action="store_true", help="skip the 1152-shard batched leg")
    ap.add_argument("--no-large", action="store_true", help="skip the 64 x 64 MiB batched leg")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving leg length (0 = skip)")
    ap.add_argument("--no-fused", action="store_true", help="skip the fused quantise / dequantise leg")
    ap.add_argument("--fused-elems", type=int, default=N_BYTES,
                    help="elements in the fused leg (fewer only for profiling captures)")
    ap.add_argument("--batched-shards", type=int, default=1152,
                    help="shards in the batched leg (fewer only for profiling captures)")
    ap.add_argument("--batched-shape", default=None,
                    help="chunk,encode_ctas_per_sm,decode_ctas_per_sm for the batched leg instead of "
                         "autotuning (profiling captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = _dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2602_17849_gb300 import _build
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    from paper_2602_17849_gb300 import inputs, qlc

    x = inputs.make_e4m3("t4", N_BYTES, seed=rank, device=dev)  # each replica codes its own tensor
    torch.cuda.empty_cache()  # drop the generator's temporaries
    codec = qlc.Codec(N_BYTES, CHUNK, SCHEME, dev)
    cont = codec.new_container()
    y = torch.empty(N_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        qlc.qlc_histogram(x, codec.hist, stream=stream)
        if ev:
            ev[1].record(stream)
        qlc.qlc_build_lut(codec.hist, SCHEME, codec.lut, stream=stream)
        if ev:
            ev[2].record(stream)
        qlc.qlc_encode(x, codec.lut, CHUNK, cont, codec.ws, codec.out_bytes, codec.status, stream=stream)
        if ev:
            ev[3].record(stream)
        qlc.qlc_decode(cont, y, codec.n_out, codec.status, stream=stream)
        if ev:
            ev[4].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    codec.check()
    c_bytes = int(codec.out_bytes.item())
    assert torch.equal(x, y), "round trip is not bit-exact"

    # per-kernel durations (events between launches, same stream)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        end.record(stream)
        torch.cuda.synchronize()
        time.sleep(0.1)
    if world > 1:
        dist.barrier()
    ms_max = max_over_ranks(start.elapsed_time(end) / args.steps, world, dev)
    codec.check()
    assert torch.equal(x, y), "round trip is not bit-exact"

    seg = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in evs])  # ms
    hist_ms, lut_ms, enc_ms, dec_ms = seg.mean(axis=0)

    # ---- e2e through the C ABI with pinned host buffers
    e2e = e2e_leg(dev, x, args.e2e_steps) if args.e2e_steps > 0 else None
    nb = c_bytes

    # ---- roofline of the dominant kernel
    peak, peak_kind = _peaks()
    r = c_bytes / N_BYTES
    kern = {"hist": (hist_ms, N_BYTES, "hist_lut.cu"), "lut": (lut_ms, 256 * 8 + 800, "hist_lut.cu"),
            "encode": (enc_ms, N_BYTES + c_bytes, "encode.cu"),
            "decode": (dec_ms, N_BYTES + c_bytes, "decode.cu")}
    dom = max(kern, key=lambda k: kern[k][0])
    d_ms, d_bytes, d_file = kern[dom]
    achieved = d_bytes / (d_ms * 1e-3) / 1e9
    traffic = _traffic_for(d_file)

    # compressibility (a6): code-only from the histogram, container from its size
    h = codec.hist.cpu().numpy().astype(np.int64)
    lut = codec.lut.cpu().numpy()
    lens = (lut[32:544].view(np.uint16) & 15).astype(np.int64)
    code_bits = int((h * lens).sum())

    line = {
        "metric": "QLC encode+decode round trip, raw GB/s", "value": replica_throughput(world, N_BYTES, ms_max),
        "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic",
        "config": _config(world),
        "kernels_ms": {"histogram": hist_ms, "build_lut": lut_ms, "encode": enc_ms, "decode": dec_ms},
        "encode_gbs": N_BYTES / ((hist_ms + lut_ms + enc_ms) * 1e-3) / 1e9,
        "encode_lut_given_gbs": N_BYTES / (enc_ms * 1e-3) / 1e9,
        "decode_gbs": N_BYTES / (dec_ms * 1e-3) / 1e9,
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                     "algorithmic_bytes": d_bytes},
        "roofline_all": {k: {"achieved": v[1] / (v[0] * 1e-3) / 1e9, "frac": v[1] / (v[0] * 1e-3) / 1e9 / peak}
                         for k, v in kern.items() if k != "lut"},
        "compressibility": {"container": 1 - r, "code_only": 1 - code_bits / (8 * N_BYTES),
                            "container_bytes": c_bytes},
        "e2e": e2e or {"value": None, "unit": "GB/s", "h2d_bytes_per_step": N_BYTES + nb,
                       "d2h_bytes_per_step": 8 + nb + N_BYTES},
        "gpu_launches": 4 * args.steps,
        "clocks": clk.summary(),
    }
    if not args.no_batched:
        shape = tuple(int(v) for v in args.batched_shape.split(",")) if args.batched_shape else None
        line["batched"] = batched_leg(dev, max(3, args.steps // 2), args.warmup, peak, args.batched_shards, shape)
    if not args.no_large:
        line["batched_large"] = large_leg(dev, max(3, args.steps // 2), args.warmup, peak)
    if not args.no_fused:
        line["fused_quantize"] = fused_leg(dev, max(3, args.steps // 2), args.warmup, peak, args.fused_elems)
    if args.serve_seconds > 0:
        line["serving"] = serve_leg(dev, args.serve_seconds)
    if rank == 0 and world == 1 and args.cpu_budget > 0:
        # the oracle on every host core (spawned workers), and on one core
        xh = x.cpu().numpy()
        cores = host_cores()
        pool = OraclePool(cores)
        b, s = pool.run(xh, budget_s=args.cpu_budget * 2 / 3)
        pool.close()
        b1, s1 = cpu_oracle_roundtrip(xh, budget_s=args.cpu_budget / 3)
        line["cpu_baseline"] = {"value": b / s / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
                                "sample": f"{b >> 20} MiB of the tensor in 16 MiB slices (wrapping around), "
                                          f"one oracle encode+decode per slice, {cores} worker processes, "
                                          f"{s:.1f} s wall",
                                "one_core": {"value": b1 / s1 / 1e9, "cores": 1,
                                             "sample": f"{b1 >> 20} MiB in consecutive 16 MiB slices, {s1:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
