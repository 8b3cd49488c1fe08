"""Continuous-batching compression service over the batched C ABI.

Requests (compress: raw e4m3 bytes -> container; decompress: container ->
bytes) arrive at any time.  The scheduler admits them in arrival order while
their device memory (output buffer and a share of workspace) fits an HBM
budget, packs every admitted request that is not yet on the GPU into one
batch (one qlc_encode_batch and one qlc_decode_batch), and launches it on a
free stream from a small pool, so batches overlap on the device.  Finished
batches (CUDA events) release their memory and complete their futures; new
arrivals are admitted as memory frees up.  LUTs, workspaces and buffers stay
resident in one device arena.

Host logic only: the device work is the library's batched kernels.  The
executor is pluggable so that the scheduling logic is testable on CPU.
"""
from __future__ import annotations

import bisect
import dataclasses
import time
from typing import Callable, Optional

ALIGN = 256


class OutOfBudget(Exception):
    pass


class Arena:
    """First-fit allocator over [0, capacity) with coalescing free blocks.

    Offsets are ALIGN-aligned.  Used both for the budget (admission) and for
    placing buffers inside one pre-allocated device tensor."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.free = [(0, self.capacity)]  # sorted (offset, size)
        self.used = 0
        self.live = {}

    @staticmethod
    def _round(n: int) -> int:
        return max(ALIGN, (int(n) + ALIGN - 1) // ALIGN * ALIGN)

    def alloc(self, n: int) -> int:
        n = self._round(n)
        for i, (off, size) in enumerate(self.free):
            if size >= n:
                if size == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, size - n)
                self.used += n
                self.live[off] = n
                return off
        raise OutOfBudget(n)

    def release(self, off: int) -> None:
        n = self.live.pop(off)
        self.used -= n
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, n))
        # coalesce with the neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)

    def fits(self, n: int) -> bool:
        n = self._round(n)
        return any(size >= n for _, size in self.free)


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                 # "compress" | "decompress"
    n_in: int                 # input bytes (raw symbols or container bytes)
    n_out: int                # output capacity needed
    in_ref: object            # executor-specific reference to the input
    arrival: float            # seconds, server clock
    out_off: Optional[int] = None
    ws_off: Optional[int] = None
    launched: Optional[float] = None
    done: Optional[float] = None
    result: object = None
    status: int = 0
    cancelled: bool = False

    @property
    def latency(self) -> Optional[float]:
        return None if self.done is None else self.done - self.arrival


class Server:
    """Continuous-batching scheduler.

    executor must provide: mem_for(req) -> bytes of device memory the request
    needs while in flight; launch(batch_reqs) -> handle; poll(handle) -> bool
    (finished?); finish(handle, reqs) -> fills req.result / req.status.
    """

    def __init__(self, executor, budget_bytes: int, max_in_flight: int = 4,
                 max_batch: int = 4096, clock: Callable[[], float] = time.perf_counter,
                 on_complete: Optional[Callable[[Request], None]] = None):
        self.ex = executor
        self.on_complete = on_complete  # sees each result before its memory is reused
        self.arena = Arena(budget_bytes)
        self.max_in_flight = max_in_flight
        self.max_batch = max_batch
        self.clock = clock
        self.pending: list[Request] = []     # arrived, not admitted
        self.admitted: list[Request] = []    # memory held, not launched
        self.in_flight: list[tuple[object, list[Request]]] = []
        self.completed: list[Request] = []
        self.rejected: list[Request] = []

    # -- requests
    def submit(self, req: Request) -> None:
        if self.ex.mem_for(req) > self.arena.capacity:
            req.status = -1               # can never fit: rejected at once
            self.rejected.append(req)
            return
        self.pending.append(req)

    def cancel(self, req: Request) -> bool:
        """Cancel a request that is not on the GPU yet; frees its memory."""
        if req in self.pending:
            self.pending.remove(req)
        elif req in self.admitted:
            self.admitted.remove(req)
            self.arena.release(req.out_off)
        else:
            return False
        req.cancelled = True
        return True

    # -- scheduling
    def _admit(self) -> None:
        while self.pending:
            req = self.pending[0]
            need = self.ex.mem_for(req)
            if not self.arena.fits(need):
                break                      # arrival order: later ones wait too
            req.out_off = self.arena.alloc(need)
            self.admitted.append(self.pending.pop(0))

    def _launch(self) -> None:
        while self.admitted and len(self.in_flight) < self.max_in_flight:
            batch = self.admitted[: self.max_batch]
            self.admitted = self.admitted[self.max_batch:]
            now = self.clock()
            for r in batch:
                r.launched = now
            self.in_flight.append((self.ex.launch(batch), batch))

    def _reap(self) -> None:
        still = []
        for handle, batch in self.in_flight:
            if self.ex.poll(handle):
                self.ex.finish(handle, batch)
                now = self.clock()
                for r in batch:
                    r.done = now
                    if self.on_complete is not None:
                        self.on_complete(r)
                    self.arena.release(r.out_off)
                    self.completed.append(r)
            else:
                still.append((handle, batch))
        self.in_flight = still

    def step(self) -> None:
        self._reap()
        self._admit()
        self._launch()

    def idle(self) -> bool:
        return not (self.pending or self.admitted or self.in_flight)

    def drain(self, timeout_s: float = 60.0) -> None:
        t0 = self.clock()
        while not self.idle():
            self.step()
            if self.clock() - t0 > timeout_s:
                raise TimeoutError("requests still in flight")


def run_poisson(server: Server, make_request, rate_hz: float, duration_s: float, seed: int,
                sleep: Callable[[float], None] = lambda s: None, young_gc_every: int = 0):
    """Drive the server with Poisson arrivals for duration_s seconds of server
    clock; make_request(i, arrival, rng) builds request i.  Returns the list
    of requests in arrival order.

    young_gc_every > 0: Python's automatic collection is off for the run and
    only the young generation is collected, every young_gc_every loop
    iterations.  A full collection walks every live request and stalled the
    loop for tens of milliseconds, which set the p99 latency; a young one
    takes well under a millisecond.  The collector is switched back on
    afterwards if it was on."""
    import gc

    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=int(rate_hz * duration_s * 1.5) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < duration_s]
    reqs = []
    gc_on = gc.isenabled()
    if young_gc_every > 0:
        gc.disable()
    try:
        t0 = server.clock()
        i = k = 0
        while i < len(arrivals) or not server.idle():
            now = server.clock() - t0
            while i < len(arrivals) and arrivals[i] <= now:
                r = make_request(i, t0 + float(arrivals[i]), rng)
                reqs.append(r)
                server.submit(r)
                i += 1
            server.step()
            k += 1
            if young_gc_every > 0 and k % young_gc_every == 0:
                gc.collect(0)
            if i < len(arrivals) and server.idle():
                sleep(max(0.0, float(arrivals[i]) - (server.clock() - t0)))
    finally:
        if young_gc_every > 0 and gc_on:
            gc.enable()
    return reqs


def percentiles(values, ps=(50, 99)):
    import numpy as np
    v = np.asarray(sorted(values), dtype=np.float64)
    if v.size == 0:
        return {p: None for p in ps}
    return {p: float(np.percentile(v, p)) for p in ps}


class CudaExecutor:
    """Runs batches with the library's batched kernels on a pool of streams.

    pool: CUDA uint8 tensor holding the request inputs (raw data for compress,
    containers for decompress); a request's in_ref is its byte offset there.
    device_arena: CUDA uint8 tensor of the budget's size; the Server's Arena
    hands out byte offsets into it.  A request's block is charged for its
    input, its output and its share of workspace (the admission budget covers
    in + out + workspace); the output sits at the block's start.  Small
    per-batch scratch (descriptors, histograms, LUTs, workspace, the status
    word and the output sizes) is allocated with the batch and freed when it
    completes.  Each stream owns two pinned host buffers: descriptors go up
    from one without a host wait, and the batch's status word and output
    sizes come back into the other, copied before the batch's completion
    event, so finishing a batch reads host memory only."""

    def __init__(self, pool, device_arena, chunk_symbols: int = 4096, schemes=(1,), n_streams: int = 4,
                 max_batch: int = 4096):
        import torch

        from . import qlc
        self.torch, self.qlc = torch, qlc
        self.pool = pool
        self.dev_arena = device_arena
        self.cs = chunk_symbols
        self.schemes = list(schemes)
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream(device=pool.device) for _ in range(n_streams)]
        self.free_streams = list(range(n_streams))
        self.base = device_arena.data_ptr()
        # per stream: descriptor rows (qlc_desc = 6 x 64-bit) and [status, sizes...] per part
        self.pin_desc = [torch.empty(max_batch * 6, dtype=torch.int64, pin_memory=True) for _ in range(n_streams)]
        self.pin_meta = [torch.empty(max_batch + 2, dtype=torch.int64, pin_memory=True) for _ in range(n_streams)]

    def out_bytes(self, req: Request) -> int:
        if req.kind == "compress":
            return self.qlc.qlc_encoded_size(req.n_in, self.cs)
        return req.n_out

    def mem_for(self, req: Request) -> int:
        q = self.qlc
        n_sym = req.n_in if req.kind == "compress" else req.n_out
        ws = q.qlc_batch_workspace_size(1, n_sym, self.cs if req.kind == "compress" else 128)
        extra = (256 * 8 + q.LUT_BYTES) if req.kind == "compress" else 0
        return _al(self.out_bytes(req)) + _al(req.n_in) + _al(ws + extra)

    def launch(self, batch):
        torch, q = self.torch, self.qlc
        if len(batch) > self.max_batch:
            raise ValueError("batch larger than the executor's max_batch")
        dev = self.pool.device
        sid = self.free_streams.pop(0)
        st = self.streams[sid]
        handle = {"stream": sid, "event": torch.cuda.Event(), "parts": []}
        pool_base = self.pool.data_ptr()
        rows_np = self.pin_desc[sid].numpy().reshape(-1, 6)
        pin_meta = self.pin_meta[sid]
        row0 = meta0 = 0
        with torch.cuda.stream(st):
            for kind in ("compress", "decompress"):
                reqs = [r for r in batch if r.kind == kind]
                if not reqs:
                    continue
                n = len(reqs)
                meta = torch.zeros(n + 1, dtype=torch.int64, device=dev)  # status word, then sizes
                status = meta[:1].view(torch.int32)[:1]
                mp = meta.data_ptr()
                if kind == "compress":
                    luts = torch.empty(n * q.LUT_BYTES, dtype=torch.uint8, device=dev)
                    hists = torch.empty(n * 256, dtype=torch.int64, device=dev)
                    lp = luts.data_ptr()
                    rows = [(pool_base + r.in_ref, r.n_in, self.base + r.out_off, self.out_bytes(r),
                             lp + i * q.LUT_BYTES, mp + 8 * (i + 1)) for i, r in enumerate(reqs)]
                    ws = torch.empty(q.qlc_batch_workspace_size(n, sum(r.n_in for r in reqs), self.cs),
                                     dtype=torch.uint8, device=dev)
                else:
                    rows = [(pool_base + r.in_ref, r.n_in, self.base + r.out_off, r.n_out, 0, mp + 8 * (i + 1))
                            for i, r in enumerate(reqs)]
                    ws = torch.empty(q.qlc_batch_workspace_size(n, sum(r.n_out for r in reqs), 128),
                                     dtype=torch.uint8, device=dev)
                rows_np[row0:row0 + n] = rows
                descs = torch.empty(n * 48, dtype=torch.uint8, device=dev)
                descs.copy_(self.pin_desc[sid][row0 * 6:(row0 + n) * 6].view(torch.uint8), non_blocking=True)
                if kind == "compress":
                    q.qlc_histogram_batch(descs, n, hists, False, ws, stream=st)
                    q.qlc_build_lut_batch(hists, n, self.schemes, luts, stream=st)
                    q.qlc_encode_batch(descs, n, self.cs, ws, status, stream=st)
                    keep = (descs, meta, luts, hists, ws)
                else:
                    q.qlc_decode_batch(descs, n, ws, status, stream=st)
                    keep = (descs, meta, ws)
                pin_meta[meta0:meta0 + n + 1].copy_(meta, non_blocking=True)
                handle["parts"].append((kind, reqs, meta0, keep))
                row0 += n
                meta0 += n + 1
            handle["event"].record(st)
        return handle

    def poll(self, handle) -> bool:
        return handle["event"].query()

    def finish(self, handle, batch) -> None:
        meta = self.pin_meta[handle["stream"]].numpy()
        for kind, reqs, m0, _keep in handle["parts"]:
            st = int(meta[m0]) & 0xFFFFFFFF
            for i, r in enumerate(reqs):
                r.status = st
                r.result = (r.out_off, int(meta[m0 + 1 + i]))   # output bytes at this arena offset
        self.free_streams.append(handle["stream"])

    def result_bytes(self, req: Request):
        """Host copy of a finished request's output (container or decoded bytes)."""
        off, nb = req.result
        return self.dev_arena[off:off + nb].cpu().numpy()


def _al(n: int) -> int:
    return (int(n) + ALIGN - 1) // ALIGN * ALIGN


class CudaWorkload:
    """Device-resident inputs for a serving run: a pool of seeded Student-t
    e4m3 data for compress requests and pre-encoded, verified containers (of
    log-uniform sizes) for decompress requests, all in one CUDA tensor."""

    def __init__(self, device, data_bytes: int, n_containers: int, min_size: int, max_size: int,
                 seed: int, chunk_symbols: int = 4096):
        import numpy as np
        import torch

        from . import inputs, qlc
        self.min_size, self.max_size, self.cs = min_size, max_size, chunk_symbols
        rng = np.random.Generator(np.random.PCG64(seed))
        data = inputs.make_e4m3("t4", data_bytes, seed=seed, device=device)
        sizes = [self.draw_size(rng) for _ in range(n_containers)]
        srcs = [int(rng.integers(0, (data_bytes - s) // 16 + 1)) * 16 for s in sizes]
        caps = [qlc.qlc_encoded_size(s, chunk_symbols) for s in sizes]
        total = data_bytes + sum(_al(c) for c in caps)
        self.pool = torch.zeros(_al(total), dtype=torch.uint8, device=device)
        self.pool[:data_bytes].copy_(data)
        del data
        self.data_bytes = data_bytes
        self.containers = []  # (offset in pool, container bytes, n, source offset)
        off = _al(data_bytes)
        for s, src, cap in zip(sizes, srcs, caps):
            codec = qlc.Codec(s, chunk_symbols, 1, device)
            codec.encode_into(self.pool[src:src + s], self.pool[off:off + cap])
            torch.cuda.synchronize()
            codec.check()
            nb = int(codec.out_bytes.item())
            back = qlc.decode(self.pool[off:off + nb])
            if not torch.equal(back, self.pool[src:src + s]):
                raise RuntimeError("pre-encoded container does not round-trip")
            self.containers.append((off, nb, s, src))
            off += _al(cap)

    def draw_size(self, rng) -> int:
        import math
        n = math.exp(rng.uniform(math.log(self.min_size), math.log(self.max_size)))
        return max(16, int(n) // 16 * 16)

    def make_request(self, i: int, arrival: float, rng) -> Request:
        if rng.random() < 0.5:
            n = self.draw_size(rng)
            off = int(rng.integers(0, (self.data_bytes - n) // 16 + 1)) * 16
            return Request(i, "compress", n, 0, off, arrival)
        off, nb, n, _src = self.containers[int(rng.integers(0, len(self.containers)))]
        return Request(i, "decompress", nb, n, off, arrival)


def serve_run(device, rate_hz: float, duration_s: float, budget_bytes: int, workload: CudaWorkload,
              seed: int, n_streams: int = 4, chunk_symbols: int = 4096, on_complete=None):
    """One Poisson serving run on the GPU; returns (requests, executor, server, wall seconds).
    on_complete(request, executor) sees each result before its memory is reused."""
    import torch
    arena_t = torch.empty(budget_bytes, dtype=torch.uint8, device=device)
    ex = CudaExecutor(workload.pool, arena_t, chunk_symbols=chunk_symbols, n_streams=n_streams)
    srv = Server(ex, budget_bytes, max_in_flight=n_streams, max_batch=ex.max_batch,
                 on_complete=(lambda r: on_complete(r, ex)) if on_complete else None)
    t0 = time.perf_counter()
    reqs = run_poisson(srv, workload.make_request, rate_hz, duration_s, seed,
                       sleep=lambda s: time.sleep(min(s, 0.0005)), young_gc_every=64)
    srv.drain()
    torch.cuda.synchronize()
    return reqs, ex, srv, time.perf_counter() - t0
