"""Host logic of the continuous-batching server, on CPU with a fake executor:
the arena allocator, admission by budget in arrival order, rejection,
cancellation, overlapping in-flight batches, completion, and results that do
not depend on what else is in the batch."""
import hashlib

import numpy as np
import pytest

from paper_2602_17849_gb300.serve import Arena, OutOfBudget, Request, Server, percentiles, run_poisson


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor:
    """Completes a batch `delay` seconds of fake clock after launch; the
    result of a request depends only on the request."""

    def __init__(self, clock, delay=0.002, mem_scale=1):
        self.clock = clock
        self.delay = delay
        self.mem_scale = mem_scale
        self.launches = []
        self.max_concurrent = 0
        self.live = 0

    def mem_for(self, req):
        return (req.n_in + req.n_out) * self.mem_scale

    def launch(self, batch):
        self.launches.append([r.rid for r in batch])
        self.live += 1
        self.max_concurrent = max(self.max_concurrent, self.live)
        return {"t_done": self.clock() + self.delay}

    def poll(self, h):
        return self.clock() >= h["t_done"]

    def finish(self, h, batch):
        self.live -= 1
        for r in batch:
            r.result = hashlib.sha256(f"{r.kind}:{r.in_ref}:{r.n_in}".encode()).hexdigest()


def test_arena_alloc_release_coalesce():
    a = Arena(1 << 20)
    offs = [a.alloc(1000) for _ in range(10)]
    assert len(set(offs)) == 10 and all(o % 256 == 0 for o in offs)
    assert a.used == 10 * 1024
    for o in offs[::2]:
        a.release(o)
    for o in offs[1::2]:
        a.release(o)
    assert a.used == 0 and a.free == [(0, 1 << 20)]
    big = a.alloc(1 << 20)
    with pytest.raises(OutOfBudget):
        a.alloc(1)
    a.release(big)
    assert a.fits(1 << 20)


def test_admission_budget_order_and_completion():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    srv = Server(ex, budget_bytes=1 << 20, max_in_flight=3, clock=clock)
    reqs = [Request(i, "compress" if i % 2 else "decompress", 100_000 + 1000 * i, 50_000, i, 0.0)
            for i in range(40)]
    peak = 0
    i = 0
    while i < len(reqs) or not srv.idle():
        if i < len(reqs):                          # one arrival per tick
            srv.submit(reqs[i])
            i += 1
        srv.step()
        peak = max(peak, srv.arena.used)
        assert srv.arena.used <= srv.arena.capacity
        clock.t += 0.0005
    assert len(srv.completed) == 40 and peak <= 1 << 20
    # admission is in arrival order
    launched = [rid for b in ex.launches for rid in b]
    assert launched == sorted(launched)
    assert ex.max_concurrent > 1                   # batches overlapped
    assert srv.arena.used == 0


def test_reject_too_large_and_cancel_frees():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    srv = Server(ex, budget_bytes=10_000, max_in_flight=1, clock=clock)
    huge = Request(0, "compress", 20_000, 0, 0, 0.0)
    srv.submit(huge)
    assert huge in srv.rejected and huge.status == -1
    a = Request(1, "compress", 4000, 0, 1, 0.0)
    b = Request(2, "compress", 4000, 0, 2, 0.0)
    c = Request(3, "compress", 4000, 0, 3, 0.0)
    for r in (a, b, c):
        srv.submit(r)
    srv._admit()                                   # a and b fit, c waits
    assert srv.admitted == [a, b] and srv.pending == [c]
    assert srv.cancel(b) and b.cancelled
    srv._admit()                                   # b's memory went to c
    assert srv.admitted == [a, c]
    while not srv.idle():
        srv.step()
        clock.t += 0.001
    assert {r.rid for r in srv.completed} == {1, 3}


def _run_mix(young_gc_every=0):
    """A 50 ms Poisson run at 20k requests/s on the fake executor."""
    clock = FakeClock()
    ex = FakeExecutor(clock, delay=0.001)
    srv = Server(ex, budget_bytes=4 << 20, max_in_flight=4, clock=clock)

    def make(i, arrival, rng):
        n = int(np.exp(rng.uniform(np.log(4096), np.log(1 << 20))))
        kind = "compress" if rng.random() < 0.5 else "decompress"
        return Request(i, kind, n, n // 2, int(rng.integers(0, 1 << 30)), arrival)

    def tick(_):
        clock.t += 0.0002
    orig = srv.step

    def step():
        orig()
        clock.t += 0.0001
    srv.step = step
    reqs = run_poisson(srv, make, rate_hz=20_000, duration_s=0.05, seed=3000, sleep=tick,
                       young_gc_every=young_gc_every)
    return reqs, ex


def test_continuous_batching_results_independent_of_mix():
    reqs, ex = _run_mix()
    assert len(reqs) > 500 and all(r.done is not None for r in reqs)
    assert len(ex.launches) > 1 and max(len(b) for b in ex.launches) > 1
    lat = percentiles([r.latency for r in reqs])
    assert lat[50] <= lat[99]
    # the same request alone gives the same result
    for r in reqs[::97]:
        clock = FakeClock()
        ex1 = FakeExecutor(clock)
        srv = Server(ex1, budget_bytes=4 << 20, clock=clock)
        alone = Request(r.rid, r.kind, r.n_in, r.n_out, r.in_ref, 0.0)
        srv.submit(alone)
        while not srv.idle():
            srv.step()
            clock.t += 0.001
        assert alone.result == r.result


def test_drain_times_out_when_a_batch_never_finishes():
    clock = FakeClock()
    ex = FakeExecutor(clock, delay=1e9)
    srv = Server(ex, budget_bytes=1 << 20, clock=lambda: clock())
    srv.submit(Request(0, "compress", 100, 0, 0, 0.0))

    def ticking():
        clock.t += 1.0
        return clock.t
    srv.clock = ticking
    with pytest.raises(TimeoutError):
        srv.drain(timeout_s=5.0)


def test_run_with_young_gc_only_restores_the_collector_and_changes_no_result():
    """With automatic collection off and young-generation collections only,
    the same arrivals give the same batches and results, and the collector is
    on again afterwards, with nothing frozen or unfrozen."""
    import gc
    assert gc.isenabled()
    frozen = gc.get_freeze_count()
    a, ex_a = _run_mix(0)
    b, ex_b = _run_mix(8)
    assert gc.isenabled() and gc.get_freeze_count() == frozen
    assert [r.result for r in a] == [r.result for r in b]
    assert [len(x) for x in ex_a.launches] == [len(x) for x in ex_b.launches]
