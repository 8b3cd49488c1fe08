"""Continuous-batching serving on the GPU: a Poisson stream of mixed compress
and decompress requests under an HBM budget; every result is checked against
the oracle (containers) or the original bytes (decompress), and a sample of
requests re-run alone gives byte-identical results to the same requests
served in the mix."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def test_serving_mix_equals_alone_and_oracle():
    from paper_2602_17849_gb300 import _build
    _build.build()
    from paper_2602_17849_gb300 import serve
    dev = torch.device("cuda")
    wl = serve.CudaWorkload(dev, data_bytes=64 << 20, n_containers=24, min_size=4096,
                            max_size=4 << 20, seed=3000)
    mixed = {}

    def keep(r, ex):  # results of every 13th request, copied before their memory is reused
        if r.rid % 13 == 0:
            mixed[r.rid] = ex.result_bytes(r)
    reqs, ex, srv, wall = serve.serve_run(dev, rate_hz=2000, duration_s=0.25, budget_bytes=256 << 20,
                                          workload=wl, seed=3001, on_complete=keep)
    assert len(reqs) > 200 and not srv.rejected
    assert all(r.done is not None and r.status == 0 for r in reqs)
    pool = wl.pool
    sample = [r for r in reqs if r.rid in mixed]
    assert len(sample) > 15
    for r in sample:
        got = mixed[r.rid]
        if r.kind == "compress":
            src = pool[r.in_ref:r.in_ref + r.n_in].cpu().numpy()
            assert np.array_equal(got, oracle.encode(src, scheme_id=1, chunk_symbols=4096)), r.rid
        else:
            off, nb, n, src_off = next(c for c in wl.containers if c[0] == r.in_ref)
            assert np.array_equal(got, pool[src_off:src_off + n].cpu().numpy()), r.rid
    # each sampled request alone, on a fresh server
    for r in sample[:8]:
        arena_t = torch.empty(64 << 20, dtype=torch.uint8, device=dev)
        ex1 = serve.CudaExecutor(pool, arena_t)
        got = {}
        s1 = serve.Server(ex1, 64 << 20, on_complete=lambda q: got.__setitem__(q.rid, ex1.result_bytes(q)))
        alone = serve.Request(r.rid, r.kind, r.n_in, r.n_out, r.in_ref, 0.0)
        s1.submit(alone)
        s1.drain()
        assert alone.status == 0
        assert np.array_equal(got[r.rid], mixed[r.rid]), r.rid


def test_serving_at_full_scale_sample_matches_oracle():
    """The serving workload at full scale (Poisson 20,000 requests/s, sizes
    log-uniform 4 KiB - 64 MiB, 8 GiB budget, 4 streams) for two seconds; a
    sample of the completed requests (every 331st, up to 12, any size) is
    copied aside on the device as it completes and compared byte for byte
    with the oracle's container (compress) or the source bytes (decompress)."""
    from paper_2602_17849_gb300 import _build
    _build.build()
    from paper_2602_17849_gb300 import serve
    dev = torch.device("cuda")
    wl = serve.CudaWorkload(dev, data_bytes=1 << 30, n_containers=32, min_size=4 << 10,
                            max_size=64 << 20, seed=3000)
    slot_bytes = (64 << 20) + (24 << 20)          # a 64 MiB input's worst-case container fits
    keep = torch.empty(12 * slot_bytes, dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream(device=dev)
    kept = []

    def sample(r, ex):
        if r.rid % 331 or len(kept) >= 12 or r.status != 0:
            return
        off, nb = r.result
        slot = len(kept) * slot_bytes
        with torch.cuda.stream(side):
            keep[slot:slot + nb].copy_(ex.dev_arena[off:off + nb], non_blocking=True)
        kept.append((r, slot, nb))

    reqs, ex, srv, wall = serve.serve_run(dev, rate_hz=20_000, duration_s=2.0, budget_bytes=8 << 30,
                                          workload=wl, seed=3001, on_complete=sample)
    torch.cuda.synchronize()
    assert len(reqs) > 30_000
    assert all(r.done is not None and r.status == 0 for r in reqs)
    assert len(kept) == 12
    kinds = {r.kind for r, _, _ in kept}
    assert kinds == {"compress", "decompress"}
    for r, slot, nb in kept:
        got = keep[slot:slot + nb].cpu().numpy()
        if r.kind == "compress":
            src = wl.pool[r.in_ref:r.in_ref + r.n_in].cpu().numpy()
            want = oracle.encode(src, scheme_id=1, chunk_symbols=4096)
        else:
            _off, _nb, n, src_off = next(c for c in wl.containers if c[0] == r.in_ref)
            want = wl.pool[src_off:src_off + n].cpu().numpy()
        assert np.array_equal(got, want), (r.rid, r.kind, r.n_in)
