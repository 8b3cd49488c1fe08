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
