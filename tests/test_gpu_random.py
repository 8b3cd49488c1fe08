"""Randomised GPU parity against the oracle (fixed seed, fixed case count):
sizes log-uniform from 0 to 3 Mi symbols, every input kind, Table 1, Table 2
and searched schemes, every chunk size 128..4096; each container byte-exact
and each decode of the oracle's container exact; plus random batches with
empty shards and per-shard scheme choice."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_17849_gb300 import inputs

pytestmark = pytest.mark.gpu

KINDS = ["t4", "gauss", "laplace", "laplace_outliers", "relu_t4", "ffn2", "uniform_bytes", "constant"]


@pytest.fixture(scope="module")
def qlc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2602_17849_gb300 import _build
    _build.build()
    from paper_2602_17849_gb300 import qlc as q
    return q


def test_random_tensors_match_oracle(qlc):
    rng = np.random.default_rng(20260217)
    for case in range(400):
        n = int(np.exp(rng.uniform(0, np.log(3e6)))) if rng.random() < 0.95 else int(rng.integers(0, 40))
        kind = KINDS[rng.integers(len(KINDS))]
        cs = 128 * int(rng.integers(1, 33))
        x = inputs.make_e4m3(kind, n, seed=int(rng.integers(1 << 30))).numpy() if n else np.zeros(0, np.uint8)
        r = rng.random()
        if r < 0.4:
            sid, area = 1, oracle.scheme(1)
        elif r < 0.7:
            sid, area = 2, oracle.scheme(2)
        else:
            sc, _ = qlc.qlc_scheme_search(oracle.histogram(x))
            sid, area = sc.id, (np.array(sc.area_n[:], np.uint16), np.array(sc.area_bits[:], np.uint8))
        want = oracle.encode(x, scheme_id=sid, chunk_symbols=cs, area=area)
        xd = torch.from_numpy(x).cuda() if n else torch.zeros(16, dtype=torch.uint8, device="cuda")[:0]
        codec = qlc.Codec(max(n, 1), cs, qlc.make_scheme(area[0], area[1], sid))
        cont = codec.new_container()
        codec.encode_into(xd, cont)
        torch.cuda.synchronize()
        codec.check()
        got = cont[: int(codec.out_bytes.item())].cpu().numpy()
        assert np.array_equal(got, want), (case, n, kind, cs, sid)
        y = torch.empty(max(n, 16), dtype=torch.uint8, device="cuda")
        codec.decode_into(torch.from_numpy(want).cuda(), y, in_bytes=want.size)
        torch.cuda.synchronize()
        codec.check()
        assert np.array_equal(y[:n].cpu().numpy(), x), (case, n, kind, cs, sid)


def test_random_batches_match_oracle(qlc):
    rng = np.random.default_rng(31)
    for case in range(12):
        k = int(rng.integers(1, 40))
        sizes = [int(np.exp(rng.uniform(0, np.log(1e6)))) if rng.random() < 0.9 else 0 for _ in range(k)]
        shards = [inputs.make_e4m3(KINDS[rng.integers(6)], s, seed=int(rng.integers(1 << 30)), device="cuda")
                  if s else torch.zeros(16, dtype=torch.uint8, device="cuda")[:0] for s in sizes]
        cs = 128 * int(rng.integers(1, 33))
        b = qlc.Batch(shards, cs, schemes=(1, 2))
        b.encode()
        b.decode()
        torch.cuda.synchronize()
        b.check()
        for i, s in enumerate(shards):
            assert torch.equal(b.output(i), s), (case, i, sizes[i], cs)
            sid = int(b.luts.view(-1, qlc.LUT_BYTES)[i, 24].item())   # scheme id chosen for shard i
            want = oracle.encode(s.cpu().numpy(), scheme_id=sid, chunk_symbols=cs)
            assert np.array_equal(b.container(i)[: int(b.c_bytes[i].item())].cpu().numpy(), want), (case, i)
