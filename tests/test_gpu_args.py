"""Argument validation of the C ABI: misaligned or missing pointers and bad
sizes are refused on the host with QLC_ERR_ARG / QLC_ERR_CAPACITY before any
launch, and a batch descriptor with a bad pointer is reported through the
status word while the other shards are coded normally."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_17849_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qlc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2602_17849_gb300 import _build
    _build.build()
    from paper_2602_17849_gb300 import qlc as q
    return q


def _status_of(fn):
    from paper_2602_17849_gb300 import qlc as q
    try:
        fn()
    except q.QlcError as e:
        return e.status
    return q.OK


def test_host_side_argument_errors(qlc):
    n = 100_000
    x = inputs.make_e4m3("t4", n + 64, seed=1, device="cuda")
    codec = qlc.Codec(n, 1024, 1)
    cont = codec.new_container()
    qlc.qlc_histogram(x[:n], codec.hist)
    qlc.qlc_build_lut(codec.hist, 1, codec.lut)
    raw = torch.zeros(8192, dtype=torch.uint8, device="cuda")
    r0 = raw.data_ptr()                                  # 512-byte aligned; r0 + k is misaligned
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    E = qlc
    cases = {
        "histogram misaligned input": lambda: qlc.qlc_histogram(x[1:n + 1], codec.hist),
        "histogram misaligned hist": lambda: qlc.qlc_histogram(x[:n], r0 + 4),
        "lut misaligned hist": lambda: qlc.qlc_build_lut(r0 + 4, 1, codec.lut),
        "lut misaligned lut": lambda: qlc.qlc_build_lut(codec.hist, 1, r0 + 8),
        "lut invalid scheme": lambda: qlc.qlc_build_lut(codec.hist, qlc.make_scheme([8] * 8, [3] * 8), codec.lut),
        "encode misaligned input": lambda: qlc.qlc_encode(x[1:n + 1], codec.lut, 1024, cont, codec.ws,
                                                          codec.out_bytes, codec.status),
        "encode misaligned lut": lambda: qlc.qlc_encode(x[:n], r0 + 4, 1024, cont, codec.ws,
                                                        codec.out_bytes, codec.status),
        "encode misaligned out_bytes": lambda: qlc.qlc_encode(x[:n], codec.lut, 1024, cont, codec.ws,
                                                              r0 + 4, codec.status),
        "encode misaligned status": lambda: qlc.qlc_encode(x[:n], codec.lut, 1024, cont, codec.ws,
                                                           codec.out_bytes, r0 + 2),
        "encode bad chunk": lambda: qlc.qlc_encode(x[:n], codec.lut, 1000, cont, codec.ws,
                                                   codec.out_bytes, codec.status),
        "encode chunk too large": lambda: qlc.qlc_encode(x[:n], codec.lut, 8192, cont, codec.ws,
                                                         codec.out_bytes, codec.status),
        "decode misaligned n_out": lambda: qlc.qlc_decode(cont, x, r0 + 4, st),
        "decode misaligned input": lambda: qlc.qlc_decode(cont[8:], x, codec.n_out, st),
        "quantize misaligned hist": lambda: qlc.qlc_quantize_e4m3(
            torch.zeros(64, device="cuda"), raw[:64], r0 + 256, r0 + 1024 + 4, st),
        "quantize misaligned codes": lambda: qlc.qlc_quantize_e4m3(
            torch.zeros(64, device="cuda"), raw[1:65], r0 + 256, None, st),
        "dequantize misaligned scales": lambda: qlc.qlc_dequantize_e4m3(
            raw[:64], r0 + 258, torch.zeros(64, device="cuda")),
    }
    for name, fn in cases.items():
        assert _status_of(fn) == E.ERR_ARG, name
    small = torch.empty(1000, dtype=torch.uint8, device="cuda")
    assert _status_of(lambda: qlc.qlc_encode(x[:n], codec.lut, 1024, small, codec.ws, codec.out_bytes,
                                             codec.status)) == E.ERR_CAPACITY
    assert _status_of(lambda: qlc.qlc_encode(x[:n], codec.lut, 1024, cont, codec.ws[:16], codec.out_bytes,
                                             codec.status)) == E.ERR_CAPACITY
    torch.cuda.synchronize()
    assert int(codec.status.item()) == 0 and int(st.item()) == 0   # nothing was launched
    # the valid call still works after all the refusals
    qlc.qlc_encode(x[:n], codec.lut, 1024, cont, codec.ws, codec.out_bytes, codec.status)
    torch.cuda.synchronize()
    codec.check()
    want = oracle.encode(x[:n].cpu().numpy(), scheme_id=1, chunk_symbols=1024)
    assert np.array_equal(cont[: int(codec.out_bytes.item())].cpu().numpy(), want)


def test_batch_descriptor_with_misaligned_lut_is_skipped(qlc):
    """One shard's descriptor points at a misaligned LUT: the encode reports
    QLC_ERR_ARG and the other shards' containers are still byte-exact."""
    sizes = [70_000, 123_456, 5_000]
    shards = [inputs.make_e4m3("t4", s, seed=10 + i, device="cuda") for i, s in enumerate(sizes)]
    b = qlc.Batch(shards, 1024)
    d = b.enc_descs.view(torch.int64).view(-1, 6)    # qlc_desc: 6 x 8 bytes
    d[1, 4] += 4                                      # shard 1's lut pointer, off by 4 bytes
    b.status.zero_()
    b.encode()
    torch.cuda.synchronize()
    assert int(b.status.item()) == qlc.ERR_ARG
    b.status.zero_()
    for i in (0, 2):
        want = oracle.encode(shards[i].cpu().numpy(), scheme_id=1, chunk_symbols=1024)
        got = b.container(i)[: int(b.c_bytes[i].item())].cpu().numpy()
        assert np.array_equal(got, want), i
