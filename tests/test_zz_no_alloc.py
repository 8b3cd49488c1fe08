"""qlc_encode_noalloc: encoding for callers that cannot allocate device memory.

Some callers (a plugin whose host framework owns all device memory, a request
path that must not call cudaMalloc) cannot provide the workspace qlc_encode
asks for.  qlc_encode_noalloc uses a fixed scratch array built into the
library instead.  Its containers must equal qlc_encode's byte for byte (the
codec is exact, so the tolerance is zero), also on a second call that reuses
the array after a first one.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2602_17849_gb300 import _build
    _build.build()
    from paper_2602_17849_gb300 import qlc
    L = qlc.lib
    P, sz, u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32
    L.qlc_encode_noalloc.argtypes = [P, sz, P, u32, P, sz, P, P, P]
    L.qlc_encode_noalloc.restype = ctypes.c_int
    return qlc, L


def _same_as_encode(qlc, L, x, cs):
    """Encodes x with qlc_encode (caller workspace) and with qlc_encode_noalloc
    and checks that the containers are identical."""
    n = x.numel()
    stream = torch.cuda.current_stream()
    codec = qlc.Codec(n, cs, 1)
    ref = codec.new_container()
    codec.encode_into(x, ref)                   # histogram, LUT, qlc_encode
    torch.cuda.synchronize()
    codec.check()
    ref_bytes = int(codec.out_bytes.item())

    out = torch.full((codec.cap,), 0x5A, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = L.qlc_encode_noalloc(x.data_ptr(), n, codec.lut.data_ptr(), cs, out.data_ptr(),
                              codec.cap, nb.data_ptr(), st.data_ptr(), stream.cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert int(nb.item()) == ref_bytes
    assert torch.equal(out[:ref_bytes], ref[:ref_bytes])


def test_noalloc_encode_equals_encode_on_two_calls():
    assert torch.cuda.is_available()
    qlc, L = _lib()
    from paper_2602_17849_gb300 import inputs
    for seed, n, cs in [(1, 3 * 32 * 4096 + 12345, 4096), (2, 1 << 20, 1024)]:
        _same_as_encode(qlc, L, inputs.make_e4m3("t4", n, seed=seed).cuda(), cs)


def test_noalloc_accepts_exactly_the_limit():
    """65536 groups of 32 chunks is the largest input the built-in array
    holds; at chunk 128 that is 256 MiB, and the container still equals
    qlc_encode's."""
    qlc, L = _lib()
    from paper_2602_17849_gb300 import inputs
    cs = 128
    x = inputs.make_e4m3("t4", 65536 * 32 * cs, seed=7, device="cuda")
    _same_as_encode(qlc, L, x, cs)
    del x
    torch.cuda.empty_cache()


def test_noalloc_rejects_too_many_groups():
    qlc, L = _lib()
    buf = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    lut = torch.zeros(800, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    n = (65536 + 1) * 32 * 128                      # one group over the built-in limit
    rc = L.qlc_encode_noalloc(buf.data_ptr(), n, lut.data_ptr(), 128, buf.data_ptr(), buf.numel(),
                              nb.data_ptr(), st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == qlc.ERR_CAPACITY
