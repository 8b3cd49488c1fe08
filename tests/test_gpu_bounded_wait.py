"""The encoder's look-back waits are bounded: a wait for a value nobody
writes gives up after about a second, reports QLC_ERR_TIMEOUT through the
status word, and leaves the GPU usable (no fault, no hang)."""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def test_stalled_lookback_times_out_and_gpu_stays_usable():
    from paper_2602_17849_gb300 import _build, inputs
    _build.build()
    from paper_2602_17849_gb300 import qlc
    L = qlc.lib
    P, sz, u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32
    L.qlc_test_encode_stalled_lookback.argtypes = [P, sz, P, u32, P, sz, P, sz, P, P, P]
    L.qlc_test_encode_stalled_lookback.restype = ctypes.c_int
    n, cs = 5 * 32 * 1024, 1024
    x = inputs.make_e4m3("t4", n, seed=4).cuda()
    codec = qlc.Codec(n, cs, 1)
    qlc.qlc_histogram(x, codec.hist)
    qlc.qlc_build_lut(codec.hist, 1, codec.lut)
    out = codec.new_container()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = L.qlc_test_encode_stalled_lookback(x.data_ptr(), n, codec.lut.data_ptr(), cs, out.data_ptr(),
                                            out.numel(), codec.ws.data_ptr(), codec.ws.numel(),
                                            codec.out_bytes.data_ptr(), codec.status.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(codec.status.item()) == qlc.ERR_TIMEOUT
    assert 0.5 < dt < 30.0
    # the context is still usable: a normal encode works and matches the oracle
    codec.status.zero_()
    codec.encode_into(x, out)
    torch.cuda.synchronize()
    codec.check()
    nb = int(codec.out_bytes.item())
    assert np.array_equal(out[:nb].cpu().numpy(), oracle.encode(x.cpu().numpy(), chunk_symbols=cs))
