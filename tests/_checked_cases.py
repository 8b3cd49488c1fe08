"""Small parity cases run against the checked build of the library (every
data-dependent index range-checked, QLC_CHECKED).  Run as a script in a
process whose QLC_LIBRARY names libqlc_checked.so: after every operation no
check may have failed (qlc_test_check_take() == 0), the statuses must be the
ones the oracle gives, and every byte must equal the oracle's.  Prints the
number of cases and exits 0 when all pass."""
import ctypes
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2602_17849_gb300 import inputs, qlc  # noqa: E402
from tests import _container as C  # noqa: E402

qlc.lib.qlc_test_check_take.restype = ctypes.c_uint32
cases = 0


def clean(what):
    global cases
    site = int(qlc.lib.qlc_test_check_take())
    if site:
        raise SystemExit(f"{what}: index check failed at file {site >> 16} line {site & 0xFFFF}")
    cases += 1


def round_trip(x, sid, cs):
    n = x.size
    xd = torch.from_numpy(x).cuda() if n else torch.zeros(16, dtype=torch.uint8, device="cuda")[:0]
    codec = qlc.Codec(max(n, 1), cs, sid)
    cont = codec.new_container()
    codec.encode_into(xd, cont)
    torch.cuda.synchronize()
    codec.check()
    nb = int(codec.out_bytes.item())
    y = torch.full((max(n, 1),), 0xAB, dtype=torch.uint8, device="cuda")
    codec.decode_into(cont, y, in_bytes=nb)
    torch.cuda.synchronize()
    codec.check()
    clean(f"round trip n={n} scheme={sid} chunk={cs}")
    assert np.array_equal(cont[:nb].cpu().numpy(), oracle.encode(x, scheme_id=sid, chunk_symbols=cs)), (n, cs)
    assert np.array_equal(y[:n].cpu().numpy(), x), (n, cs)


def decode_status(cont, cap):
    d = torch.from_numpy(cont).cuda() if cont.size else torch.zeros(16, dtype=torch.uint8, device="cuda")
    y = torch.zeros(max(cap, 1), dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    qlc.qlc_decode(d, y, n_out, st, in_bytes=cont.size, out_cap=cap)
    torch.cuda.synchronize()
    clean("corrupt container")
    return int(st.item()), y[:cap].cpu().numpy()


def main():
    assert os.path.basename(qlc.lib._name) == "libqlc_checked.so", qlc.lib._name
    assert int(qlc.lib.qlc_test_check_take()) == 0   # a checked build answers 0, not 0xFFFFFFFF
    # single tensors: sizes around tiles, chunks and groups, every kind, both tables
    for i, n in enumerate([0, 1, 127, 128, 4095, 4097, 32 * 128 + 1, 3 * 32 * 4096 + 77, 1 << 20]):
        for cs in (128, 1024, 4096):
            kind = ("t4", "uniform_bytes", "constant", "relu_t4")[(i + cs) % 4]
            round_trip(inputs.make_e4m3(kind, n, seed=i).numpy(), 1 + (i % 2), cs)
    # corrupt containers: statuses as the oracle's, no index check firing
    x = inputs.make_e4m3("t4", 3 * 32 * 1024 + 999, seed=9).numpy()
    cont = oracle.encode(x, chunk_symbols=1024)
    rng = np.random.Generator(np.random.PCG64(17))
    P = C.parse(cont)["payload_start"]
    positions = list(range(0, 64, 3)) + [64, 100, 319] + list(range(320, P, 7)) + \
        [int(v) for v in rng.integers(P, cont.size, 60)]
    for pos in positions:
        c = cont.copy()
        c[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        ost, oy, _ = oracle.decode(c, cap=x.size)
        gst, gy = decode_status(c, x.size)
        assert gst == ost, pos
        if ost == oracle.OK:
            assert np.array_equal(gy, oy), pos
    for cut in (0, 10, 319, P - 1, cont.size - 16, cont.size - 1):
        assert decode_status(cont[:cut], x.size)[0] == oracle.ERR_CORRUPT, cut
    # a batch of mixed shards, empty ones included
    sizes = [0, 1, 17, 128, 4095, 4097, 32 * 1024, 32 * 4096 + 5, 300_001, 65_536, 777, 16]
    kinds = [("t4", "gauss", "laplace", "relu_t4", "uniform_bytes")[i % 5] for i in range(len(sizes))]
    _, shards = inputs.make_shards(sizes, kinds, [50 + i for i in range(len(sizes))], "cuda")
    for cs in (128, 4096):
        b = qlc.Batch(shards, cs, schemes=(1, 2))
        b.encode()
        b.decode()
        torch.cuda.synchronize()
        b.check()
        clean(f"batch chunk={cs}")
        for i, s in enumerate(shards):
            assert torch.equal(b.output(i), s), i
    # block-32 quantisation with the histogram, then decode straight to fp32
    n = 40_000 + 13
    xf = inputs.make_f32("t4", n, seed=3)
    codes = torch.empty(n, dtype=torch.uint8, device="cuda")
    scales = torch.empty((n + 31) // 32, dtype=torch.float32, device="cuda")
    fc = qlc.Codec(n, 1024, 1)
    qlc.qlc_quantize_e4m3(xf.cuda(), codes, scales, fc.hist, fc.status)
    qlc.qlc_build_lut(fc.hist, 1, fc.lut)
    fcont = fc.new_container()
    fc.encode_into(codes, fcont, build_lut=False)
    torch.cuda.synchronize()
    fb = int(fc.out_bytes.item())
    yf = torch.empty(n, dtype=torch.float32, device="cuda")
    qlc.qlc_decode_dequantize(fcont, scales, yf, fc.n_out, fc.status, in_bytes=fb)
    torch.cuda.synchronize()
    fc.check()
    clean("quantise, encode, decode to fp32")
    ost, ocodes, oscales = oracle.quantize_block32(xf.numpy())
    assert ost == 0 and np.array_equal(codes.cpu().numpy(), ocodes)
    want = oracle.dequantize_block32(ocodes, oscales)
    assert np.array_equal(yf.cpu().numpy().view(np.uint32), want.view(np.uint32))
    # larger sizes: every quantiser warp steps through its input ring several
    # times before a ragged last step, and the decoder's grid is one CTA per
    # group with the block scales read four at a time
    rng2 = np.random.default_rng(23)
    n = (1 << 23) + 37
    for dt in (torch.float32, torch.bfloat16):
        xq = inputs.make_f32("t4", n, seed=5, device="cuda").to(dt)
        codes = torch.empty(n, dtype=torch.uint8, device="cuda")
        scales = torch.empty((n + 31) // 32, dtype=torch.float32, device="cuda")
        hist = torch.zeros(256, dtype=torch.int64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        qlc.qlc_quantize_e4m3(xq, codes, scales, hist, st)
        torch.cuda.synchronize()
        clean(f"quantise {dt} n={n}")
        assert int(st.item()) == 0
        assert torch.equal(hist, torch.bincount(codes.long(), minlength=256))
        blocks = np.append(rng2.choice(n // 32, 256, replace=False), n // 32)  # and the ragged last block
        xh = xq.cpu()
        xh = (oracle.bf16_to_f32(xh.view(torch.int16).numpy().view(np.uint16)) if dt == torch.bfloat16
              else xh.numpy())
        ch, sh = codes.cpu().numpy(), scales.cpu().numpy()
        for blk in blocks:
            lo, hi = 32 * int(blk), min(32 * int(blk) + 32, n)
            ost, oc, osc = oracle.quantize_block32(xh[lo:hi])
            assert ost == 0 and np.array_equal(ch[lo:hi], oc) and sh[blk].view(np.uint32) == osc[0].view(np.uint32)
    n = 48 << 20
    xf = inputs.make_f32("t4", n, seed=6, device="cuda")
    codes = torch.empty(n, dtype=torch.uint8, device="cuda")
    scales = torch.empty(n // 32, dtype=torch.float32, device="cuda")
    fc = qlc.Codec(n, 4096, 1)
    qlc.qlc_quantize_e4m3(xf, codes, scales, fc.hist, fc.status)
    qlc.qlc_build_lut(fc.hist, 1, fc.lut)
    fcont = fc.new_container()
    fc.encode_into(codes, fcont, build_lut=False)
    torch.cuda.synchronize()
    fb = int(fc.out_bytes.item())
    yf = torch.empty(n, dtype=torch.float32, device="cuda")
    qlc.qlc_decode_dequantize(fcont, scales, yf, fc.n_out, fc.status, in_bytes=fb)
    ref = torch.empty(n, dtype=torch.float32, device="cuda")
    qlc.qlc_dequantize_e4m3(codes, scales, ref)
    yc = torch.empty(n, dtype=torch.uint8, device="cuda")
    qlc.qlc_decode(fcont, yc, fc.n_out, fc.status, in_bytes=fb)
    torch.cuda.synchronize()
    fc.check()
    clean(f"quantise, encode, decode and decode to fp32, n={n}")
    assert torch.equal(yc, codes)
    assert torch.equal(yf.view(torch.int32), ref.view(torch.int32))
    print(f"checked build: {cases} cases, no index check failed")


if __name__ == "__main__":
    main()
