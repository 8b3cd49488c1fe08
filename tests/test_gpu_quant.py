"""GPU parity of the fused block-32 e4m3 entry points (Section 3) against the
oracle: quantisation with the histogram counted in the same pass, plain
dequantisation, and decoding straight to values.  Codes, scales, histogram
counts and every output value (compared as bit patterns) must match exactly:
the oracle takes the same fp32 decisions (scale = absmax / 480, x / scale,
value * scale) as the kernels."""
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


def _floats(n, seed):
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(n, generator=g) * torch.exp(torch.randn(n, generator=g) * 2)
    if n >= 96:
        x[:32] = 0.0                                          # an all-zero block
        x[32:64] = -0.0 * x[32:64]                            # negative zeros and values
        x[40] = -0.0
        x[64:96] = torch.tensor(1e-44) * torch.arange(32)     # scale rounds to 0
    if n >= 160:
        x[96:128] = torch.tensor(2.0 ** -140)                 # subnormal scale
        x[128:160] = torch.tensor([2.0 ** -10, -(2.0 ** -10), 7.5, 480.0] * 8)  # ties, extremes
    if n >= 256:
        # scale 1: the saturation midpoint 464 and its fp32 neighbours, 448, 480
        x[160:192] = torch.tensor([480.0, 464.0, -464.0, 463.99997, 464.00003, 448.0, -480.0, 232.0] * 4)
        # scales just above and below 2^-125, where the kernel switches to the exact division
        x[192:224] = torch.tensor([480.0 * 2.0 ** -125 * 1.0000001, 3.0 * 2.0 ** -126, -(2.0 ** -120), 0.0] * 8)
        x[224:256] = torch.tensor([480.0 * 2.0 ** -125 * 0.9999999, 464.0 * 2.0 ** -125, 2.0 ** -130, 1e-40] * 8)
    return x


def _gpu_quantize(qlc, x):
    n = x.numel()
    xd = x.cuda()
    codes = torch.empty(max(n, 16), dtype=torch.uint8, device="cuda")
    scales = torch.empty(max((n + 31) // 32, 4), dtype=torch.float32, device="cuda")
    hist = torch.zeros(256, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    qlc.qlc_quantize_e4m3(xd, codes, scales, hist, st)
    torch.cuda.synchronize()
    return (int(st.item()), codes[:n].cpu().numpy(), scales[: (n + 31) // 32].cpu().numpy(),
            hist.cpu().numpy().astype(np.uint64))


def _as_f32_host(x: torch.Tensor) -> np.ndarray:
    if x.dtype == torch.bfloat16:
        return oracle.bf16_to_f32(x.view(torch.int16).numpy().view(np.uint16))
    return x.numpy()


# (1 << 23) + 37: every warp of the resident grid takes several steps through its
# input ring, and the ragged last step follows full ones
@pytest.mark.parametrize("n", [1, 31, 32, 33, 127, 128, 129, 255, 257, 1000, 32 * 4096 + 17, 1 << 20,
                               (1 << 23) + 37])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_quantize_matches_oracle(qlc, n, dtype):
    x = _floats(n, seed=n).to(dtype)
    st, codes, scales, hist = _gpu_quantize(qlc, x)
    ost, ocodes, oscales = oracle.quantize_block32(_as_f32_host(x))
    assert st == ost == 0
    assert np.array_equal(codes, ocodes)
    assert np.array_equal(scales.view(np.uint32), oscales.view(np.uint32))
    assert np.array_equal(hist, oracle.histogram(ocodes))


def test_quantize_non_finite_is_an_argument_error(qlc):
    for bad in (float("nan"), float("inf"), float("-inf")):
        x = _floats(4096, seed=2)
        x[1234] = bad
        st, _, _, _ = _gpu_quantize(qlc, x)
        ost, _, _ = oracle.quantize_block32(x.numpy())
        assert st == ost == oracle.ERR_ARG


# (1 << 24) + 9: several 512-code warp steps per warp and a ragged last step
@pytest.mark.parametrize("n", [1, 17, 32, 1000, 32 * 4096 + 17, (1 << 24) + 9])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_dequantize_matches_oracle(qlc, n, dtype):
    rng = np.random.default_rng(n)
    codes = rng.integers(0, 256, n, dtype=np.uint8)
    scales = (rng.standard_normal((n + 31) // 32) ** 2 * 0.01).astype(np.float32)
    scales[0] = 0.0
    if scales.size > 3:
        scales[1] = 3.0e35   # values near the fp32 maximum
        scales[2] = 1e-40    # a subnormal scale: subnormal products
    out = torch.empty(max(n, 16), dtype=dtype, device="cuda")
    qlc.qlc_dequantize_e4m3(torch.from_numpy(codes).cuda(), torch.from_numpy(scales).cuda(), out, n=n)
    torch.cuda.synchronize()
    want = oracle.dequantize_block32(codes, scales)
    got = out[:n].cpu()
    if dtype == torch.bfloat16:
        assert np.array_equal(got.view(torch.int16).numpy().view(np.uint16), oracle.f32_to_bf16(want))
    else:
        assert np.array_equal(got.numpy().view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("n,cs", [(1, 128), (4097, 1024), (32 * 4096 + 333, 4096), (3 * (1 << 20) + 5, 4096)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_fused_pipeline_matches_oracle(qlc, n, cs, dtype):
    """x -> quantise + histogram -> LUT -> encode -> decode straight to values:
    the container is the oracle's container of the oracle's codes, and the
    values are the oracle's dequantised codes, bit for bit."""
    x = _floats(n, seed=100 + n).to(dtype)
    xd = x.cuda()
    codec = qlc.Codec(max(n, 1), cs, 1)
    codes = torch.empty(max(n, 16), dtype=torch.uint8, device="cuda")
    scales = torch.empty(max((n + 31) // 32, 4), dtype=torch.float32, device="cuda")
    qlc.qlc_quantize_e4m3(xd, codes, scales, codec.hist, codec.status)
    qlc.qlc_build_lut(codec.hist, 1, codec.lut)
    cont = codec.new_container()
    codec.encode_into(codes[:n], cont, build_lut=False)
    torch.cuda.synchronize()
    codec.check()
    nbytes = int(codec.out_bytes.item())
    y = torch.empty(max(n, 16), dtype=dtype, device="cuda")
    qlc.qlc_decode_dequantize(cont, scales, y, codec.n_out, codec.status, in_bytes=nbytes)
    torch.cuda.synchronize()
    codec.check()
    assert int(codec.n_out.item()) == n
    ost, ocodes, oscales = oracle.quantize_block32(_as_f32_host(x))
    assert ost == 0
    want_c = oracle.encode(ocodes, scheme_id=1, chunk_symbols=cs)
    assert np.array_equal(cont[:nbytes].cpu().numpy(), want_c)
    dst, dcodes, _ = oracle.decode(want_c)
    assert dst == 0
    want = oracle.dequantize_block32(dcodes, oscales)
    got = y[:n].cpu()
    if dtype == torch.bfloat16:
        assert np.array_equal(got.view(torch.int16).numpy().view(np.uint16), oracle.f32_to_bf16(want))
    else:
        assert np.array_equal(got.numpy().view(np.uint32), want.view(np.uint32))


def test_decode_dequantize_corrupt_and_capacity(qlc):
    x = inputs.make_e4m3("t4", 50_000, seed=4)
    c = oracle.encode(x.numpy(), scheme_id=1, chunk_symbols=1024)
    scales = torch.ones(2000, dtype=torch.float32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    small = torch.empty(49_999, dtype=torch.float32, device="cuda")
    qlc.qlc_decode_dequantize(torch.from_numpy(c).cuda(), scales, small, n_out, st)
    torch.cuda.synchronize()
    assert int(st.item()) == qlc.ERR_CAPACITY and int(n_out.item()) == 50_000
    bad = c.copy()
    bad[400] ^= 0x5A                                      # chunk_bits[0]
    st.zero_()
    y = torch.empty(50_000, dtype=torch.float32, device="cuda")
    qlc.qlc_decode_dequantize(torch.from_numpy(bad).cuda(), scales, y, n_out, st)
    torch.cuda.synchronize()
    ost, _, _ = oracle.decode(bad)
    assert int(st.item()) == ost == oracle.ERR_CORRUPT


def test_full_size_fused_sampled(qlc):
    """64 Mi fp32 elements (256 MiB): the device histogram equals the oracle's
    histogram of the device codes; 2048 sampled blocks match the oracle's
    quantisation; decoding straight to values equals plain dequantisation of
    the codes, and sampled values match the oracle."""
    n = 64 << 20
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(n, generator=g, device="cuda") * torch.exp(torch.randn(n, generator=g, device="cuda"))
    codes = torch.empty(n, dtype=torch.uint8, device="cuda")
    scales = torch.empty(n // 32, dtype=torch.float32, device="cuda")
    codec = qlc.Codec(n, 4096, 1)
    qlc.qlc_quantize_e4m3(x, codes, scales, codec.hist, codec.status)
    qlc.qlc_build_lut(codec.hist, 1, codec.lut)
    cont = codec.new_container()
    codec.encode_into(codes, cont, build_lut=False)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    qlc.qlc_decode_dequantize(cont, scales, y, codec.n_out, codec.status, in_bytes=None)
    ref = torch.empty(n, dtype=torch.float32, device="cuda")
    qlc.qlc_dequantize_e4m3(codes, scales, ref)
    torch.cuda.synchronize()
    codec.check()
    assert torch.equal(y.view(torch.int32), ref.view(torch.int32))
    ch = codes.cpu().numpy()
    assert np.array_equal(codec.hist.cpu().numpy().astype(np.uint64), oracle.histogram(ch))
    rng = np.random.default_rng(8)
    blocks = rng.choice(n // 32, 2048, replace=False)
    xs = x.view(-1, 32)[torch.from_numpy(blocks).cuda()].cpu().numpy().reshape(-1)
    ost, oc, osc = oracle.quantize_block32(xs)
    assert ost == 0
    assert np.array_equal(ch.reshape(-1, 32)[blocks].reshape(-1), oc)
    assert np.array_equal(scales.cpu().numpy()[blocks].view(np.uint32), osc.view(np.uint32))
    want = oracle.dequantize_block32(oc, osc)
    got = y.view(-1, 32)[torch.from_numpy(blocks).cuda()].cpu().numpy().reshape(-1)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def _near_midpoint_blocks(n_blocks, seed, lo=-80.0, hi=80.0):
    """Blocks whose quotients x / scale sit on, or within 4 ulps of, the
    midpoints between neighbouring e4m3 magnitudes (where rounding x / scale
    and rounding a nearby value can differ).  Element 0 of a block is its
    absmax, which fixes the block's scale; scales are log-uniform over
    [2^lo, 2^hi]."""
    rng = np.random.default_rng(seed)
    mags = np.array([oracle.e4m3_value(c) for c in range(0x80)], np.float64)
    mids = (mags[:-1] + mags[1:]) / 2
    x = np.zeros((n_blocks, 32), np.float32)
    for b in range(n_blocks):
        amax = np.float32(480.0 * 2.0 ** rng.uniform(lo, hi))
        scale = np.float32(amax / np.float32(480.0))
        m = mids[rng.integers(len(mids), size=31)]
        v = (m * np.float64(scale)).astype(np.float32)
        v = (v.view(np.int32) + rng.integers(-4, 5, size=31).astype(np.int32)).view(np.float32)
        v = np.minimum(np.abs(v), amax) * np.where(rng.random(31) < 0.5, -1, 1).astype(np.float32)
        x[b, 0] = amax * (1 if rng.random() < 0.5 else -1)
        x[b, 1:] = v
    return x.reshape(-1)


@pytest.mark.parametrize("lo,hi", [(-80.0, 80.0), (-125.5, -124.5), (-130.0, -120.0)])
def test_quantize_near_midpoints(qlc, lo, hi):
    """Quotients on and next to the rounding midpoints (and scales around the
    2^-125 limit of the reciprocal) quantise exactly as the oracle does."""
    x = _near_midpoint_blocks(4096, seed=int(lo * 10) & 0xFFFF, lo=lo, hi=hi)
    st, codes, scales, hist = _gpu_quantize(qlc, torch.from_numpy(x))
    ost, ocodes, oscales = oracle.quantize_block32(x)
    assert st == ost == 0
    assert np.array_equal(scales.view(np.uint32), oscales.view(np.uint32))
    assert np.array_equal(codes, ocodes)
    assert np.array_equal(hist, oracle.histogram(ocodes))


def test_scale_for_every_mantissa(qlc):
    """Block scales against numpy's float32 division for every mantissa of
    amax in [1, 2), and for amax in the binades where the kernel switches
    between its corrected product and the division (2^-101, 2^-100) and at
    the top of the float range."""
    m = 1 << 23
    a = (np.arange(m, dtype=np.uint32) | np.uint32(0x3F800000)).view(np.float32)
    rng = np.random.default_rng(5)
    edge = np.concatenate([
        (rng.integers(0, m, 4096, dtype=np.uint32) | np.uint32(26 << 23)).view(np.float32),   # 2^-101
        (rng.integers(0, m, 4096, dtype=np.uint32) | np.uint32(27 << 23)).view(np.float32),   # 2^-100
        (rng.integers(0, m, 4096, dtype=np.uint32) | np.uint32(254 << 23)).view(np.float32),  # 2^127
        np.array([np.float32(2.0 ** -100), np.nextafter(np.float32(2.0 ** -100), np.float32(0)),
                  np.finfo(np.float32).max, np.float32(1e-45)], dtype=np.float32)])
    amax = np.concatenate([a, edge])
    x = torch.zeros(amax.size, 32, dtype=torch.float32, device="cuda")
    am = torch.from_numpy(amax).cuda()
    x[:, 0] = am
    x[:, 7] = -am * 0.25
    x = x.reshape(-1)
    n = x.numel()
    codes = torch.empty(n, dtype=torch.uint8, device="cuda")
    scales = torch.empty(n // 32, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    qlc.qlc_quantize_e4m3(x, codes, scales, None, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    want = amax / np.float32(480.0)
    assert np.array_equal(scales.cpu().numpy().view(np.uint32), want.view(np.uint32))
