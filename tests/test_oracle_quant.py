"""Pins of the oracle's block-32 e4m3 quantisation (Section 3: eXmY e4m3 with
a scale per block of 32), the reference for the fused quantise / dequantise
entry points.  The oracle places |v| between two neighbouring magnitudes by
scanning all 128 and compares it with their midpoint.  It is checked against
the format's defining values, exact ties, saturation, an independent
frexp-based quantiser (the input generator's, in PyTorch), the rounding error
bound, and PyTorch's own bf16 conversion."""
import numpy as np
import torch

import oracle
from paper_2602_17849_gb300 import inputs


def test_e4m3_defining_values():
    assert oracle.e4m3_value(0x00) == 0.0
    assert oracle.e4m3_value(0x01) == 2.0 ** -9          # smallest subnormal
    assert oracle.e4m3_value(0x07) == 7 * 2.0 ** -9      # largest subnormal
    assert oracle.e4m3_value(0x08) == 2.0 ** -6          # smallest normal
    assert oracle.e4m3_value(0x38) == 1.0                # exponent 7 = bias
    assert oracle.e4m3_value(0x7F) == 480.0              # all-finite: no NaN code
    assert oracle.e4m3_value(0xFF) == -480.0
    v = oracle.e4m3_value(0x80)
    assert v == 0.0 and np.signbit(v)
    # the generator's table is a second, independent transcription
    assert [oracle.e4m3_value(c) for c in range(256)] == inputs.e4m3_values().tolist()


def test_nearest_fixes_every_grid_point():
    for c in range(256):
        assert oracle.e4m3_nearest(np.float32(oracle.e4m3_value(c))) == c


def test_nearest_ties_go_to_the_even_code_and_saturate():
    pos = [oracle.e4m3_value(c) for c in range(128)]
    for c in range(127):
        mid = np.float32((pos[c] + pos[c + 1]) / 2)       # exact in fp32
        want = c if c % 2 == 0 else c + 1
        assert oracle.e4m3_nearest(mid) == want, c
        assert oracle.e4m3_nearest(-mid) == want | 0x80
        up = np.nextafter(mid, np.float32(np.inf))
        dn = np.nextafter(mid, np.float32(0))
        assert oracle.e4m3_nearest(up) == c + 1 and oracle.e4m3_nearest(dn) == c
    for big in (480.0, 480.5, 495.9, 496.0, 1e6, 3e38):
        assert oracle.e4m3_nearest(big) == 0x7F and oracle.e4m3_nearest(-big) == 0xFF
    assert oracle.e4m3_nearest(2.0 ** -10) == 0x00        # half the smallest step: tie to 0
    assert oracle.e4m3_nearest(np.nextafter(np.float32(2.0 ** -10), np.float32(1))) == 0x01
    assert oracle.e4m3_nearest(-2.0 ** -12) == 0x80       # sign kept


def test_nearest_matches_an_independent_quantiser():
    rng = np.random.default_rng(5)
    mag = np.exp(rng.uniform(np.log(2.0 ** -14), np.log(600.0), 200_000)).astype(np.float32)
    v = mag * rng.choice(np.array([-1, 1], np.float32), mag.size)
    want = inputs._round_e4m3(torch.from_numpy(v)).numpy()
    got = np.array([oracle.e4m3_nearest(x) for x in v[:20_000]], np.uint8)
    assert np.array_equal(got, want[:20_000])
    # the whole array through the block quantiser with unit scales: blocks
    # whose absmax is 480 exactly make x / scale == x
    blocks = v.reshape(-1, 32).copy()
    blocks = np.clip(blocks, -479.0, 479.0)
    blocks[:, 0] = 480.0
    st, codes, scales = oracle.quantize_block32(blocks.reshape(-1))
    assert st == 0 and np.all(scales == 1.0)
    assert np.array_equal(codes, inputs._round_e4m3(torch.from_numpy(blocks.reshape(-1))).numpy())


def test_block32_quantise_matches_the_generator():
    g = torch.Generator().manual_seed(9)
    for n in (1, 31, 32, 33, 1000, 32 * 777 + 5):
        x = torch.randn(n, generator=g) * torch.exp(torch.randn(n, generator=g) * 3)
        x[: min(n, 64)] = 0.0                              # zero blocks (and a partial one)
        st, codes, scales = oracle.quantize_block32(x.numpy())
        assert st == 0
        assert np.array_equal(codes, inputs.quantize_block32(x).numpy()), n
        amax = np.abs(np.pad(x.numpy(), (0, (-n) % 32)).reshape(-1, 32)).max(axis=1)
        assert np.array_equal(scales == 0, amax == 0)


def test_quantise_error_bound_and_absmax():
    rng = np.random.default_rng(11)
    x = (rng.standard_t(4, 32 * 4096) * np.exp(rng.normal(0, 2, 32 * 4096))).astype(np.float32)
    st, codes, scales = oracle.quantize_block32(x)
    assert st == 0
    y = oracle.dequantize_block32(codes, scales).astype(np.float64)
    vals = np.array([oracle.e4m3_value(c) for c in range(256)])
    # nearest code: the error is at most half the gap to the neighbouring code
    grid = np.sort(np.unique(np.abs(vals)))
    s = np.repeat(scales.astype(np.float64), 32)
    a = np.abs(x.astype(np.float64)) / np.where(s > 0, s, 1)
    idx = np.clip(np.searchsorted(grid, a), 1, grid.size - 1)
    half_gap = (grid[idx] - grid[idx - 1]) / 2
    err = np.abs(y - x) / np.where(s > 0, s, 1)
    assert np.all(err <= half_gap * (1 + 1e-6) + 1e-7 * a)
    # each block's absmax element maps to +-480
    xb = x.reshape(-1, 32)
    cb = codes.reshape(-1, 32)
    am = np.argmax(np.abs(xb), axis=1)
    assert np.all(cb[np.arange(cb.shape[0]), am] & 0x7F == 0x7F)


def test_scale_underflow_gives_zero_codes():
    x = np.zeros(64, np.float32)
    x[:32] = np.float32(1e-44) * np.arange(32, dtype=np.float32)   # absmax / 480 rounds to 0
    x[32:] = np.float32(2.0 ** -140)                               # subnormal scale, ratio 512
    st, codes, scales = oracle.quantize_block32(x)
    assert st == 0 and scales[0] == 0 and np.all(codes[:32] == 0)
    assert scales[1] > 0 and np.all(codes[32:] == 0x7F)


def test_non_finite_input_is_an_argument_error():
    for bad in (np.nan, np.inf, -np.inf):
        x = np.ones(100, np.float32)
        x[70] = bad
        st, _, _ = oracle.quantize_block32(x)
        assert st == oracle.ERR_ARG


def test_dequantise_is_value_times_scale():
    codes = np.arange(256, dtype=np.uint8).repeat(2)          # 512 codes, 16 blocks
    scales = np.float32(2.0) ** np.arange(-8, 8, dtype=np.float32)
    y = oracle.dequantize_block32(codes, scales)
    vals = inputs.e4m3_values()
    want = (vals[codes] * np.repeat(scales, 32).astype(np.float64)).astype(np.float32)
    assert np.array_equal(y.view(np.uint32), want.view(np.uint32))  # powers of 2: exact


def test_bf16_conversions_match_torch():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(100_000) * np.exp(rng.normal(0, 8, 100_000))).astype(np.float32)
    # exact ties: the low 16 bits are 0x8000
    t = x.view(np.uint32).copy()
    t[:5000] = (t[:5000] & 0xFFFF0000) | 0x8000
    x = t.view(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = oracle.f32_to_bf16(x)
    assert np.array_equal(got, want)
    back = oracle.bf16_to_f32(got)
    assert np.array_equal(back, torch.from_numpy(got.view(np.int16)).view(torch.bfloat16).float().numpy())
