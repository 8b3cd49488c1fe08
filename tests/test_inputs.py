"""The seeded synthetic e4m3 generator: value table, rounding, saturation,
block-32 scaling, determinism and the statistics of the stand-in workloads."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_17849_gb300 import inputs


def test_e4m3_value_table():
    v = inputs.e4m3_values()
    assert np.all(np.isfinite(v))
    assert v.max() == 480.0 and v.min() == -480.0
    assert v[0x00] == 0.0 and v[0x80] == 0.0 and np.signbit(v[0x80])
    assert v[0x01] == 2.0 ** -9 and v[0x08] == 2.0 ** -6 and v[0x38] == 1.0
    pos = v[:128]
    assert np.all(np.diff(pos) > 0)                 # positive codes are monotone
    assert np.array_equal(v[128:], -pos)


def test_quantiser_hits_every_grid_point_exactly():
    v = torch.tensor(inputs.e4m3_values(), dtype=torch.float32)
    codes = inputs._round_e4m3(v)
    assert codes.tolist() == list(range(256))


def test_quantiser_rounds_half_to_even_and_saturates():
    v = inputs.e4m3_values()
    pos = v[:128]
    mids = torch.tensor((pos[:-1] + pos[1:]) / 2, dtype=torch.float32)
    codes = inputs._round_e4m3(mids).numpy().astype(int)
    lo = np.arange(127)
    want = np.where(lo % 2 == 0, lo, lo + 1)      # tie goes to the even mantissa
    assert np.array_equal(codes, want)
    assert inputs._round_e4m3(torch.tensor([490.0, 1e6, -1e6])).tolist() == [0x7F, 0x7F, 0xFF]
    assert inputs._round_e4m3(torch.tensor([2.0 ** -11, -2.0 ** -11])).tolist() == [0x00, 0x80]


def test_block32_scaling():
    x = torch.randn(32 * 50 + 7, generator=torch.Generator().manual_seed(1))
    q = inputs.quantize_block32(x).numpy()
    v = inputs.e4m3_values()[q]
    xb = x.numpy()
    for b in range(0, x.numel(), 32):
        blk = xb[b:b + 32]
        i = int(np.argmax(np.abs(blk)))
        assert abs(v[b + i]) == 480.0                         # absmax maps to 480
        assert np.all(np.sign(v[b:b + 32]) * np.sign(blk) >= 0)
    assert inputs.quantize_block32(torch.zeros(64)).tolist() == [0] * 64


def test_deterministic_by_seed():
    a = inputs.make_e4m3("t4", 10_000, seed=3)
    b = inputs.make_e4m3("t4", 10_000, seed=3)
    c = inputs.make_e4m3("t4", 10_000, seed=4)
    assert torch.equal(a, b) and not torch.equal(a, c)
    assert a.dtype == torch.uint8


@pytest.mark.parametrize("kind,lo,hi", [("t4", 6.3, 6.9), ("gauss", 6.1, 6.7), ("laplace", 6.4, 7.0),
                                        ("laplace_outliers", 6.6, 7.2), ("relu_t4", 3.0, 6.3),
                                        ("ffn2", 5.95, 6.3),
                                        ("uniform_bytes", 7.99, 8.0)])
def test_stand_in_entropies(kind, lo, hi):
    """Entropies of the stand-ins bracket the paper's 6.69 bits (FFN1, Section 4)
    and, for the post-ReLU data, lie below it as FFN2's 6.11 bits does (Section 6)."""
    x = inputs.make_e4m3(kind, 1 << 19, seed=0).numpy()
    H = oracle.entropy(oracle.histogram(x))
    assert lo <= H <= hi


def test_cfg3_shard_sizes():
    sizes, kinds, seeds = inputs.cfg3_shards()
    assert len(sizes) == 1152 and all(s % 128 == 0 for s in sizes)
    assert min(sizes) >= 64 << 10 and max(sizes) <= 16 << 20
    assert 2.5e9 < sum(sizes) < 4.5e9
    assert kinds[:3] == ["t4", "gauss", "laplace"] and seeds[0] == 1000


def test_make_f32_is_what_make_e4m3_quantises():
    for kind in ("t4", "gauss", "laplace_outliers", "ffn2"):
        x = inputs.make_f32(kind, 70_001, seed=5, piece=1 << 15)
        assert torch.equal(inputs.quantize_block32(x), inputs.make_e4m3(kind, 70_001, seed=5, piece=1 << 15))
