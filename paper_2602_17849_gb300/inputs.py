"""Seeded synthetic e4m3 inputs standing in for the paper's Gemma-2B SFT tensors.

The paper measures FFN activations of Gemma-2B during SFT, sharded over 64
TPUs, quantised to the all-finite eXmY e4m3 format with block size 32
(Section 3).  Those tensors are not available, so inputs are drawn here from
heavy-tailed distributions and quantised the same way.  This module holds the
input generators only -- no part of the codec's arithmetic -- and both the CUDA
path and the CPU oracle consume the bytes it returns.

e4m3 (eXmY, all 256 encodings finite): sign = bit 7, exponent = bits 6..3 with
bias 7, mantissa = bits 2..0.  Exponent 0 is subnormal, m * 2^-9; otherwise
(1 + m/8) * 2^(e-7).  The largest magnitude is 1.875 * 2^8 = 480.

Block-32 quantisation: per 32 consecutive elements, scale = absmax / 480 in
fp32; x / scale is rounded to the nearest e4m3 value (ties to even mantissa),
saturating at 480; the sign is kept, so -0 can occur; an all-zero block
becomes 0x00.
"""
from __future__ import annotations

import math

import numpy as np
import torch

E4M3_MAX = 480.0
BLOCK = 32

KINDS = ("t4", "gauss", "laplace", "laplace_outliers", "relu_t4", "ffn2", "uniform_bytes", "constant")


def e4m3_values() -> np.ndarray:
    """float64[256]: the value of every e4m3 (eXmY) byte."""
    v = np.zeros(256, np.float64)
    for c in range(256):
        s = -1.0 if c & 0x80 else 1.0
        e = (c >> 3) & 0xF
        m = c & 7
        mag = m * 2.0 ** -9 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
        v[c] = s * mag
    return v


def _round_e4m3(v: torch.Tensor) -> torch.Tensor:
    """uint8 codes of fp32 values |v| <= ~480, round to nearest even, saturating."""
    a = v.abs()
    _, e = torch.frexp(a)                      # a = m * 2^e, m in [0.5, 1)
    k = torch.clamp(e - 1, min=-6)             # a in [2^k, 2^(k+1)) for normals
    step = torch.ldexp(torch.ones_like(a), k - 3)
    q = torch.round(a / step) * step           # torch.round: half to even
    q = torch.clamp(q, max=E4M3_MAX)
    _, e2 = torch.frexp(q)
    normal = q >= 2.0 ** -6
    ebin = (e2 - 1).to(torch.int32)
    mant_n = torch.round((q / torch.ldexp(torch.ones_like(q), e2 - 1) - 1.0) * 8.0).to(torch.int32)
    mant_s = torch.round(q * 512.0).to(torch.int32)
    code = torch.where(normal, ((ebin + 7) << 3) | mant_n, mant_s)
    code = torch.where(q == 0, torch.zeros_like(code), code)
    sign = torch.signbit(v).to(torch.int32) << 7
    return (code | sign).to(torch.uint8)


def quantize_block32(x: torch.Tensor) -> torch.Tensor:
    """Block-32 absmax e4m3 quantisation of a 1-D fp32 tensor -> uint8 codes."""
    x = x.reshape(-1).to(torch.float32)
    n = x.numel()
    pad = (-n) % BLOCK
    if pad:
        x = torch.cat([x, torch.zeros(pad, dtype=x.dtype, device=x.device)])
    xb = x.view(-1, BLOCK)
    amax = xb.abs().amax(dim=1, keepdim=True)
    scale = amax / E4M3_MAX
    safe = torch.where(amax > 0, scale, torch.ones_like(scale))
    v = xb / safe
    codes = _round_e4m3(v)
    codes = torch.where(amax > 0, codes, torch.zeros_like(codes))
    return codes.reshape(-1)[:n].contiguous()


def _uniform_open(n: int, gen: torch.Generator, device) -> torch.Tensor:
    """fp32 uniforms in (0, 1]."""
    return 1.0 - torch.rand(n, generator=gen, device=device, dtype=torch.float32)


def _draw(kind: str, n: int, gen: torch.Generator, device) -> torch.Tensor:
    if kind == "t4":
        # Student-t with 4 degrees of freedom: Z / sqrt(V / 4), V ~ chi2(4) = -2 ln(U1 U2)
        z = torch.randn(n, generator=gen, device=device, dtype=torch.float32)
        u1 = _uniform_open(n, gen, device)
        u2 = _uniform_open(n, gen, device)
        v = -2.0 * (torch.log(u1) + torch.log(u2))
        return z * torch.sqrt(4.0 / torch.clamp(v, min=1e-30))
    if kind == "gauss":
        return torch.randn(n, generator=gen, device=device, dtype=torch.float32)
    if kind in ("laplace", "laplace_outliers"):
        # Laplace(b=1) as the difference of two unit exponentials
        e1 = -torch.log(_uniform_open(n, gen, device))
        e2 = -torch.log(_uniform_open(n, gen, device))
        x = e1 - e2
        if kind == "laplace_outliers":
            # 1% of the elements replaced by N(0, 20^2)
            mask = torch.rand(n, generator=gen, device=device) < 0.01
            out = 20.0 * torch.randn(n, generator=gen, device=device, dtype=torch.float32)
            x = torch.where(mask, out, x)
        return x
    if kind == "ffn2":
        # FFN2-activation-like input (Section 6: one symbol, zero, is far more
        # frequent than the rest): Student-t(4) activations with 18% of the
        # elements exactly zero; entropy ~6.13 bits against the paper's 6.11
        x = _draw("t4", n, gen, device)
        return torch.where(torch.rand(n, generator=gen, device=device) < 0.18, torch.zeros_like(x), x)
    if kind == "relu_t4":
        # post-nonlinearity (FFN2-like) input: ReLU of Student-t(4) activations,
        # so one symbol (zero) dominates, as Section 6 describes
        return torch.relu(_draw("t4", n, gen, device))
    raise ValueError(kind)


def make_e4m3(kind: str, n: int, seed: int, device="cpu", piece: int = 1 << 26) -> torch.Tensor:
    """n seeded synthetic e4m3 bytes (uint8 tensor on `device`).

    kinds: t4 (activations), gauss (weights), laplace (gradients),
    laplace_outliers (Laplace b=1 with 1% N(0, 20^2) outliers), ffn2 (18%
    exact zeros, FFN2-like), relu_t4 (post-ReLU, half zeros), uniform_bytes
    (incompressible), constant.
    Generated in pieces of `piece` elements (a multiple of 32) so that large
    tensors do not need large fp32 temporaries.
    """
    device = torch.device(device)
    if kind not in KINDS:
        raise ValueError(kind)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    if kind == "uniform_bytes":
        return torch.randint(0, 256, (n,), generator=gen, device=device, dtype=torch.int32).to(torch.uint8)
    if kind == "constant":
        return torch.full((n,), 113, dtype=torch.uint8, device=device)
    out = torch.empty(n, dtype=torch.uint8, device=device)
    piece = max(BLOCK, piece - piece % BLOCK)
    for s in range(0, n, piece):
        m = min(piece, n - s)
        out[s:s + m] = quantize_block32(_draw(kind, m, gen, device))
    return out


def make_f32(kind: str, n: int, seed: int, device="cpu", piece: int = 1 << 26) -> torch.Tensor:
    """The fp32 values that make_e4m3 quantises (same kinds, seeds and pieces
    of draws), for the fused quantise entry points: quantize_block32 of this
    tensor equals make_e4m3(kind, n, seed, device)."""
    device = torch.device(device)
    if kind in ("uniform_bytes", "constant") or kind not in KINDS:
        raise ValueError(kind)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.empty(n, dtype=torch.float32, device=device)
    piece = max(BLOCK, piece - piece % BLOCK)
    for s in range(0, n, piece):
        m = min(piece, n - s)
        out[s:s + m] = _draw(kind, m, gen, device)
    return out


def cfg3_shards(n_shards: int = 1152, lo: int = 64 << 10, hi: int = 16 << 20, base_seed: int = 1000):
    """Shard sizes and kinds of the batched workload: sizes log-uniform in
    [lo, hi] rounded to a multiple of 128, drawn with seed base_seed + i;
    kinds cycle activations (t4), weights (gauss), gradients (laplace)."""
    sizes, kinds, seeds = [], [], []
    cycle = ("t4", "gauss", "laplace")
    for i in range(n_shards):
        r = np.random.Generator(np.random.PCG64(base_seed + i))
        sz = math.exp(r.uniform(math.log(lo), math.log(hi)))
        sz = max(128, int(round(sz / 128.0)) * 128)
        sizes.append(sz)
        kinds.append(cycle[i % 3])
        seeds.append(base_seed + i)
    return sizes, kinds, seeds


def make_shards(sizes, kinds, seeds, device="cpu"):
    """One arena with every shard at a 16-byte aligned offset; returns
    (arena, list of shard views)."""
    offs, o = [], 0
    for n in sizes:
        offs.append(o)
        o += (n + 15) // 16 * 16
    arena = torch.zeros(max(o, 16), dtype=torch.uint8, device=device)
    views = []
    for off, n, kind, seed in zip(offs, sizes, kinds, seeds):
        v = arena[off:off + n]
        if n:
            v.copy_(make_e4m3(kind, n, seed, device=device))
        views.append(v)
    return arena, views


def cfg3_batch(device="cpu", n_shards: int = 1152):
    """The batched workload: 1152 shards, log-uniform 64 KiB - 16 MiB,
    activations / weights / gradients (Student-t, Gaussian, Laplace)."""
    sizes, kinds, seeds = cfg3_shards(n_shards)
    return make_shards(sizes, kinds, seeds, device)


def cfg4_batch(device="cpu", n_shards: int = 64, size: int = 64 << 20):
    """Batched large: 64 shards x 64 MiB of Laplace(b=1) with 1% N(0, 20^2)
    outliers, seeds 2000 + i."""
    return make_shards([size] * n_shards, ["laplace_outliers"] * n_shards,
                       [2000 + i for i in range(n_shards)], device)
