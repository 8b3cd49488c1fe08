"""Autotuner for the batched launch shape and chunk size.

Times candidate (chunk_symbols, encode CTAs per SM, decode warps per SM)
settings on a sample of a batch with CUDA events and keeps the fastest round
trip (histogram + LUT + encode + decode) whose container overhead stays within
a bound.  Results are cached in JSON keyed by GPU name and a size bucket.
All timed work is library kernels launched through the C ABI.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import qlc

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")

CHUNKS = (2048, 4096)
ENC_CTAS = (2, 3)
DEC_CTAS = (12, 16, 20)


def _key(total: int, n_shards: int) -> str:
    name = torch.cuda.get_device_name().replace(" ", "_")
    return f"{name}:total2^{int(math.log2(max(total, 1)))}:shards2^{int(math.log2(max(n_shards, 1)))}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _time(fn, reps: int = 3) -> float:
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune(shards, schemes=(1,), shared_lut: bool = False, max_overhead_pp: float = 0.1,
         sample_shards: int = 256, use_cache: bool = True, write_cache: bool = True):
    """Best {'chunk_symbols', 'encode_ctas_per_sm', 'decode_ctas_per_sm'} for
    this batch.  Candidates are timed on up to `sample_shards` shards spread
    over the batch; a chunk size is only eligible when the container overhead
    (bytes beyond the payload bits) stays under max_overhead_pp of the input."""
    total = sum(x.numel() for x in shards)
    key = _key(total, len(shards))
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]
    step = max(1, len(shards) // sample_shards)
    sample = shards[::step][:sample_shards]
    n_sample = sum(x.numel() for x in sample)
    best, best_ms = None, math.inf
    results = []
    for cs in CHUNKS:
        b = qlc.Batch(sample, cs, schemes=schemes, shared_lut=shared_lut)
        b.encode()
        torch.cuda.synchronize()
        b.check()
        # container bytes beyond the code bits: the index, header, LUT, padding
        lut = b.luts.view(-1, qlc.LUT_BYTES)[:, 32:544].contiguous().view(torch.int16).to(torch.int64) & 15
        h = b.hists.view(-1, 256)
        code_bits = int((h * lut).sum().item())
        overhead_pp = 100.0 * (int(b.c_bytes.sum().item()) - code_bits / 8) / max(n_sample, 1)
        if overhead_pp > max_overhead_pp:
            results.append(dict(chunk_symbols=cs, overhead_pp=overhead_pp, eligible=False))
            continue
        for ec in ENC_CTAS:
            for dc in DEC_CTAS:
                b.launch = (ec, dc)
                ms = _time(lambda: (b.encode(), b.decode()))
                results.append(dict(chunk_symbols=cs, encode_ctas_per_sm=ec, decode_ctas_per_sm=dc,
                                    ms=ms, overhead_pp=overhead_pp))
                if ms < best_ms:
                    best_ms = ms
                    best = dict(chunk_symbols=cs, encode_ctas_per_sm=ec, decode_ctas_per_sm=dc,
                                sample_ms=ms, overhead_pp=overhead_pp)
    if best is None:  # nothing met the overhead bound: the largest chunk has the least index
        best = dict(chunk_symbols=max(CHUNKS), encode_ctas_per_sm=max(ENC_CTAS),
                    decode_ctas_per_sm=max(DEC_CTAS), sample_ms=None, overhead_pp=None)
    best["candidates"] = results
    if write_cache:
        cache = _load()
        cache[key] = best
        try:
            with open(CACHE, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return best
