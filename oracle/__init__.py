"""Plain CPU oracle for Quad Length Codes (arXiv 2602.17849) -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (``paper_2602_17849_gb300``) never imports it and shares no code with it.

This module is argument marshalling (numpy <-> ctypes) around ``qlc_oracle.c``,
which holds every step of the arithmetic; see that file's header for the
paper passages it follows and the readings it takes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qlc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, ERR_ARG, ERR_CAPACITY, ERR_CORRUPT = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile qlc_oracle.c into oracle/liboracle.so with the host gcc."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                           os.path.getmtime(os.path.join(_HERE, "qlc_oracle.h")))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.oracle_scheme.argtypes = [i32, P, P]
        L.oracle_scheme_valid.argtypes = [P, P]
        L.oracle_histogram.argtypes = [P, u64, P]
        L.oracle_rank.argtypes = [P, P, P]
        L.oracle_codeword.argtypes = [P, P, i32, P]
        L.oracle_decode_codeword.argtypes = [P, P, u32, i32]
        L.oracle_container_bound.argtypes = [u64, u32]
        L.oracle_container_bound.restype = u64
        L.oracle_encode.argtypes = [P, u64, P, P, i32, P, u32, P, u64, P]
        L.oracle_decode.argtypes = [P, u64, P, u64, P]
        L.oracle_huffman_lengths.argtypes = [P, P]
        L.oracle_entropy.argtypes = [P]
        L.oracle_entropy.restype = ctypes.c_double
        L.oracle_code_bits.argtypes = [P, P, P]
        L.oracle_code_bits.restype = u64
        L.oracle_huffman_roundtrip.argtypes = [P, u64, P]
        L.oracle_huffman_roundtrip.restype = u64
        L.oracle_e4m3_value.argtypes = [ctypes.c_uint8]
        L.oracle_e4m3_value.restype = ctypes.c_double
        L.oracle_e4m3_nearest.argtypes = [ctypes.c_float]
        L.oracle_e4m3_nearest.restype = ctypes.c_uint8
        L.oracle_quantize_block32.argtypes = [P, u64, P, P]
        L.oracle_dequantize_block32.argtypes = [P, P, u64, P]
        L.oracle_bf16_to_f32.argtypes = [P, u64, P]
        L.oracle_f32_to_bf16.argtypes = [P, u64, P]
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _u8(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8).reshape(-1))


def _hist(h) -> np.ndarray:
    h = np.ascontiguousarray(np.asarray(h, dtype=np.uint64).reshape(-1))
    assert h.size == 256
    return h


def scheme(scheme_id: int):
    """(symbols per area u16[8], suffix bits u8[8]) of Table 1 (id 1) or Table 2 (id 2)."""
    n = np.zeros(8, np.uint16)
    b = np.zeros(8, np.uint8)
    if lib().oracle_scheme(int(scheme_id), _p(n), _p(b)) != OK:
        raise ValueError(f"unknown scheme id {scheme_id}")
    return n, b


def _area(area):
    n = np.ascontiguousarray(np.asarray(area[0], dtype=np.uint16))
    b = np.ascontiguousarray(np.asarray(area[1], dtype=np.uint8))
    return n, b


def scheme_valid(area) -> bool:
    n, b = _area(area)
    return bool(lib().oracle_scheme_valid(_p(n), _p(b)))


def histogram(x) -> np.ndarray:
    x = _u8(x)
    h = np.zeros(256, np.uint64)
    lib().oracle_histogram(_p(x), x.size, _p(h))
    return h


def rank(hist):
    """(sym_of_rank, rank_of_sym): the decoder and inverse LUTs of Section 7."""
    h = _hist(hist)
    sor = np.zeros(256, np.uint8)
    ros = np.zeros(256, np.uint8)
    lib().oracle_rank(_p(h), _p(sor), _p(ros))
    return sor, ros


def codeword(area, r: int):
    """(code, length) of rank r."""
    n, b = _area(area)
    code = np.zeros(1, np.uint32)
    ln = lib().oracle_codeword(_p(n), _p(b), int(r), _p(code))
    if ln == 0:
        raise ValueError("bad rank")
    return int(code[0]), int(ln)


def decode_codeword(area, code: int, length: int) -> int:
    n, b = _area(area)
    return int(lib().oracle_decode_codeword(_p(n), _p(b), int(code), int(length)))


def container_bound(n: int, chunk_symbols: int) -> int:
    return int(lib().oracle_container_bound(int(n), int(chunk_symbols)))


def encode(x, scheme_id: int = 1, sym_of_rank=None, chunk_symbols: int = 4096,
           area=None, cap: int | None = None):
    """Container bytes of x (uint8 numpy array).

    sym_of_rank defaults to the ranking of x's own histogram.  Raises
    RuntimeError with the oracle status on failure.
    """
    x = _u8(x)
    if area is None:
        area = scheme(scheme_id)
    n_area, b_area = _area(area)
    if sym_of_rank is None:
        sym_of_rank, _ = rank(histogram(x))
    sor = _u8(sym_of_rank)
    bound = container_bound(x.size, chunk_symbols)
    if cap is None:
        cap = bound if bound > 0 else 1
    out = np.zeros(max(cap, 1), np.uint8)
    nbytes = np.zeros(1, np.uint64)
    st = lib().oracle_encode(_p(x), x.size, _p(n_area), _p(b_area), int(scheme_id), _p(sor),
                             int(chunk_symbols), _p(out), int(cap), _p(nbytes))
    if st != OK:
        raise RuntimeError(f"oracle_encode status {st}")
    return out[: int(nbytes[0])].copy()


def decode(container, cap: int | None = None):
    """(status, decoded bytes, n from the header)."""
    c = _u8(container)
    n_out = np.zeros(1, np.uint64)
    if cap is None:
        cap = int(np.frombuffer(c[8:16].tobytes(), np.uint64)[0]) if c.size >= 16 else 0
        cap = min(cap, 1 << 34)
    out = np.zeros(max(cap, 1), np.uint8)
    st = lib().oracle_decode(_p(c), c.size, _p(out), int(cap), _p(n_out))
    n = int(n_out[0])
    return int(st), out[: min(n, cap)].copy(), n


def huffman_lengths(hist) -> np.ndarray:
    h = _hist(hist)
    ln = np.zeros(256, np.uint8)
    lib().oracle_huffman_lengths(_p(h), _p(ln))
    return ln


def entropy(hist) -> float:
    return float(lib().oracle_entropy(_p(_hist(hist))))


def code_bits(hist, area) -> int:
    h = _hist(hist)
    n, b = _area(area)
    return int(lib().oracle_code_bits(_p(h), _p(n), _p(b)))


def huffman_roundtrip(x, hist=None) -> int:
    x = _u8(x)
    h = histogram(x) if hist is None else _hist(hist)
    return int(lib().oracle_huffman_roundtrip(_p(x), x.size, _p(h)))


def huffman_bits(hist) -> int:
    h = _hist(hist)
    return int((huffman_lengths(h).astype(np.uint64) * h).sum())


def e4m3_value(c: int) -> float:
    """Value of one e4m3 byte (Section 3, all-finite eXmY)."""
    return float(lib().oracle_e4m3_value(int(c)))


def e4m3_nearest(v: float) -> int:
    """Nearest e4m3 byte to the fp32 value v (ties to the even code)."""
    return int(lib().oracle_e4m3_nearest(float(v)))


def bf16_to_f32(x) -> np.ndarray:
    """uint16 bf16 bit patterns -> float32 (exact)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint16).reshape(-1))
    out = np.zeros(x.size, np.float32)
    lib().oracle_bf16_to_f32(_p(x), x.size, _p(out))
    return out


def f32_to_bf16(x) -> np.ndarray:
    """float32 -> uint16 bf16 bit patterns, round to nearest even."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1))
    out = np.zeros(x.size, np.uint16)
    lib().oracle_f32_to_bf16(_p(x), x.size, _p(out))
    return out


def quantize_block32(x):
    """(status, codes uint8[n], scales float32[ceil(n/32)]) of float32 x."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1))
    codes = np.zeros(max(x.size, 1), np.uint8)
    scales = np.zeros(max((x.size + 31) // 32, 1), np.float32)
    st = lib().oracle_quantize_block32(_p(x), x.size, _p(codes), _p(scales))
    return int(st), codes[: x.size].copy(), scales[: (x.size + 31) // 32].copy()


def dequantize_block32(codes, scales) -> np.ndarray:
    """float32 values of e4m3 codes with one scale per 32 elements."""
    c = _u8(codes)
    sc = np.ascontiguousarray(np.asarray(scales, dtype=np.float32).reshape(-1))
    assert sc.size >= (c.size + 31) // 32
    out = np.zeros(max(c.size, 1), np.float32)
    lib().oracle_dequantize_block32(_p(c), _p(sc), c.size, _p(out))
    return out[: c.size].copy()
