"""Python binding of libqlc (include/qlc.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name and takes
PyTorch tensors for device buffers (uint8 / int64 views of device memory) and
the current CUDA stream.  All compute runs in the library's CUDA kernels; if
libqlc.so is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

OK, ERR_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_TIMEOUT, ERR_CUDA, ERR_CHECK = range(7)
CHUNKS_PER_GROUP = 32
HEADER_BYTES = 64
INDEX_OFFSET = 320
LUT_BYTES = 800
SCHEME_BYTES = 32


class QlcError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class qlc_scheme(ctypes.Structure):
    _fields_ = [("area_n", ctypes.c_uint16 * 8), ("area_bits", ctypes.c_uint8 * 8),
                ("id", ctypes.c_uint8), ("reserved", ctypes.c_uint8 * 7)]


class qlc_lut(ctypes.Structure):
    _fields_ = [("scheme", qlc_scheme), ("enc", ctypes.c_uint16 * 256), ("dec", ctypes.c_uint8 * 256)]


class qlc_desc(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("in_bytes", ctypes.c_uint64), ("out", ctypes.c_void_p),
                ("out_cap", ctypes.c_uint64), ("lut", ctypes.c_void_p), ("out_bytes", ctypes.c_void_p)]


class qlc_launch(ctypes.Structure):
    _fields_ = [("encode_ctas_per_sm", ctypes.c_uint16), ("decode_ctas_per_sm", ctypes.c_uint16),
                ("reserved", ctypes.c_uint32)]


assert ctypes.sizeof(qlc_scheme) == SCHEME_BYTES and ctypes.sizeof(qlc_lut) == LUT_BYTES
assert ctypes.sizeof(qlc_desc) == 48 and ctypes.sizeof(qlc_launch) == 8


def _load() -> ctypes.CDLL:
    # QLC_LIBRARY names another build of the same library (the tests' checked build)
    path = os.environ.get("QLC_LIBRARY", _build.LIB)
    if not os.path.exists(path):
        raise ImportError(f"libqlc is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, sz, u32, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_int
    L.qlc_version.restype = i32
    L.qlc_status_string.argtypes = [i32]
    L.qlc_status_string.restype = ctypes.c_char_p
    L.qlc_scheme_table.argtypes = [i32, P]
    L.qlc_scheme_check.argtypes = [P]
    L.qlc_histogram.argtypes = [P, sz, P, i32, P]
    L.qlc_build_lut.argtypes = [P, P, P, P]
    L.qlc_build_lut_host.argtypes = [P, P, P]
    L.qlc_build_lut_best.argtypes = [P, P, i32, P, P]
    L.qlc_encoded_size.argtypes = [sz, u32]
    L.qlc_encoded_size.restype = sz
    L.qlc_encode_workspace_size.argtypes = [sz, u32]
    L.qlc_encode_workspace_size.restype = sz
    L.qlc_encode.argtypes = [P, sz, P, u32, P, sz, P, sz, P, P, P]
    L.qlc_decode.argtypes = [P, sz, P, sz, P, P, P]
    L.qlc_peek_header.argtypes = [P, sz, P, P]
    L.qlc_scheme_search.argtypes = [P, P, P]
    L.qlc_scheme_search.restype = i32
    u64 = ctypes.c_uint64
    L.qlc_encode_noalloc.argtypes = [P, sz, P, u32, P, sz, P, P, P]
    L.qlc_batch_workspace_size.argtypes = [i32, u64, u32]
    L.qlc_batch_workspace_size.restype = sz
    L.qlc_histogram_batch.argtypes = [P, i32, P, i32, P, sz, P]
    L.qlc_build_lut_batch.argtypes = [P, i32, P, i32, P, P]
    L.qlc_encode_batch.argtypes = [P, i32, u32, P, sz, P, P, P]
    L.qlc_decode_batch.argtypes = [P, i32, P, sz, P, P, P]
    L.qlc_quantize_e4m3.argtypes = [P, i32, sz, P, P, P, i32, P, P]
    L.qlc_dequantize_e4m3.argtypes = [P, P, sz, P, i32, P]
    L.qlc_decode_dequantize.argtypes = [P, sz, P, P, i32, sz, P, P, P]
    for f in ("qlc_scheme_table", "qlc_histogram", "qlc_build_lut", "qlc_build_lut_host",
              "qlc_build_lut_best", "qlc_encode", "qlc_decode", "qlc_peek_header", "qlc_encode_noalloc",
              "qlc_histogram_batch", "qlc_build_lut_batch", "qlc_encode_batch", "qlc_decode_batch",
              "qlc_quantize_e4m3", "qlc_dequantize_e4m3", "qlc_decode_dequantize"):
        getattr(L, f).restype = i32
    return L


lib = _load()


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


def _check(st: int, what: str):
    if st != OK:
        raise QlcError(st, what)


def _nbytes(t: torch.Tensor) -> int:
    return t.numel() * t.element_size()


# ----------------------------------------------------------------- C ABI names

def qlc_version() -> int:
    return int(lib.qlc_version())


def status_string(st: int) -> str:
    return lib.qlc_status_string(int(st)).decode()


qlc_status_string = status_string


def qlc_scheme_table(scheme_id: int) -> qlc_scheme:
    s = qlc_scheme()
    _check(lib.qlc_scheme_table(int(scheme_id), ctypes.byref(s)), "qlc_scheme_table")
    return s


def make_scheme(area_n, area_bits, scheme_id: int = 0) -> qlc_scheme:
    s = qlc_scheme()
    for i in range(8):
        s.area_n[i] = int(area_n[i])
        s.area_bits[i] = int(area_bits[i])
    s.id = int(scheme_id)
    return s


def as_scheme(scheme) -> qlc_scheme:
    if isinstance(scheme, qlc_scheme):
        return scheme
    if isinstance(scheme, int):
        return qlc_scheme_table(scheme)
    n, b = scheme[0], scheme[1]
    return make_scheme(n, b, scheme[2] if len(scheme) > 2 else 0)


def qlc_scheme_check(scheme) -> bool:
    s = as_scheme(scheme)
    return bool(lib.qlc_scheme_check(ctypes.byref(s)))


def qlc_histogram(d_in: torch.Tensor, d_hist: torch.Tensor, accumulate: bool = False,
                  n: int | None = None, stream=None) -> torch.Tensor:
    """d_in: CUDA uint8; d_hist: CUDA int64[256] (uint64 counts)."""
    n = _nbytes(d_in) if n is None else n
    _check(lib.qlc_histogram(_ptr(d_in), n, _ptr(d_hist), int(bool(accumulate)), _stream(stream)),
           "qlc_histogram")
    return d_hist


def qlc_build_lut(d_hist: torch.Tensor, scheme, d_lut: torch.Tensor, stream=None) -> torch.Tensor:
    """d_lut: CUDA uint8[800] receiving a qlc_lut."""
    s = as_scheme(scheme)
    _check(lib.qlc_build_lut(_ptr(d_hist), ctypes.byref(s), _ptr(d_lut), _stream(stream)),
           "qlc_build_lut")
    return d_lut


def qlc_build_lut_best(d_hist: torch.Tensor, schemes, d_lut: torch.Tensor, stream=None) -> torch.Tensor:
    arr = (qlc_scheme * len(schemes))(*[as_scheme(s) for s in schemes])
    _check(lib.qlc_build_lut_best(_ptr(d_hist), arr, len(schemes), _ptr(d_lut), _stream(stream)),
           "qlc_build_lut_best")
    return d_lut


def qlc_build_lut_host(hist, scheme) -> qlc_lut:
    h = (ctypes.c_uint64 * 256)(*[int(v) for v in hist])
    s = as_scheme(scheme)
    out = qlc_lut()
    _check(lib.qlc_build_lut_host(h, ctypes.byref(s), ctypes.byref(out)), "qlc_build_lut_host")
    return out


def qlc_scheme_search(hist):
    """(best qlc_scheme of the family for this histogram, its payload bits)."""
    h = (ctypes.c_uint64 * 256)(*[int(v) for v in hist])
    out = qlc_scheme()
    bits = ctypes.c_uint64()
    _check(lib.qlc_scheme_search(h, ctypes.byref(out), ctypes.byref(bits)), "qlc_scheme_search")
    return out, int(bits.value)


def qlc_encoded_size(n: int, chunk_symbols: int = 4096) -> int:
    return int(lib.qlc_encoded_size(int(n), int(chunk_symbols)))


def qlc_encode_workspace_size(n: int, chunk_symbols: int = 4096) -> int:
    return int(lib.qlc_encode_workspace_size(int(n), int(chunk_symbols)))


def qlc_encode(d_in: torch.Tensor, d_lut: torch.Tensor, chunk_symbols: int, d_out: torch.Tensor,
               d_ws: torch.Tensor, d_out_bytes: torch.Tensor, d_status: torch.Tensor,
               n: int | None = None, stream=None) -> None:
    n = _nbytes(d_in) if n is None else n
    _check(lib.qlc_encode(_ptr(d_in), n, _ptr(d_lut), int(chunk_symbols), _ptr(d_out), _nbytes(d_out),
                          _ptr(d_ws), _nbytes(d_ws) if d_ws is not None else 0, _ptr(d_out_bytes),
                          _ptr(d_status), _stream(stream)), "qlc_encode")


def qlc_decode(d_in: torch.Tensor, d_out: torch.Tensor, d_n_out: torch.Tensor, d_status: torch.Tensor,
               in_bytes: int | None = None, out_cap: int | None = None, stream=None) -> None:
    in_bytes = _nbytes(d_in) if in_bytes is None else in_bytes
    out_cap = _nbytes(d_out) if out_cap is None else out_cap
    _check(lib.qlc_decode(_ptr(d_in), in_bytes, _ptr(d_out), out_cap, _ptr(d_n_out), _ptr(d_status),
                          _stream(stream)), "qlc_decode")


DTYPE_F32, DTYPE_BF16 = 0, 1


def _dtype_of(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return DTYPE_F32
    if t.dtype == torch.bfloat16:
        return DTYPE_BF16
    raise QlcError(ERR_ARG, f"dtype {t.dtype} (float32 or bfloat16)")


def qlc_quantize_e4m3(d_x: torch.Tensor, d_codes: torch.Tensor, d_scales: torch.Tensor,
                      d_hist: torch.Tensor | None, d_status: torch.Tensor, accumulate: bool = False,
                      n: int | None = None, stream=None) -> None:
    """d_x: CUDA float32 or bfloat16; d_codes: uint8[n]; d_scales: float32[ceil(n/32)];
    d_hist: int64[256] or None."""
    n = d_x.numel() if n is None else n
    _check(lib.qlc_quantize_e4m3(_ptr(d_x), _dtype_of(d_x), n, _ptr(d_codes), _ptr(d_scales),
                                 _ptr(d_hist) if d_hist is not None else None, int(bool(accumulate)),
                                 _ptr(d_status), _stream(stream)), "qlc_quantize_e4m3")


def qlc_dequantize_e4m3(d_codes: torch.Tensor, d_scales: torch.Tensor, d_out: torch.Tensor,
                        n: int | None = None, stream=None) -> None:
    """d_out: CUDA float32 or bfloat16 with at least n elements."""
    n = d_codes.numel() if n is None else n
    _check(lib.qlc_dequantize_e4m3(_ptr(d_codes), _ptr(d_scales), n, _ptr(d_out), _dtype_of(d_out),
                                   _stream(stream)), "qlc_dequantize_e4m3")


def qlc_decode_dequantize(d_in: torch.Tensor, d_scales: torch.Tensor, d_out: torch.Tensor,
                          d_n_out: torch.Tensor, d_status: torch.Tensor, in_bytes: int | None = None,
                          stream=None) -> None:
    """Decode a container straight to float32 / bfloat16 values (d_out's dtype)."""
    in_bytes = _nbytes(d_in) if in_bytes is None else in_bytes
    _check(lib.qlc_decode_dequantize(_ptr(d_in), in_bytes, _ptr(d_scales), _ptr(d_out), _dtype_of(d_out),
                                     d_out.numel(), _ptr(d_n_out), _ptr(d_status), _stream(stream)),
           "qlc_decode_dequantize")


def qlc_peek_header(hdr: bytes):
    buf = ctypes.create_string_buffer(bytes(hdr), len(hdr))
    n = ctypes.c_uint64()
    c = ctypes.c_uint64()
    _check(lib.qlc_peek_header(buf, len(hdr), ctypes.byref(n), ctypes.byref(c)), "qlc_peek_header")
    return int(n.value), int(c.value)


def qlc_encode_noalloc(d_in: torch.Tensor, d_lut: torch.Tensor, chunk_symbols: int, d_out: torch.Tensor,
                       d_out_bytes: torch.Tensor, d_status: torch.Tensor, n: int | None = None,
                       stream=None) -> None:
    n = _nbytes(d_in) if n is None else n
    _check(lib.qlc_encode_noalloc(_ptr(d_in), n, _ptr(d_lut), int(chunk_symbols), _ptr(d_out),
                                  _nbytes(d_out), _ptr(d_out_bytes), _ptr(d_status), _stream(stream)),
           "qlc_encode_noalloc")


def qlc_batch_workspace_size(n_shards: int, total_symbols: int, chunk_symbols: int = 4096) -> int:
    return int(lib.qlc_batch_workspace_size(int(n_shards), int(total_symbols), int(chunk_symbols)))


def _launch(launch):
    if launch is None:
        return None
    if isinstance(launch, qlc_launch):
        return ctypes.byref(launch)
    e, d = launch
    return ctypes.byref(qlc_launch(int(e), int(d), 0))


def qlc_histogram_batch(d_descs: torch.Tensor, n_shards: int, d_hists: torch.Tensor, shared: bool,
                        d_ws: torch.Tensor, stream=None) -> None:
    _check(lib.qlc_histogram_batch(_ptr(d_descs), int(n_shards), _ptr(d_hists), int(bool(shared)),
                                   _ptr(d_ws), _nbytes(d_ws), _stream(stream)), "qlc_histogram_batch")


def qlc_build_lut_batch(d_hists: torch.Tensor, n_luts: int, schemes, d_luts: torch.Tensor,
                        stream=None) -> None:
    schemes = schemes if isinstance(schemes, (list, tuple)) else [schemes]
    arr = (qlc_scheme * len(schemes))(*[as_scheme(x) for x in schemes])
    _check(lib.qlc_build_lut_batch(_ptr(d_hists), int(n_luts), arr, len(schemes), _ptr(d_luts),
                                   _stream(stream)), "qlc_build_lut_batch")


def qlc_encode_batch(d_descs: torch.Tensor, n_shards: int, chunk_symbols: int, d_ws: torch.Tensor,
                     d_status: torch.Tensor, launch=None, stream=None) -> None:
    _check(lib.qlc_encode_batch(_ptr(d_descs), int(n_shards), int(chunk_symbols), _ptr(d_ws), _nbytes(d_ws),
                                _ptr(d_status), _launch(launch), _stream(stream)), "qlc_encode_batch")


def qlc_decode_batch(d_descs: torch.Tensor, n_shards: int, d_ws: torch.Tensor, d_status: torch.Tensor,
                     launch=None, stream=None) -> None:
    _check(lib.qlc_decode_batch(_ptr(d_descs), int(n_shards), _ptr(d_ws), _nbytes(d_ws), _ptr(d_status),
                                _launch(launch), _stream(stream)), "qlc_decode_batch")


def descs_tensor(rows, device) -> torch.Tensor:
    """Device array of qlc_desc from (in, in_bytes, out, out_cap, lut, out_bytes) tuples of ints."""
    arr = (qlc_desc * len(rows))(*[qlc_desc(*[int(v) for v in r]) for r in rows])
    host = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
    return host.to(device)


def _align16(v: int) -> int:
    return (v + 15) // 16 * 16


# ------------------------------------------------------------ conveniences

class Codec:
    """Device buffers for encoding/decoding tensors of up to `max_n` symbols.

    All buffers are allocated once (PyTorch caching allocator) and reused;
    encode() and decode() launch only the library's kernels.
    """

    def __init__(self, max_n: int, chunk_symbols: int = 4096, scheme=1, device="cuda"):
        self.device = torch.device(device)
        self.chunk_symbols = int(chunk_symbols)
        self.max_n = int(max_n)
        self.scheme = scheme
        cap = qlc_encoded_size(self.max_n, self.chunk_symbols)
        if cap == 0:
            raise QlcError(ERR_ARG, "chunk_symbols")
        z = dict(device=self.device)
        self.cap = cap
        self.hist = torch.zeros(256, dtype=torch.int64, **z)
        self.lut = torch.zeros(LUT_BYTES, dtype=torch.uint8, **z)
        self.ws = torch.zeros(max(16, qlc_encode_workspace_size(self.max_n, self.chunk_symbols)),
                              dtype=torch.uint8, **z)
        self.out_bytes = torch.zeros(1, dtype=torch.int64, **z)
        self.n_out = torch.zeros(1, dtype=torch.int64, **z)
        self.status = torch.zeros(1, dtype=torch.int32, **z)

    def new_container(self) -> torch.Tensor:
        return torch.empty(self.cap, dtype=torch.uint8, device=self.device)

    def encode_into(self, x: torch.Tensor, out: torch.Tensor, stream=None, build_lut: bool = True) -> None:
        """Histogram -> LUT (self.scheme, or the best of a list) -> container."""
        n = x.numel()
        if build_lut:
            qlc_histogram(x, self.hist, n=n, stream=stream)
            if isinstance(self.scheme, list):  # several candidates: the best for this histogram
                qlc_build_lut_best(self.hist, self.scheme, self.lut, stream=stream)
            else:
                qlc_build_lut(self.hist, self.scheme, self.lut, stream=stream)
        qlc_encode(x, self.lut, self.chunk_symbols, out, self.ws, self.out_bytes, self.status,
                   n=n, stream=stream)

    def decode_into(self, container: torch.Tensor, out: torch.Tensor, stream=None,
                    in_bytes: int | None = None) -> None:
        qlc_decode(container, out, self.n_out, self.status, in_bytes=in_bytes, stream=stream)

    def check(self) -> None:
        st = int(self.status.item())
        if st != OK:
            self.status.zero_()
            raise QlcError(st, "device")


def encode(x: torch.Tensor, scheme=1, chunk_symbols: int = 4096) -> torch.Tensor:
    """Container of a CUDA uint8 tensor, trimmed to its size (synchronises)."""
    codec = Codec(max(x.numel(), 1), chunk_symbols, scheme, x.device)
    out = codec.new_container()
    codec.encode_into(x.reshape(-1), out)
    codec.check()
    return out[: int(codec.out_bytes.item())]


def decode(container: torch.Tensor) -> torch.Tensor:
    """Decoded bytes of a CUDA container (synchronises to size the output)."""
    n, total = qlc_peek_header(container[:HEADER_BYTES].cpu().numpy().tobytes())
    out = torch.empty(max(n, 1), dtype=torch.uint8, device=container.device)
    n_out = torch.zeros(1, dtype=torch.int64, device=container.device)
    status = torch.zeros(1, dtype=torch.int32, device=container.device)
    qlc_decode(container, out, n_out, status, out_cap=n)
    st = int(status.item())
    if st != OK:
        raise QlcError(st, "qlc_decode")
    return out[:n]


class Batch:
    """Many shards encoded / decoded with one launch per step (qlc_*_batch).

    shards: CUDA uint8 tensors (16-byte aligned starts).  One LUT per shard,
    or one shared LUT built from the histogram of all shards.  Containers and
    decoded outputs live in two arenas allocated once; encode() / decode()
    launch only library kernels and never synchronise; capture() records both
    as CUDA graphs.
    """

    def __init__(self, shards, chunk_symbols: int = 4096, schemes=(1,), shared_lut: bool = False,
                 launch=None, device=None):
        self.device = torch.device(device) if device is not None else shards[0].device
        self.shards = list(shards)
        self.n = len(self.shards)
        self.chunk_symbols = int(chunk_symbols)
        self.schemes = list(schemes) if isinstance(schemes, (list, tuple)) else [schemes]
        self.shared = bool(shared_lut)
        self.launch = launch
        self.sizes = [s.numel() for s in self.shards]
        self.total = sum(self.sizes)
        caps = [qlc_encoded_size(n, self.chunk_symbols) for n in self.sizes]
        if min(caps) == 0:
            raise QlcError(ERR_ARG, "chunk_symbols")
        self.cap_off = [0]
        for c in caps:
            self.cap_off.append(self.cap_off[-1] + _align16(c))
        self.out_off = [0]
        for n in self.sizes:
            self.out_off.append(self.out_off[-1] + _align16(max(n, 1)))
        z = dict(device=self.device)
        self.containers = torch.empty(self.cap_off[-1], dtype=torch.uint8, **z)
        self.decoded = torch.empty(self.out_off[-1], dtype=torch.uint8, **z)
        n_luts = 1 if self.shared else self.n
        self.hists = torch.zeros(n_luts * 256, dtype=torch.int64, **z)
        self.luts = torch.zeros(n_luts * LUT_BYTES, dtype=torch.uint8, **z)
        self.c_bytes = torch.zeros(self.n, dtype=torch.int64, **z)
        self.n_out = torch.zeros(self.n, dtype=torch.int64, **z)
        self.status = torch.zeros(1, dtype=torch.int32, **z)
        self.ws = torch.zeros(qlc_batch_workspace_size(self.n, self.total, self.chunk_symbols),
                              dtype=torch.uint8, **z)
        cb, lb = self.containers.data_ptr(), self.luts.data_ptr()
        enc = []
        for i, x in enumerate(self.shards):
            lut = lb if self.shared else lb + i * LUT_BYTES
            enc.append((x.data_ptr(), self.sizes[i], cb + self.cap_off[i], caps[i], lut,
                        self.c_bytes.data_ptr() + 8 * i))
        self.enc_descs = descs_tensor(enc, self.device)
        db = self.decoded.data_ptr()
        dec = [(cb + self.cap_off[i], caps[i], db + self.out_off[i], self.sizes[i], 0,
                self.n_out.data_ptr() + 8 * i) for i in range(self.n)]
        self.dec_descs = descs_tensor(dec, self.device)
        self.graphs = {}

    def container(self, i: int) -> torch.Tensor:
        return self.containers[self.cap_off[i]:self.cap_off[i + 1]]

    def output(self, i: int) -> torch.Tensor:
        return self.decoded[self.out_off[i]:self.out_off[i] + self.sizes[i]]

    def encode(self, stream=None, build_luts: bool = True) -> None:
        if build_luts:
            qlc_histogram_batch(self.enc_descs, self.n, self.hists, self.shared, self.ws, stream=stream)
            qlc_build_lut_batch(self.hists, 1 if self.shared else self.n, self.schemes, self.luts, stream=stream)
        qlc_encode_batch(self.enc_descs, self.n, self.chunk_symbols, self.ws, self.status, self.launch,
                         stream=stream)

    def decode(self, stream=None) -> None:
        qlc_decode_batch(self.dec_descs, self.n, self.ws, self.status, self.launch, stream=stream)

    def capture(self) -> None:
        """Record encode() and decode() as CUDA graphs (replay with replay())."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):  # warm up outside the capture
            self.encode(stream=s)
            self.decode(stream=s)
        torch.cuda.current_stream(self.device).wait_stream(s)
        for name, fn in (("encode", self.encode), ("decode", self.decode)):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn(stream=torch.cuda.current_stream(self.device))
            self.graphs[name] = g

    def replay(self, name: str) -> None:
        self.graphs[name].replay()

    def check(self) -> None:
        st = int(self.status.item())
        if st != OK:
            self.status.zero_()
            raise QlcError(st, "batch")
