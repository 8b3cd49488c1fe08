"""Container-v1 parsing for tests, written from the documented byte layout
(header 64 B, decoder LUT 256 B, u64 group offsets, u16 chunk bit counts,
zero pad to 16 B, payload).  Independent of both the oracle and the CUDA path."""
import struct

import numpy as np

CHUNKS_PER_GROUP = 32


def align16(v):
    return (v + 15) // 16 * 16


def parse(buf):
    b = bytes(np.asarray(buf, dtype=np.uint8).tobytes())
    magic, version, scheme_id, flags, n, cs, n_chunks = struct.unpack_from("<4sHBBQII", b, 0)
    area_n = struct.unpack_from("<8H", b, 24)
    area_bits = struct.unpack_from("<8B", b, 40)
    payload_bytes, reserved = struct.unpack_from("<QQ", b, 48)
    dec = np.frombuffer(b[64:320], np.uint8)
    n_groups = (n_chunks + CHUNKS_PER_GROUP - 1) // CHUNKS_PER_GROUP
    group_off = np.frombuffer(b[320:320 + 8 * n_groups], np.uint64)
    cb0 = 320 + 8 * n_groups
    chunk_bits = np.frombuffer(b[cb0:cb0 + 2 * n_chunks], np.uint16)
    P = align16(cb0 + 2 * n_chunks)
    return dict(magic=magic, version=version, scheme_id=scheme_id, flags=flags, n=n,
                chunk_symbols=cs, n_chunks=n_chunks, area_n=area_n, area_bits=area_bits,
                payload_bytes=payload_bytes, reserved=reserved, dec=dec, n_groups=n_groups,
                group_off=group_off, chunk_bits=chunk_bits, payload_start=P,
                index_pad=b[cb0 + 2 * n_chunks:P], payload=b[P:P + payload_bytes],
                total=P + payload_bytes)


def bits_to_bytes(bitstring):
    """MSB-first packing of a '0'/'1' string, zero-padded to a multiple of 16 bytes."""
    nbytes = align16((len(bitstring) + 7) // 8)
    s = bitstring + "0" * (nbytes * 8 - len(bitstring))
    return bytes(int(s[i:i + 8], 2) for i in range(0, len(s), 8))
