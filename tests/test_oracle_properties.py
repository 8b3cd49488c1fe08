"""Properties that pin the oracle beyond the printed examples: round trips,
the exact bit-count identity, optimality of the rank order (rearrangement
inequality), Huffman optimality against brute force, entropy special cases
and a library routine, container layout and corruption handling."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2602_17849_gb300 import inputs
from tests import _container as C


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("n", [0, 1, 15, 16, 127, 128, 129, 4095, 4096, 4097, 32 * 128 - 1,
                               32 * 128, 32 * 128 + 1, 100_003])
@pytest.mark.parametrize("cs", [128, 1024, 4096])
def test_round_trip_sizes(n, cs):
    x = _rng(n + cs).integers(0, 256, n, dtype=np.uint8) ** 2 // 255  # skewed bytes
    x = x.astype(np.uint8)
    cont = oracle.encode(x, chunk_symbols=cs)
    p = C.parse(cont)
    assert p["magic"] == b"QLC1" and p["version"] == 1 and p["n"] == n
    assert p["chunk_symbols"] == cs and p["n_chunks"] == -(-n // cs)
    assert p["total"] == len(cont) and len(cont) % 16 == 0
    assert len(cont) <= oracle.container_bound(n, cs)
    st, out, m = oracle.decode(cont)
    assert st == oracle.OK and m == n and np.array_equal(out, x)


@pytest.mark.parametrize("kind", ["t4", "gauss", "laplace", "laplace_outliers", "relu_t4", "ffn2",
                                  "uniform_bytes", "constant"])
@pytest.mark.parametrize("sid", [1, 2])
def test_round_trip_synthetic(kind, sid):
    x = inputs.make_e4m3(kind, 200_000, seed=7).numpy()
    cont = oracle.encode(x, scheme_id=sid, chunk_symbols=1024)
    st, out, _ = oracle.decode(cont)
    assert st == oracle.OK and np.array_equal(out, x)


def test_adversarial_streams():
    ident = np.arange(256, dtype=np.uint8)
    for x in [np.full(9000, 255, np.uint8),                       # all 11-bit codes
              np.zeros(9000, np.uint8),                           # all rank 0
              np.tile(np.array([0, 255], np.uint8), 4500),        # alternate 6/11 bits
              np.arange(256 * 40, dtype=np.int64).astype(np.uint8)]:
        cont = oracle.encode(x, sym_of_rank=ident, chunk_symbols=128)
        st, out, _ = oracle.decode(cont)
        assert st == oracle.OK and np.array_equal(out, x)


def test_payload_bits_equal_count_times_length():
    """Total payload bits = sum_s count[s] * len(rank[s]), exactly."""
    for seed, kind in enumerate(["t4", "laplace_outliers", "uniform_bytes"]):
        x = inputs.make_e4m3(kind, 300_001, seed=seed).numpy()
        h = oracle.histogram(x)
        assert int(h.sum()) == x.size
        assert np.array_equal(h, np.bincount(x, minlength=256).astype(np.uint64))
        for sid in (1, 2):
            p = C.parse(oracle.encode(x, scheme_id=sid, chunk_symbols=4096))
            assert int(p["chunk_bits"].astype(np.int64).sum()) == oracle.code_bits(h, oracle.scheme(sid))


def test_rank_order_minimises_bits():
    """Rearrangement inequality: with counts sorted descending against
    non-decreasing code lengths, no swap of two symbols' codes lowers the total."""
    x = inputs.make_e4m3("t4", 100_000, seed=3).numpy()
    h = oracle.histogram(x).astype(np.int64)
    for sid in (1, 2):
        area = oracle.scheme(sid)
        _, ros = oracle.rank(h)
        ln = np.array([oracle.codeword(area, int(ros[s]))[1] for s in range(256)])
        base = int((h * ln).sum())
        assert base == oracle.code_bits(h, area)
        for s in range(256):
            for t in range(s + 1, 256):
                assert base - h[s] * ln[s] - h[t] * ln[t] + h[s] * ln[t] + h[t] * ln[s] >= base
        # code lengths never decrease with rank
        lens = [oracle.codeword(area, r)[1] for r in range(256)]
        assert lens == sorted(lens)


def _brute_force_prefix_code(counts):
    """Minimum sum count*len over length vectors with Kraft sum <= 1."""
    k = len(counts)
    best = None
    for lens in itertools.product(range(1, k), repeat=k):
        if sum(Fraction(1, 2 ** l) for l in lens) <= 1:
            v = sum(c * l for c, l in zip(counts, lens))
            best = v if best is None else min(best, v)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_huffman_matches_brute_force(seed):
    r = _rng(100 + seed)
    k = int(r.integers(2, 7))
    counts = [int(v) for v in r.integers(1, 60, k)]
    h = np.zeros(256, np.uint64)
    syms = r.choice(256, k, replace=False)
    for s, c in zip(syms, counts):
        h[s] = c
    assert oracle.huffman_bits(h) == _brute_force_prefix_code(counts)


def test_huffman_bounds_and_dyadic():
    x = inputs.make_e4m3("t4", 400_000, seed=11).numpy()
    h = oracle.histogram(x)
    H = oracle.entropy(h)
    E = oracle.huffman_bits(h) / x.size
    assert H <= E < H + 1
    assert oracle.huffman_roundtrip(x) == oracle.huffman_bits(h)
    # dyadic PMF: p = 1/2, 1/4, 1/8, 1/8 -> E[len] = H = 1.75
    h = np.zeros(256, np.uint64)
    h[[3, 9, 200, 17]] = [4, 2, 1, 1]
    assert oracle.huffman_bits(h) == 14 and oracle.entropy(h) == 1.75
    # one symbol: one bit per symbol
    h = np.zeros(256, np.uint64)
    h[5] = 10
    assert oracle.huffman_bits(h) == 10


def test_entropy_special_cases_and_library():
    assert oracle.entropy(np.full(256, 3, np.uint64)) == 8.0
    h = np.zeros(256, np.uint64)
    h[[1, 2]] = 5
    assert oracle.entropy(h) == 1.0
    scipy_stats = pytest.importorskip("scipy.stats")
    x = inputs.make_e4m3("laplace", 50_000, seed=2).numpy()
    h = oracle.histogram(x)
    assert math.isclose(oracle.entropy(h), scipy_stats.entropy(h.astype(np.float64), base=2),
                        rel_tol=1e-12)


def test_paper_ordering_on_synthetic_activations():
    """Sections 4-5: entropy bound > Huffman > QLC (Table 1) in compressibility.
    The paper's own 16.3% / 15.9% / 13.9% come from Gemma-2B tensors that are
    not available (parity unpinned); the synthetic stand-in must keep the order."""
    x = inputs.make_e4m3("t4", 1 << 20, seed=0).numpy()
    h = oracle.histogram(x)
    ideal = (8 - oracle.entropy(h)) / 8
    huff = 1 - oracle.huffman_bits(h) / (8 * x.size)
    qlc = 1 - oracle.code_bits(h, oracle.scheme(1)) / (8 * x.size)
    assert ideal > huff > qlc > 0.10
    assert 0.12 < ideal < 0.22


def test_adaptation_ordering_on_ffn2_stand_in():
    """Section 6: on an FFN2-like PMF (one dominant symbol, zero) the adapted
    scheme (Table 2) beats Table 1 by a few percentage points and stays a few
    points below Huffman; entropy bound > Huffman > Table 2 > Table 1.  The
    paper's own 23.6 / 23.2 / 19.0 / 16.7 % are measured on Gemma-2B tensors
    (parity unpinned); the stand-in must keep the ordering and the gaps' signs."""
    x = inputs.make_e4m3("ffn2", 1 << 20, seed=0).numpy()
    h = oracle.histogram(x)
    n = x.size
    ideal = (8 - oracle.entropy(h)) / 8
    huff = 1 - oracle.huffman_bits(h) / (8 * n)
    t1 = 1 - oracle.code_bits(h, oracle.scheme(1)) / (8 * n)
    t2 = 1 - oracle.code_bits(h, oracle.scheme(2)) / (8 * n)
    assert ideal > huff > t2 > t1
    assert 0.01 < t2 - t1 < 0.05 and 0.02 < huff - t2 < 0.07
    assert int(np.argmax(h)) == 0                     # zero is the dominant symbol


def test_container_layout_and_index():
    x = inputs.make_e4m3("t4", 5 * 32 * 1024 + 777, seed=5).numpy()
    cont = oracle.encode(x, chunk_symbols=1024)
    p = C.parse(cont)
    assert p["n_groups"] == 6 and p["n_chunks"] == 5 * 32 + 1
    assert p["flags"] == 0 and p["reserved"] == 0 and p["scheme_id"] == 1
    assert p["payload_start"] % 16 == 0 and set(p["index_pad"]) <= {0}
    off = 0
    for g in range(p["n_groups"]):
        assert p["group_off"][g] == off
        bits = int(p["chunk_bits"][32 * g:32 * (g + 1)].astype(np.int64).sum())
        off += C.align16((bits + 7) // 8)
    assert off == p["payload_bytes"]
    sor, _ = oracle.rank(oracle.histogram(x))
    assert np.array_equal(p["dec"], sor)


def _flip(cont, byte, bit=0):
    c = cont.copy()
    c[byte] ^= np.uint8(1 << bit)
    return c


def test_corrupt_containers_rejected():
    x = inputs.make_e4m3("t4", 70_000, seed=9).numpy()
    cont = oracle.encode(x, chunk_symbols=1024)
    p = C.parse(cont)
    cb0 = 320 + 8 * p["n_groups"]
    bad = {
        "magic": _flip(cont, 0),
        "version": _flip(cont, 4),
        "flags": _flip(cont, 7),
        "n": _flip(cont, 10),
        "chunk_symbols": _flip(cont, 16, 3),
        "scheme_n": _flip(cont, 24),
        "scheme_bits": _flip(cont, 40),
        "reserved": _flip(cont, 56),
        "dec_not_perm": _flip(cont, 64),
        "group_off": _flip(cont, 320 + 8, 4),
        "chunk_bits": _flip(cont, cb0 + 2 * 5),
        "payload_bytes": _flip(cont, 48, 4),
        "truncated": cont[:-16],
        "short": cont[:100],
    }
    for name, c in bad.items():
        st, _, _ = oracle.decode(c, cap=x.size)
        assert st == oracle.ERR_CORRUPT, name
    st, _, n = oracle.decode(cont, cap=x.size - 1)
    assert st == oracle.ERR_CAPACITY and n == x.size


def test_non_canonical_last_area_suffix_decodes_raw():
    """Reading R1: the decoder takes the 8 suffix bits of the last area as the
    rank itself, also below the area's first rank (never emitted)."""
    ident = np.arange(256, dtype=np.uint8)
    cont = oracle.encode(np.array([200], np.uint8), sym_of_rank=ident, chunk_symbols=128)
    p = C.parse(cont)
    c = cont.copy()
    P = p["payload_start"]
    # codeword 111 11001000 (rank 200) -> 111 00000101 (rank 5, below 88)
    bits = "111" + format(5, "08b")
    c[P:P + 2] = np.frombuffer(C.bits_to_bytes(bits)[:2], np.uint8)
    st, out, _ = oracle.decode(c)
    assert st == oracle.OK and out.tolist() == [5]


def test_encode_rejects_bad_arguments():
    x = np.zeros(10, np.uint8)
    with pytest.raises(RuntimeError):
        oracle.encode(x, chunk_symbols=100)
    with pytest.raises(RuntimeError):
        oracle.encode(x, sym_of_rank=np.zeros(256, np.uint8))
    bad_area = (np.array([8, 8, 8, 8, 8, 16, 32, 160], np.uint16), oracle.scheme(1)[1])
    assert not oracle.scheme_valid(bad_area)
    with pytest.raises(RuntimeError):
        oracle.encode(x, area=bad_area, scheme_id=0)
    with pytest.raises(RuntimeError):
        oracle.encode(x, cap=100)
