"""Property tests (CPU, hypothesis): the oracle's round trip and container
invariants over arbitrary byte strings, chunk sizes and schemes, and the
library's host-side LUT builder and scheme search against the oracle on
arbitrary histograms, ties included.  Skipped where hypothesis is not
installed."""
import numpy as np
import pytest

import oracle
from tests import _container as C

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

# byte strings drawn from a few symbols (long runs, skewed PMFs) or from all 256
small_alphabet = st.lists(st.sampled_from([0, 1, 0x71, 0xF1, 0x69, 0x80, 255]), max_size=6000)
any_bytes = st.binary(max_size=6000).map(list)
chunk = st.integers(1, 32).map(lambda k: 128 * k)


@settings(max_examples=120, deadline=None)
@given(data=st.one_of(small_alphabet, any_bytes), cs=chunk, sid=st.sampled_from([1, 2]))
def test_oracle_round_trip_and_container_invariants(data, cs, sid):
    """decode(encode(x)) = x; the index's chunk bit counts add up to
    sum(count * length) (Sections 5 and 7); every group starts on a 16-byte
    boundary and holds exactly its chunks' bits, zero-padded."""
    x = np.asarray(data, np.uint8)
    cont = oracle.encode(x, scheme_id=sid, chunk_symbols=cs)
    st_, y, n = oracle.decode(cont)
    assert st_ == oracle.OK and n == x.size and np.array_equal(y, x)
    p = C.parse(cont)
    assert p["n"] == x.size and p["chunk_symbols"] == cs and p["total"] == cont.size
    assert int(p["chunk_bits"].sum()) == oracle.code_bits(oracle.histogram(x), oracle.scheme(sid))
    assert p["n_chunks"] == (x.size + cs - 1) // cs
    bits = p["chunk_bits"].astype(np.int64)
    off = 0
    for g in range(p["n_groups"]):
        assert int(p["group_off"][g]) == off
        gbits = int(bits[32 * g:32 * g + 32].sum())
        off += C.align16((gbits + 7) // 8)
    assert off == p["payload_bytes"]


@pytest.fixture(scope="module")
def qlc():
    from paper_2602_17849_gb300 import _build
    _build.build()
    from paper_2602_17849_gb300 import qlc as q
    return q


counts = st.lists(st.sampled_from([0, 0, 1, 2, 3, 7, 1000, 2 ** 31, 2 ** 40]), min_size=256, max_size=256)


@settings(max_examples=150, deadline=None)
@given(h=counts, sid=st.sampled_from([1, 2]))
def test_host_lut_equals_oracle_on_arbitrary_histograms(qlc, h, sid):
    """Ranks by decreasing count, ties to the smaller symbol (Section 7), and
    each symbol's codeword (Tables 1 and 2), for histograms full of ties and
    zero counts."""
    h = np.asarray(h, np.uint64)
    lut = qlc.qlc_build_lut_host(h, sid)
    sor, ros = oracle.rank(h)
    assert list(lut.dec) == sor.tolist()
    area = oracle.scheme(sid)
    for s in range(256):
        code, ln = oracle.codeword(area, int(ros[s]))
        assert lut.enc[s] == (code << 4) | ln


@settings(max_examples=60, deadline=None)
@given(h=counts)
def test_scheme_search_never_worse_than_the_tables(qlc, h):
    """The searched scheme is valid and codes the histogram in no more bits
    than Table 1 or Table 2 (Section 6: the scheme adapts to the PMF)."""
    h = np.asarray(h, np.uint64)
    sc, bits = qlc.qlc_scheme_search(h)
    area = (np.array(sc.area_n[:], np.uint16), np.array(sc.area_bits[:], np.uint8))
    assert oracle.scheme_valid(area)
    assert bits == oracle.code_bits(h, area)
    assert bits <= min(oracle.code_bits(h, oracle.scheme(1)), oracle.code_bits(h, oracle.scheme(2)))
