"""Pins the CPU oracle to what the paper prints (Tables 1-4, the Section 7
worked example and frequency order) and to hand-worked bit strings derived
from the tables.  None of the expected values comes from the oracle itself."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import _container as C


def _table(golden, name):
    rows = []
    for area, acode, n, bits, length, rng in golden(name):
        lo, hi = (int(v) for v in rng.split("-"))
        rows.append(dict(area=int(area), acode=acode, n=int(n), bits=int(bits),
                         length=int(length), lo=lo, hi=hi))
    return rows


@pytest.mark.parametrize("sid,fname", [(1, "table1_scheme.txt"), (2, "table2_scheme.txt")])
def test_scheme_tables_match_paper(golden, sid, fname):
    rows = _table(golden, fname)
    n, b = oracle.scheme(sid)
    assert [r["n"] for r in rows] == n.tolist()
    assert [r["bits"] for r in rows] == b.tolist()
    # the printed table is self-consistent: ranges tile 0..255, length = 3 + bits,
    # area code = the 3-bit area index
    assert rows[0]["lo"] == 0 and rows[-1]["hi"] == 255
    for i, r in enumerate(rows):
        assert r["hi"] - r["lo"] + 1 == r["n"]
        assert r["length"] == 3 + r["bits"]
        assert r["acode"] == format(i, "03b")
        if i:
            assert r["lo"] == rows[i - 1]["hi"] + 1
    assert oracle.scheme_valid((n, b))


@pytest.mark.parametrize("sid,fname", [(1, "table1_scheme.txt"), (2, "table2_scheme.txt")])
def test_every_rank_code_follows_printed_table(golden, sid, fname):
    """Each rank's code = its area's printed area code, then its offset in the
    area's printed range (raw rank for the 8-bit area, as Table 3 prints)."""
    rows = _table(golden, fname)
    area = oracle.scheme(sid)
    for r in range(256):
        row = next(x for x in rows if x["lo"] <= r <= x["hi"])
        code, ln = oracle.codeword(area, r)
        s = format(code, f"0{ln}b")
        assert ln == row["length"]
        assert s[:3] == row["acode"]
        suffix = r if row["bits"] == 8 else r - row["lo"]
        assert s[3:] == format(suffix, f"0{row['bits']}b")


def test_table3_printed_codewords(golden):
    area = oracle.scheme(1)
    for sym, rank, code in golden("table3_encoder_lut.txt"):
        c, ln = oracle.codeword(area, int(rank))
        assert format(c, f"0{ln}b") == code.replace("_", "")


def test_decode_example_section7(golden):
    area = oracle.scheme(1)
    (acode, suffix, rank), = golden("decode_example.txt")
    bits = acode + suffix
    assert oracle.decode_codeword(area, int(bits, 2), len(bits)) == int(rank)


def test_lut_order_tables_3_and_4(golden):
    """A histogram whose frequency order is the one Section 7 and Tables 3/4
    print must give exactly the printed symbol <-> rank pairs."""
    fixed = {}
    for sym, rank, _ in golden("table3_encoder_lut.txt"):
        fixed[int(rank)] = int(sym)
    for rank, sym in golden("table4_decoder_lut.txt"):
        assert fixed[int(rank)] == int(sym)
    most = [int(v) for v in golden("section7_frequency_order.txt")[0][1:]]
    least = [int(v) for v in golden("section7_frequency_order.txt")[1][1:]]
    for i, s in enumerate(most):
        fixed.setdefault(i, s)
        assert fixed[i] == s
    for i, s in enumerate(least):
        fixed.setdefault(252 + i, s)
        assert fixed[252 + i] == s
    rest = [s for s in range(256) if s not in fixed.values()]
    order = []
    it = iter(rest)
    for r in range(256):
        order.append(fixed[r] if r in fixed else next(it))
    hist = np.zeros(256, np.uint64)
    for r, s in enumerate(order):
        hist[s] = 10_000 - 7 * r          # strictly decreasing with rank
    sor, ros = oracle.rank(hist)
    for r, s in fixed.items():
        assert sor[r] == s and ros[s] == r
    area = oracle.scheme(1)
    for sym, rank, code in golden("table3_encoder_lut.txt"):
        c, ln = oracle.codeword(area, int(ros[int(sym)]))
        assert format(c, f"0{ln}b") == code.replace("_", "")


def test_worked_streams(golden):
    for row in golden("worked_streams.txt"):
        sid, ranks, codes = int(row[0]), [int(v) for v in row[1].split(",")], row[2:]
        bits = "".join(codes)
        ident = np.arange(256, dtype=np.uint8)
        cont = oracle.encode(np.array(ranks, np.uint8), scheme_id=sid, sym_of_rank=ident,
                             chunk_symbols=128)
        p = C.parse(cont)
        assert p["payload"] == C.bits_to_bytes(bits)
        assert p["chunk_bits"].tolist() == [len(bits)]
        st, out, n = oracle.decode(cont)
        assert st == oracle.OK and out.tolist() == ranks


def test_worked_bytes_from_design_notes():
    """Byte values worked out by hand for Table 1 (ranks 0,1,2,8 -> 00 10 88;
    ranks 253,254,255 -> FF BF FB FF 80; area boundaries -> 02 7A 17 F0 37 FA C7 FF)."""
    ident = np.arange(256, dtype=np.uint8)
    cases = [([0, 1, 2, 8], "001088"), ([253, 254, 255], "ffbffbff80"),
             ([0, 39, 40, 55, 56, 87, 88, 255], "027a17f037fac7ff")]
    for ranks, hexs in cases:
        cont = oracle.encode(np.array(ranks, np.uint8), sym_of_rank=ident, chunk_symbols=128)
        p = C.parse(cont)
        want = bytes.fromhex(hexs)
        assert p["payload"][:len(want)] == want
        assert set(p["payload"][len(want):]) <= {0}


@pytest.mark.parametrize("sid,kraft", [(1, Fraction(1960, 2048)), (2, Fraction(1950, 2048))])
def test_kraft_sum_and_prefix_free(sid, kraft):
    """7/8 from the seven complete areas plus n_8 / 2^11 from the last area:
    168/2048 (Table 1) and 158/2048 (Table 2); the code is not complete."""
    area = oracle.scheme(sid)
    codes = [oracle.codeword(area, r) for r in range(256)]
    assert sum(Fraction(1, 2 ** ln) for _, ln in codes) == kraft
    strs = [format(c, f"0{ln}b") for c, ln in codes]
    assert len(set(strs)) == 256
    for i, a in enumerate(strs):
        for j, b in enumerate(strs):
            if i != j:
                assert not b.startswith(a)
    # the 3-bit area level is complete: every area code occurs
    assert {s[:3] for s in strs} == {format(i, "03b") for i in range(8)}


def test_closed_forms():
    t1, t2 = oracle.scheme(1), oracle.scheme(2)
    # constant input: every symbol gets rank 0 -> 6 bits (Table 1), 4 bits (Table 2)
    h = np.zeros(256, np.uint64)
    h[113] = 1000
    assert oracle.code_bits(h, t1) == 6000
    assert oracle.code_bits(h, t2) == 4000
    # uniform histogram: (40*6 + 16*7 + 32*8 + 168*11) / 256 = 9.59375 bits
    h = np.full(256, 4, np.uint64)
    assert Fraction(oracle.code_bits(h, t1), 1024) == Fraction(959375, 100000)
    # Table 2: (2*4 + 32*6 + 64*8 + 158*11) / 256 = 9.5703125 bits
    assert Fraction(oracle.code_bits(h, t2), 1024) == Fraction(95703125, 10000000)


def test_single_symbol_inputs_exhaustive():
    for s in range(256):
        cont = oracle.encode(np.array([s], np.uint8), chunk_symbols=128)
        p = C.parse(cont)
        assert p["payload"] == C.bits_to_bytes("000000")
        assert p["dec"][0] == s
        st, out, n = oracle.decode(cont)
        assert st == oracle.OK and n == 1 and out[0] == s


def test_two_symbol_inputs_exhaustive():
    """All 65,536 two-symbol inputs, each ranked by its own histogram: equal
    symbols -> two rank-0 codes; otherwise both counts are 1 and the smaller
    byte takes rank 0 (000000), the larger rank 1 (000001)."""
    for a in range(256):
        for b in range(256):
            cont = oracle.encode(np.array([a, b], np.uint8), chunk_symbols=128)
            p = C.parse(cont)
            if a == b:
                bits = "000000000000"
            else:
                bits = ("000000" if a < b else "000001") + ("000000" if b < a else "000001")
            assert p["payload"] == C.bits_to_bytes(bits), (a, b)
            st, out, n = oracle.decode(cont)
            assert st == oracle.OK and out.tolist() == [a, b]
