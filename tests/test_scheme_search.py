"""Scheme search (the paper's future work, Section 8): the library's exhaustive
search over the qlc_scheme family against an independent brute force in
Python and the oracle's bit count; searched schemes code and decode exactly."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2602_17849_gb300 import _build, inputs


@pytest.fixture(scope="module")
def qlc():
    _build.build()
    from paper_2602_17849_gb300 import qlc as q
    return q


def _brute_force_best(hist):
    c = np.sort(np.asarray(hist, dtype=np.int64))[::-1]
    pre = np.concatenate([[0], np.cumsum(c)])
    best = None
    for bs in itertools.combinations_with_replacement(range(8), 7):  # non-decreasing widths
        n = [1 << b for b in bs]
        base = sum(n)
        if base > 255:
            continue
        rem = 256 - base
        lasts = [8]
        if rem & (rem - 1) == 0 and rem <= 128 and rem.bit_length() - 1 >= bs[-1]:
            lasts.append(rem.bit_length() - 1)
        for lb in lasts:
            cost, b0 = 0, 0
            for w, k in zip(list(bs) + [lb], n + [rem]):
                cost += (3 + w) * int(pre[b0 + k] - pre[b0])
                b0 += k
            best = cost if best is None else min(best, cost)
    return best


@pytest.mark.parametrize("kind", ["t4", "ffn2", "gauss", "laplace_outliers", "relu_t4", "uniform_bytes",
                                  "constant"])
def test_search_is_optimal_in_its_family(qlc, kind):
    x = inputs.make_e4m3(kind, 200_000, seed=8).numpy()
    h = oracle.histogram(x)
    sc, bits = qlc.qlc_scheme_search(h)
    area = (np.array(list(sc.area_n), np.uint16), np.array(list(sc.area_bits), np.uint8))
    assert oracle.scheme_valid(area) and qlc.qlc_scheme_check(sc)
    assert bits == oracle.code_bits(h, area)                  # the oracle agrees on its cost
    assert bits == _brute_force_best(h)                       # and nothing in the family is cheaper
    assert bits <= oracle.code_bits(h, oracle.scheme(1))
    assert bits <= oracle.code_bits(h, oracle.scheme(2))
    cont = oracle.encode(x, scheme_id=0, area=area, chunk_symbols=1024)
    st, y, _ = oracle.decode(cont)
    assert st == oracle.OK and np.array_equal(y, x)


def test_search_finds_table_2_shape_gain_on_ffn2(qlc):
    """On the FFN2 stand-in the searched scheme gains over both printed tables."""
    x = inputs.make_e4m3("ffn2", 1 << 20, seed=0).numpy()
    h = oracle.histogram(x)
    _, bits = qlc.qlc_scheme_search(h)
    t1 = oracle.code_bits(h, oracle.scheme(1))
    t2 = oracle.code_bits(h, oracle.scheme(2))
    assert bits < t2 < t1
