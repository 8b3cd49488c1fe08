"""CPU checks of the C ABI: libqlc.so loads without a GPU, exports every
function include/qlc.h declares, and its host-only entry points agree with
the oracle (no device compute is called here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2602_17849_gb300 import _build, inputs
from tests import _container as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(qlc_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def qlc():
    _build.build()
    from paper_2602_17849_gb300 import qlc as q
    return q


def test_library_exports_every_declared_symbol(qlc):
    names = _declared()
    assert len(names) >= 13
    lib = ctypes.CDLL(_build.LIB)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_scheme_tables_and_check(qlc):
    for sid in (1, 2):
        s = qlc.qlc_scheme_table(sid)
        n, b = oracle.scheme(sid)
        assert list(s.area_n) == n.tolist() and list(s.area_bits) == b.tolist() and s.id == sid
        assert qlc.qlc_scheme_check(s)
    bad = qlc.make_scheme([8, 8, 8, 8, 8, 16, 32, 160], [3, 3, 3, 3, 3, 4, 5, 8])
    assert not qlc.qlc_scheme_check(bad)
    wrong_id = qlc.make_scheme(*oracle.scheme(2), scheme_id=1)
    assert not qlc.qlc_scheme_check(wrong_id)
    # validity agrees with the oracle on perturbed tables
    rng = np.random.Generator(np.random.PCG64(4))
    for _ in range(300):
        n = np.array(oracle.scheme(1)[0], np.int64)
        b = np.array(oracle.scheme(1)[1], np.int64)
        i = int(rng.integers(0, 8))
        b[i] = max(0, min(8, b[i] + int(rng.integers(-1, 2))))
        n[i] = 2 ** b[i] if b[i] < 8 else n[i]
        n[7] = 256 - n[:7].sum() if rng.random() < 0.7 else n[7]
        n = np.clip(n, 0, 65535)
        assert qlc.qlc_scheme_check(qlc.make_scheme(n, b)) == oracle.scheme_valid((n, b))


def test_host_lut_matches_oracle(qlc):
    for kind, sid in [("t4", 1), ("relu_t4", 2), ("uniform_bytes", 1), ("constant", 2)]:
        x = inputs.make_e4m3(kind, 50_000, seed=1).numpy()
        h = oracle.histogram(x)
        lut = qlc.qlc_build_lut_host(h, sid)
        sor, ros = oracle.rank(h)
        assert list(lut.dec) == sor.tolist()
        area = oracle.scheme(sid)
        for s in range(256):
            code, ln = oracle.codeword(area, int(ros[s]))
            assert lut.enc[s] == (code << 4) | ln


def test_sizes_match_oracle_bound(qlc):
    for n in [0, 1, 4095, 4096, 131072, 131073, 10 ** 7 + 3]:
        for cs in [128, 1024, 4096]:
            assert qlc.qlc_encoded_size(n, cs) == oracle.container_bound(n, cs)
            groups = -(-(-(-n // cs)) // 32)
            assert qlc.qlc_encode_workspace_size(n, cs) == 16 + 8 * groups
    assert qlc.qlc_encoded_size(100, 100) == 0


def test_peek_header_on_oracle_container(qlc):
    x = inputs.make_e4m3("t4", 123_457, seed=2).numpy()
    cont = oracle.encode(x, chunk_symbols=2048)
    n, total = qlc.qlc_peek_header(cont[:64].tobytes())
    assert n == x.size and total == cont.size == C.parse(cont)["total"]
    with pytest.raises(qlc.QlcError):
        qlc.qlc_peek_header(b"XXXX" + cont[4:64].tobytes())


def test_status_strings(qlc):
    assert qlc.status_string(0) == "ok"
    assert "corrupt" in qlc.status_string(3)
    assert qlc.qlc_version() == 1
