"""GPU parity: every step of the CUDA path through the C ABI against the CPU
oracle on the same seeded inputs.  Integer work, so the bar is bit-exact:
histogram counts, LUT entries, every container byte, every decoded byte and
the device status on corrupt input."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_17849_gb300 import inputs
from tests import _container as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qlc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2602_17849_gb300 import _build
    _build.build()
    from paper_2602_17849_gb300 import qlc as q
    return q


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _gpu_pipeline(qlc, x, sid, cs):
    """histogram -> LUT -> encode -> decode on the GPU; returns host copies."""
    n = x.size
    xd = _dev(x) if n else torch.zeros(16, dtype=torch.uint8, device="cuda")
    codec = qlc.Codec(max(n, 1), cs, sid)
    cont = codec.new_container()
    codec.encode_into(xd[:n] if n else xd[:0], cont)
    torch.cuda.synchronize()
    codec.check()
    nbytes = int(codec.out_bytes.item())
    y = torch.full((max(n, 1),), 0xAB, dtype=torch.uint8, device="cuda")
    codec.decode_into(cont, y, in_bytes=nbytes)
    torch.cuda.synchronize()
    codec.check()
    assert int(codec.n_out.item()) == n
    return dict(hist=codec.hist.cpu().numpy().astype(np.uint64), lut=codec.lut.cpu().numpy(),
                cont=cont[:nbytes].cpu().numpy(), y=y[:n].cpu().numpy())


def _check_lut(lut_bytes, hist, sid):
    sor, ros = oracle.rank(hist)
    enc = lut_bytes[32:544].view(np.uint16)
    dec = lut_bytes[544:800]
    assert np.array_equal(dec, sor)
    area = oracle.scheme(sid)
    for s in range(256):
        code, ln = oracle.codeword(area, int(ros[s]))
        assert enc[s] == (code << 4) | ln


SIZES = [1, 15, 16, 17, 31, 32, 33, 127, 128, 129, 1023, 1024, 1025, 4095, 4096, 4097,
         32 * 128 - 1, 32 * 128, 32 * 128 + 1, 32 * 1024 + 5, 32 * 4096 - 1, 32 * 4096,
         32 * 4096 + 1, 3 * 32 * 4096 + 4096 * 7 + 333]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("cs", [128, 1024, 4096])
def test_round_trip_matches_oracle_sizes(qlc, n, cs):
    x = inputs.make_e4m3("t4", n, seed=n).numpy()
    r = _gpu_pipeline(qlc, x, 1, cs)
    assert np.array_equal(r["hist"], oracle.histogram(x))
    _check_lut(r["lut"], oracle.histogram(x), 1)
    want = oracle.encode(x, scheme_id=1, chunk_symbols=cs)
    assert r["cont"].size == want.size and np.array_equal(r["cont"], want)
    assert np.array_equal(r["y"], x)


def test_empty_input(qlc):
    x = np.zeros(0, np.uint8)
    r = _gpu_pipeline(qlc, x, 1, 4096)
    want = oracle.encode(x, scheme_id=1, chunk_symbols=4096)
    assert np.array_equal(r["cont"], want) and r["cont"].size == 320
    assert r["hist"].sum() == 0


@pytest.mark.parametrize("kind", ["t4", "gauss", "laplace", "laplace_outliers", "relu_t4",
                                  "uniform_bytes", "constant"])
@pytest.mark.parametrize("sid", [1, 2])
def test_round_trip_matches_oracle_kinds(qlc, kind, sid):
    x = inputs.make_e4m3(kind, 5 * 32 * 1024 + 4321, seed=11).numpy()
    r = _gpu_pipeline(qlc, x, sid, 1024)
    assert np.array_equal(r["hist"], oracle.histogram(x))
    _check_lut(r["lut"], oracle.histogram(x), sid)
    want = oracle.encode(x, scheme_id=sid, chunk_symbols=1024)
    assert np.array_equal(r["cont"], want)
    assert np.array_equal(r["y"], x)


def test_adversarial_streams(qlc):
    """All 11-bit codes, all 6-bit codes, and alternation, with a fixed LUT."""
    ident = np.arange(256, dtype=np.uint8)
    for x in [np.full(70_001, 255, np.uint8), np.zeros(70_001, np.uint8),
              np.tile(np.array([0, 255], np.uint8), 35_000),
              np.arange(256 * 300, dtype=np.int64).astype(np.uint8)]:
        cont = oracle.encode(x, sym_of_rank=ident, chunk_symbols=1024)
        # decode the oracle's container on the GPU
        d = _dev(cont)
        y = torch.empty(x.size, dtype=torch.uint8, device="cuda")
        n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        qlc.qlc_decode(d, y, n_out, st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0 and np.array_equal(y.cpu().numpy(), x)
        # encode with the same fixed LUT on the GPU
        lut = qlc.qlc_build_lut_host(np.arange(256, 0, -1), 1)   # counts fall with the symbol
        assert list(lut.dec) == ident.tolist()
        dl = torch.frombuffer(bytearray(bytes(lut)), dtype=torch.uint8).cuda()
        out = torch.empty(qlc.qlc_encoded_size(x.size, 1024), dtype=torch.uint8, device="cuda")
        ws = torch.empty(qlc.qlc_encode_workspace_size(x.size, 1024), dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        qlc.qlc_encode(_dev(x), dl, 1024, out, ws, nb, st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert np.array_equal(out[: int(nb.item())].cpu().numpy(), cont)


def test_histogram_accumulate(qlc):
    a = inputs.make_e4m3("t4", 100_003, seed=1)
    b = inputs.make_e4m3("laplace", 77_777, seed=2)
    h = torch.zeros(256, dtype=torch.int64, device="cuda")
    qlc.qlc_histogram(a.cuda(), h)
    qlc.qlc_histogram(b.cuda(), h, accumulate=True)
    want = oracle.histogram(np.concatenate([a.numpy(), b.numpy()]))
    assert np.array_equal(h.cpu().numpy().astype(np.uint64), want)


@pytest.mark.parametrize("n", [1, 15, 16, 17, 3072 * 16 - 1, 3072 * 16, 3072 * 16 + 1, 2 * 3072 * 16 + 9,
                               152 * 3072 * 16 - 16, 152 * 3072 * 16 + 17, 10_000_019, 64 * 2**20 + 3])
def test_histogram_grid_sizes(qlc, n):
    """The histogram's grid is one CTA per 48 KiB of input up to one per SM;
    sizes around those steps, with ragged slices and tails, count exactly."""
    for kind in ("t4", "constant", "uniform_bytes"):
        x = inputs.make_e4m3(kind, n, seed=n % 1000)
        h = torch.full((256,), 7, dtype=torch.int64, device="cuda")
        qlc.qlc_histogram(x.cuda(), h)
        assert np.array_equal(h.cpu().numpy().astype(np.uint64), oracle.histogram(x.numpy())), kind


def test_build_lut_best_picks_fewer_bits(qlc):
    for kind in ("t4", "relu_t4"):
        x = inputs.make_e4m3(kind, 200_000, seed=3).numpy()
        h = oracle.histogram(x)
        b1 = oracle.code_bits(h, oracle.scheme(1))
        b2 = oracle.code_bits(h, oracle.scheme(2))
        best = 1 if b1 <= b2 else 2
        hd = torch.from_numpy(h.astype(np.int64)).cuda()
        lut = torch.zeros(800, dtype=torch.uint8, device="cuda")
        qlc.qlc_build_lut_best(hd, [1, 2], lut)
        lb = lut.cpu().numpy()
        assert lb[24] == best                          # qlc_scheme.id
        _check_lut(lb, h, best)


def _decode_status(qlc, cont, cap):
    d = _dev(cont) if cont.size else torch.zeros(16, dtype=torch.uint8, device="cuda")
    y = torch.zeros(max(cap, 1), dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    qlc.qlc_decode(d, y, n_out, st, in_bytes=cont.size, out_cap=cap)
    torch.cuda.synchronize()
    return int(st.item()), y[:cap].cpu().numpy()


def test_corrupt_containers_same_status_as_oracle(qlc):
    """Single-bit flips over the header, the LUT, the index and the payload:
    the device status equals the oracle's; where both accept, the outputs
    (possibly wrong symbols: the code has no checksum) are identical."""
    x = inputs.make_e4m3("t4", 3 * 32 * 1024 + 999, seed=9).numpy()
    cont = oracle.encode(x, chunk_symbols=1024)
    rng = np.random.Generator(np.random.PCG64(17))
    P = C.parse(cont)["payload_start"]
    positions = list(range(0, 64)) + [64, 100, 319] + list(range(320, P)) + \
        [int(v) for v in rng.integers(P, cont.size, 200)]
    for pos in positions:
        c = cont.copy()
        c[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        ost, oy, _ = oracle.decode(c, cap=x.size)
        gst, gy = _decode_status(qlc, c, x.size)
        assert gst == ost, pos
        if ost == oracle.OK:
            assert np.array_equal(gy, oy), pos
    for cut in (0, 10, 319, P - 1, cont.size - 16, cont.size - 1):
        ost, _, _ = oracle.decode(cont[:cut], cap=x.size)
        gst, _ = _decode_status(qlc, cont[:cut], x.size)
        assert gst == ost == oracle.ERR_CORRUPT, cut
    assert _decode_status(qlc, cont, x.size - 1)[0] == oracle.ERR_CAPACITY


def test_full_1mib_tensor(qlc):
    """1 MiB Student-t(4) tensor, seed 0, LUT from its own histogram, chunk 4096."""
    x = inputs.make_e4m3("t4", 1 << 20, seed=0).numpy()
    r = _gpu_pipeline(qlc, x, 1, 4096)
    want = oracle.encode(x, scheme_id=1, chunk_symbols=4096)
    assert np.array_equal(r["cont"], want) and np.array_equal(r["y"], x)
    h = oracle.histogram(x)
    code_only = 1 - oracle.code_bits(h, oracle.scheme(1)) / (8 * x.size)
    container = 1 - r["cont"].size / x.size
    assert abs(code_only - container) < 0.001           # index overhead < 0.1 pp


@pytest.mark.parametrize("kind", ["ffn2", "t4"])
def test_searched_scheme_on_gpu_matches_oracle(qlc, kind):
    """A scheme from the exhaustive search (not one of the printed tables)
    codes bit-exactly on the GPU: histogram, LUT, container and decode."""
    x = inputs.make_e4m3(kind, 3 * 32 * 1024 + 555, seed=21).numpy()
    h = oracle.histogram(x)
    sc, _ = qlc.qlc_scheme_search(h)
    area = (np.array(list(sc.area_n), np.uint16), np.array(list(sc.area_bits), np.uint8))
    r = _gpu_pipeline(qlc, x, sc, 1024)
    want = oracle.encode(x, scheme_id=int(sc.id), area=area, chunk_symbols=1024)
    assert np.array_equal(r["cont"], want)
    assert np.array_equal(r["y"], x)
