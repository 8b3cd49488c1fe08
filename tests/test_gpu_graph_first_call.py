"""A CUDA graph can be captured around the library's very first calls in a
process: the histogram kernels' one-time shared-memory setting (a function
attribute, not stream work) is legal inside stream capture.  Runs in a fresh
interpreter so that no earlier call has made the setting."""
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

SCRIPT = textwrap.dedent("""
    import numpy as np, torch, sys
    sys.path.insert(0, ".")
    import oracle
    from paper_2602_17849_gb300 import inputs, qlc
    dev = torch.device("cuda")
    x = inputs.make_e4m3("t4", 1 << 20, seed=5, device=dev)
    hist = torch.zeros(256, dtype=torch.int64, device=dev)
    shards = [inputs.make_e4m3("gauss", 50_000, seed=6, device=dev)]
    hists = torch.zeros(256, dtype=torch.int64, device=dev)
    ws = torch.zeros(qlc.qlc_batch_workspace_size(1, 50_000, 1024), dtype=torch.uint8, device=dev)
    descs = qlc.descs_tensor([(shards[0].data_ptr(), 50_000, 0, 0, 0, 0)], dev)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):
        qlc.qlc_histogram(x, hist, stream=s)
        qlc.qlc_histogram_batch(descs, 1, hists, False, ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), oracle.histogram(x.cpu().numpy()))
    assert np.array_equal(hists.cpu().numpy().astype(np.uint64), oracle.histogram(shards[0].cpu().numpy()))
    print("ok")
""")


def test_first_calls_inside_graph_capture():
    from paper_2602_17849_gb300 import _build
    _build.build()
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-2000:]
