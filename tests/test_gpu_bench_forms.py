"""The bench's CUDA-graph forms run on the stream the bench times them on.

`bench.py` measures its forms on the current stream of the process, which is
the default stream; a CUDA graph cannot be captured there, so each form
captures on a side stream and replays on the timed one.  These run the
adjoint gradient form (a graph captured with torch around the library's
calls) and the small-workload form (a graph captured by the library itself)
exactly as the bench calls them, and check that they report times and that
the replayed gradient has the bits of the gradient issued call by call.
"""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
cpb = pytest.importorskip("paper_2206_07896_gb300")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_adjoint_form_graph_on_the_default_stream(bench):
    L = cpb.lib(fma=True)
    r = bench.form_adjoint(L, cpb, torch.device("cuda:0"), torch.cuda.current_stream())
    assert "error" not in r, r
    assert r["gradient"]["ms"] > 0 and r["forward"]["ms"] > 0
    assert r["gradient_cuda_graph"]["same_bits_as_eager"]
    assert 0 < r["gradient_cuda_graph"]["ms"] <= 1.5 * r["gradient"]["ms"]


def test_small_form_on_the_default_stream(bench):
    L = cpb.lib(fma=True)
    r = bench.form_small(L, cpb, torch.device("cuda:0"), torch.cuda.current_stream())
    assert "error" not in r, r
    assert r["tuned_cuda_graph"]["ms"] > 0 and r["tuned"]["ms"] > 0
