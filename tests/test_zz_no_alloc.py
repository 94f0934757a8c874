"""sc_trace_noalloc: the trace for callers that cannot allocate device
memory (a host whose own allocator owns the GPU heap, where an extra
cudaMalloc fails or synchronizes the device).  Its scratch is a static
device array inside the library instead of a caller workspace.

Checked through the C-ABI against sc_trace with a caller workspace on the
same inputs, on two calls in a row (the shared scratch must be cleared by
each call): hit ids and per-ray test counts exact, t within the 1e-6
relative tolerance of the other GPU tests; and the device's free memory does
not drop over the second call.  This file is collected last so
that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _split(hits, counts):
    t, i, u, v = sc.split_hits(hits)
    return t.copy(), i.copy(), counts.cpu().numpy().view(np.uint32).copy()


@pytest.mark.parametrize("cull", [1, 0])
def test_noalloc_matches_workspace_trace_twice(cull):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    tris = sg.hair(512, 16, True, seed=21)
    rays = sg.pinhole(96, 64)
    b = sc.sc_bvh_build(tris, 6, 1)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    r = torch.from_numpy(rays).cuda()
    n = r.shape[0]
    ref_hits, ref_counts = sc.trace(d, r, sc.SC_CLOSEST, cull)
    torch.cuda.synchronize()
    rt, ri, rc = _split(ref_hits, ref_counts)
    bufs = [(torch.full((n, 4), -7.0, dtype=torch.float32, device="cuda"),
             torch.full((n, 2), -7, dtype=torch.int32, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):
        hits, counts = bufs[call]
        free0 = torch.cuda.mem_get_info()[0]
        sc.sc_trace_noalloc(d, r, hits, counts, sc.SC_CLOSEST, cull)
        if call == 1:
            # the first call may load the module and look up the array;
            # after it, a call takes no device memory at all
            assert torch.cuda.mem_get_info()[0] >= free0, "the second call allocated"
        t, i, c = _split(hits, counts)
        assert np.array_equal(i, ri), f"call {call}: hit ids differ"
        assert np.array_equal(c, rc), f"call {call}: per-ray counts differ"
        hit = ri >= 0
        rel = np.abs(t[hit] - rt[hit]) / np.maximum(np.abs(rt[hit]), 1e-30)
        assert (rel <= 1e-6).all() and np.array_equal(np.isinf(t), np.isinf(rt))


def test_noalloc_refuses_stream_capture():
    """A call on a capturing stream returns SC_ERR_STATE before it enqueues
    anything; the capture stays valid and replays the rest of its work."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    tris = sg.hair(64, 16, True, seed=22)
    rays = sg.pinhole(16, 16)
    b = sc.sc_bvh_build(tris, 6, 1)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    r = torch.from_numpy(rays).cuda()
    n = r.shape[0]
    hits = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    counts = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
    # an uncaptured call first, so the capture below sees no first-call setup
    sc.sc_trace_noalloc(d, r, hits, counts, sc.SC_CLOSEST, 1)
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            with pytest.raises(sc.SubcullError, match="cannot be captured"):
                sc.sc_trace_noalloc(d, r, hits, counts, sc.SC_CLOSEST, 1)
            x.add_(1.0)
    g.replay()
    torch.cuda.synchronize()
    assert x.tolist() == [1.0, 1.0, 1.0, 1.0]
