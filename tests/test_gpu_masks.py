"""Object masks built on the GPU (sc_build_opts.gpu_masks) are bit-identical
to the host build -- which test_host_vs_oracle.py ties to the oracle --
for every grid resolution, several L (including L deeper than the tree),
flat boxes (the ground quad, axis-aligned soup slabs) and compression."""
import numpy as np
import pytest

from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


SCENES = {
    "hair_ground": lambda: sg.hair(512, 16, True, seed=3),
    "soup": lambda: sg.soup(20000, seed=8),
}


@pytest.mark.parametrize("scene", sorted(SCENES))
@pytest.mark.parametrize("R,L", [(4, 1), (6, 3), (8, 3), (6, 6), (4, 80)])
def test_gpu_masks_equal_host(scene, R, L):
    _need_gpu()
    tris = SCENES[scene]()
    host = sc.sc_bvh_build(tris, R, 0, L=L).export()
    dev = sc.sc_bvh_build(tris, R, 0, L=L, gpu_masks=1).export()
    for k in ("child", "count", "box", "perm", "masks"):
        assert np.array_equal(host[k], dev[k]), k


def test_gpu_masks_compressed_and_timing_fields():
    _need_gpu()
    tris = sg.hair(2048, 16, True, seed=9)
    a = sc.sc_bvh_build(tris, 6, 1)
    b = sc.sc_bvh_build(tris, 6, 1, gpu_masks=1)
    ea, eb = a.export(), b.export()
    for k in ("masks", "clut", "cidx"):
        assert np.array_equal(ea[k], eb[k]), k
    assert b.info().ms_masks > 0.0


@pytest.mark.parametrize("comp", [0, 1])
def test_gpu_refit_equals_host_refit_and_traces_like_the_oracle(comp):
    """sc_bvh_refit on a BVH built with gpu_masks recomputes the dirty slots'
    masks on the GPU: the same bits as the host refit.  The refit image,
    uploaded again, traces like the oracle's refit BVH (ids, t, counts)."""
    _need_gpu()
    import oracle
    tris = sg.hair(1024, 16, True, seed=13)
    moved = tris.copy()
    moved[32 * 200:32 * 203] += np.float32(0.02)  # three strands
    host = sc.sc_bvh_build(tris, 6, comp)
    dev = sc.sc_bvh_build(tris, 6, comp, gpu_masks=1)
    ih, idv = sc.sc_bvh_refit(host, moved), sc.sc_bvh_refit(dev, moved)
    assert ih.dirty_nodes == idv.dirty_nodes and 0 < idv.dirty_nodes
    eh, ed = host.export(), dev.export()
    for k in eh:
        assert np.array_equal(eh[k], ed[k]), k
    ob = oracle.OracleBVH(tris).build_masks(6, 3)
    if comp:
        ob.compress(256, 8)
    ob.refit(moved).build_masks(6, 3)
    if comp:
        ob.reencode()
    rays = sg.pinhole(96, 64)
    o = ob.trace(rays, 0, 2 if comp else 1)
    d = sc.DeviceBVH(dev, sc.SC_LAYOUT_MASKED)
    hits, counts = sc.trace(d, torch.from_numpy(rays).cuda(), sc.SC_CLOSEST, 1)
    torch.cuda.synchronize()
    h = hits.cpu().numpy()
    assert np.array_equal(h[:, 1].view(np.int32), o["id"])
    assert np.array_equal(h[:, 0].view(np.int32), o["t"].view(np.int32))
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), o["counts"])
