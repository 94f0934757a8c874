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
