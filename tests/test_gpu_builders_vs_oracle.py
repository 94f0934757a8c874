"""The GPU tree and mask builders (sc_build_opts.gpu_bvh, gpu_masks) against
the oracle's own build directly: root slot, child indices, leaf ranges,
child boxes, triangle order, every slot's object mask, and (compressed) the
compression LUT and every slot's LUT index, element by element.  At the
65,536- and 1,048,578-triangle hair scenes of the benchmark (R = 6, L = 3)
and a triangle soup with flat slabs, uncompressed and compressed.  Boxes are
compared as floats (the GPU build may give a zero bound the other sign)."""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCENES = {
    "hair65k": lambda: sg.hair(2048, 16, False, seed=1),
    "hair1m": lambda: sg.hair(32768, 16, True, seed=2),
    "soup64k": lambda: sg.soup(1 << 16, seed=3),
}


@pytest.mark.parametrize("comp", [0, 1])
@pytest.mark.parametrize("scene", sorted(SCENES))
def test_gpu_build_equals_oracle_build(scene, comp):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    tris = SCENES[scene]()
    ex = sc.sc_bvh_build(tris, 6, comp, gpu_bvh=1, gpu_masks=1).export()
    ob = oracle.OracleBVH(tris).build_masks(6, 3)
    if comp:
        ob.compress(256, 8)
    child, count, box = ob.nodes()
    rc, rn, _ = ob.root()
    assert ex["root"].tolist() == [rc, rn]
    assert np.array_equal(ex["child"], child)
    assert np.array_equal(ex["count"], count)
    assert np.array_equal(ex["box"], box)  # float equality: -0 == +0
    assert np.array_equal(ex["perm"], ob.perm())
    assert np.array_equal(ex["masks"], ob.masks())
    if comp:
        clut, cidx = ob.clut()
        assert np.array_equal(ex["clut"], clut)
        assert np.array_equal(ex["cidx"], cidx)
