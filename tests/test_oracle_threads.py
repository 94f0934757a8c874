"""The oracle's threaded build (independent subtrees of the tree, the slots
of one depth level of the masks, the slots' LUT encodings) gives exactly the
serial build's tree, masks, compression LUT and indices, whatever the
thread count and subtree task size."""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg


def _build(tris, threads, task, comp):
    oracle.set_threads(threads, task)
    try:
        ob = oracle.OracleBVH(tris).build_masks(6, 3)
        if comp:
            ob.compress(256, 8)
        c, n, b = ob.nodes()
        out = dict(child=c, count=n, box=b, perm=ob.perm(), masks=ob.masks(),
                   root=ob.root(), depth=ob.max_depth)
        if comp:
            out["clut"], out["cidx"] = ob.clut()
        return out
    finally:
        oracle.set_threads(0, 0)


@pytest.mark.parametrize("threads,task", [(2, 4096), (3, 5000), (8, 0)])
def test_threaded_build_equals_serial(threads, task):
    tris = np.concatenate([sg.hair(700, 16, True, seed=51), sg.soup(6000, seed=52)])
    a = _build(tris, 1, 0, True)
    b = _build(tris, threads, task, True)
    for k in ("child", "count", "box", "perm", "masks", "clut", "cidx"):
        assert np.array_equal(a[k], b[k]), k
    assert a["root"][0] == b["root"][0] and a["root"][1] == b["root"][1]
    assert np.array_equal(a["root"][2], b["root"][2]) and a["depth"] == b["depth"]


def test_threaded_build_small_and_root_task():
    # a scene whose whole range is one subtree task, and one of a single leaf
    for tris in (sg.hair(200, 16, False, seed=53), sg.hair(2, 1, False, seed=54)):
        a = _build(tris, 1, 0, False)
        b = _build(tris, 4, 1 << 20, False)
        for k in ("child", "count", "box", "perm", "masks"):
            assert np.array_equal(a[k], b[k]), k
        assert a["root"][:2] == b["root"][:2]
