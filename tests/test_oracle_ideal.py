"""Ideal culling (Sec. 4.1's reference): the ray mask is the exact set of
cells the clipped segment meets (a double-precision cell walk) instead of
the lookup table's sweep of the entry and exit cells.  It must keep every
hit, and -- the segment lying inside the sweep -- cull at least as much as
the table with the same object masks."""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg


def _tests(o):
    return o["counts"].astype(np.int64).sum()


@pytest.mark.parametrize("R", [4, 6])
def test_ideal_culling_bounds_the_lookup_table(hair_small, R):
    tris, rays = hair_small
    plain = oracle.OracleBVH(tris).trace(rays, 0, 0)
    l3 = oracle.OracleBVH(tris).build_masks(R, 3)
    linf = oracle.OracleBVH(tris).build_masks(R, 64)
    lut3, lutinf = l3.trace(rays, 0, 1), linf.trace(rays, 0, 1)
    ideal = linf.set_ideal().trace(rays, 0, 1)
    for o in (lut3, lutinf, ideal):
        assert np.array_equal(o["id"], plain["id"]) and np.array_equal(o["t"], plain["t"])
    assert _tests(ideal) <= _tests(lutinf) <= _tests(lut3) <= _tests(plain)
    # the exact mask never needs more work than the table on any ray here
    assert (ideal["counts"] <= lutinf["counts"]).all()


def test_ideal_mask_keeps_axis_parallel_hits():
    # rays along a box axis meet a single row of cells: the exact mask must
    # still keep the leaf whose triangle they hit
    tri = np.array([[0, 0, 0, 1, 0, 0, 0, 0.1, 0]], np.float32)
    other = np.array([[0, 0.9, 0, 1, 0.9, 0, 1, 1, 0]], np.float32)
    tris = np.concatenate([tri, other, tri + np.float32(5), other + np.float32(5)])
    ob = oracle.OracleBVH(tris, max_leaf=1).build_masks(4, 64).set_ideal()
    r_hit = np.array([[-1, 0.05, 0.0, 0, 1, 0, 0, np.inf]], np.float32)
    o = ob.trace(r_hit, 0, 1)
    b = oracle.brute(tris, r_hit, 0)
    assert o["id"][0] == b[1][0]
